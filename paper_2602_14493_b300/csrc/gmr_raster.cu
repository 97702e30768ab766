// Tile binning and front-to-back alpha compositing (Sec. 2.1, standard 3DGS
// rasterization), forward and backward.
//
// Forward, per pixel, over the Gaussians listed for its tile in (depth, face)
// order: alpha = min(0.99, o * G) with G = exp(-1/2 d^T Q d); Gaussians with
// alpha < 1/255 are skipped; the pixel stops before the Gaussian that would
// take its transmittance T below 1e-4; otherwise C += c alpha T and
// T *= 1 - alpha. I = C + T bg. The final T and the list position of the last
// contributor are kept per pixel.
//
// Backward, per pixel, walks the same list from the last contributor to the
// front, recovering T_i = T_(i+1) / (1 - alpha_i) from the stored final T
// (no per-pixel lists are stored), with S the colour composited behind
// Gaussian i (plus T_final bg):
//   dL/dc_i     = alpha_i T_i g
//   dL/dalpha_i = T_i (c_i . g) - (S . g) / (1 - alpha_i)
// and alpha = o 2^(a2 dx^2 + b2 dx dy + c2 dy^2) gives the mean, conic and
// opacity terms. With q = alpha dL/dalpha, each record collects the moments
// (sum q dx, sum q dy, sum q dx^2, sum q dx dy, sum q dy^2) and the face
// sum q and sum alpha T g; the record backward turns the first two into the
// mean gradient with the conic. A warp reduces its 32 pixels' contributions
// to one Gaussian with a transposed butterfly (9 values in 14 shuffles) and
// eight lanes then issue one atomic add each; when at most 20 lanes
// contribute, those lanes add their own values instead, with three atomic
// adds each (two of them 16-byte vectors): together 11-19% faster than
// always reducing on a 20K-face mesh in 8 views of 512^2, 25-35% on meshes
// whose Gaussians cover a pixel or two.
//
// Layout: one CTA per screen tile of one view (all views of a batched call in
// one launch; the tile id selects the view), CTAs taking the tiles heaviest
// first (pair-count classes set by the binning: fewer SMs idle at the end of
// the launch). The tile is cut into 8x4 pixel
// blocks; each warp owns a rectangle of 1, 2 or 4 blocks (8x4, 8x8 or 16x8
// pixels, one pixel per lane in each block), so a thread composites 1, 2 or
// 4 pixels. Each batch of listed Gaussians is staged in shared memory
// (float4 loads of the records and face colours), with the image mean made
// relative to the pixel block's 32-aligned anchor in float-pair arithmetic.

#include <algorithm>
#include <map>
#include <mutex>

#include "gmr_internal.cuh"

namespace gmr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Pixel layout of a tile of TS x TS pixels served by NT threads: the tile is
// cut into 8x4-pixel blocks (row-major, TS/8 per row). Each warp owns a
// rectangle of PPT blocks, RW blocks wide and PPT/RW high (1 block, 8x8 or
// 16x8 pixels: the squarest region, so that a Gaussian's footprint meets as
// few warps as possible), and lane l the pixel (l % 8, l / 8) of each block.
template <int TS, int NT>
struct PixMap {
  static constexpr int PPT = TS * TS / NT;  // pixels per thread
  static_assert(PPT >= 1 && PPT * NT == TS * TS, "bad tile / thread split");
  static constexpr int NC = TS / 8;          // blocks per tile row
  static constexpr int RW = PPT >= 4 ? 2 : 1;  // region width in blocks
  static constexpr int RH = PPT / RW;          // region height in blocks
  static_assert(NC % RW == 0 && (TS / 4) % RH == 0, "bad warp region");
  static constexpr int RX = NC / RW;           // regions per tile row
  __device__ __forceinline__ static int block_of(int warp, int k) {
    const int rx = warp % RX, ry = warp / RX;
    return (ry * RH + k / RW) * NC + rx * RW + k % RW;
  }
  __device__ __forceinline__ static int block(int k) { return block_of(threadIdx.x >> 5, k); }

  __device__ __forceinline__ static uint32_t warp_bits_of(int warp) {
    uint32_t b = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) b |= 1u << block_of(warp, k);
    return b;
  }
  __device__ __forceinline__ static uint32_t warp_bits() { return warp_bits_of(threadIdx.x >> 5); }
  __device__ __forceinline__ static void local(int k, int& lx, int& ly) {
    int lane = threadIdx.x & 31, b = block(k);
    lx = (b % NC) * 8 + (lane & 7);
    ly = (b / NC) * 4 + (lane >> 3);
  }
  // The warp's rectangle of pixel centres, [x0, x1] x [y0, y1], relative to
  // the anchor (the tile's offset from it is (tox, toy)).
  __device__ __forceinline__ static void region(float tox, float toy, float& x0, float& x1, float& y0, float& y1) {
    const int b0 = block(0), bc = b0 % NC, br = b0 / NC;
    x0 = tox + (float)(8 * bc) + 0.5f;
    x1 = tox + (float)(8 * (bc + RW)) - 0.5f;
    y0 = toy + (float)(4 * br) + 0.5f;
    y1 = toy + (float)(4 * (br + RH)) - 0.5f;
  }
};

// ---------------------------------------------------------------- staging
template <int BATCH, int NW>
struct Stage {
  float4 g[BATCH];    // (ux, uy, a2, b2), mean relative to the anchor
  float4 h[BATCH];    // (c2, t2 = log2(1/(255 o)), o, 0)
  float4 col[BATCH];  // (r, g, b, 0)
  uint32_t mask[BATCH];  // 8x4 pixel blocks of the tile the Gaussian can reach
  uint32_t rid[BATCH];
  uint32_t face[BATCH];
  uint8_t list[NW][BATCH];  // per warp: batch indices that reach its blocks, in order
};

// Each warp compacts, in order, the batch entries whose mask reaches one of
// its blocks (`bits`) and whose list position is below `limit`. Returns the
// count (warp-uniform).
template <int BATCH, int NW>
__device__ __forceinline__ int warp_list(Stage<BATCH, NW>& st, int count, int first_pos, int limit, uint32_t bits) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  int n = 0;
  for (int c = 0; c < count; c += 32) {
    int i = c + lane;
    bool rel = i < count && (st.mask[i] & bits) && (first_pos + i) < limit;
    uint32_t bal = __ballot_sync(0xffffffffu, rel);
    if (rel) st.list[warp][n + __popc(bal & lt)] = (uint8_t)i;
    n += __popc(bal);
  }
  __syncwarp();
  return n;
}

// Bit mask of the tile's blocks of BW x BH pixels (NCB per row, NRB rows)
// that the Gaussian's region alpha >= 1/255 can reach. In log2 units that
// region is
// A dx^2 + B dx dy + C dy^2 <= log2(255 o) with (A, B, C) = -(a2, b2, c2);
// its bounding box has half-widths sqrt(k C / (AC - B^2/4)) and
// sqrt(k A / (AC - B^2/4)). The box is widened (k by 1e-4 relative, 1e-3 px)
// so that every skipped Gaussian has alpha below 1/255 by a margin (at least
// 1e-4 in log2 units) far above
// the rounding of the alpha evaluation: culling never changes a result.
template <int NCB, int NRB, int BW, int BH>
__device__ __forceinline__ uint32_t region_mask(float gx, float gy, float a2, float b2, float c2, float k2, float tox,
                                                float toy) {
  static_assert(NCB * NRB <= 32, "one bit per block");
  const float A = -a2, B = -b2, Cq = -c2;
  const float det = A * Cq - 0.25f * B * B;
  if (!(k2 > 0.0f) || !(det > 0.0f)) return 0u;  // k2 = log2(255 o)
  const float kk = (k2 * 1.0001f + 1e-4f) / det;
  const float hx = sqrtf(kk * Cq) + 1e-3f, hy = sqrtf(kk * A) + 1e-3f;
  uint32_t cols = 0;
#pragma unroll
  for (int c = 0; c < NCB; ++c) {
    float lo = tox + (float)(BW * c) + 0.5f;
    if (gx + hx >= lo && gx - hx <= lo + (float)(BW - 1)) cols |= 1u << c;
  }
  uint32_t m = 0;
#pragma unroll
  for (int r = 0; r < NRB; ++r) {
    float lo = toy + (float)(BH * r) + 0.5f;
    if (gy + hy >= lo && gy - hy <= lo + (float)(BH - 1)) m |= cols << (r * NCB);
  }
  return m;
}

// The tile's 8x4-pixel warp blocks (row-major, TS/8 per row)...
template <int TS>
__device__ __forceinline__ uint32_t block_mask(float gx, float gy, float a2, float b2, float c2, float k2, float tox,
                                               float toy) {
  return region_mask<TS / 8, TS / 4, 8, 4>(gx, gy, a2, b2, c2, k2, tox, toy);
}

// ... and the 4x4-pixel half-warp units of the tile (row-major, TS/4 per
// row), for the half-warp layout.
template <int TS>
__device__ __forceinline__ uint32_t unit_mask(float gx, float gy, float a2, float b2, float c2, float k2, float tox,
                                              float toy) {
  return region_mask<TS / 4, TS / 4, 4, 4>(gx, gy, a2, b2, c2, k2, tox, toy);
}

// Staging of one batch: records and colours of the listed Gaussians, the
// mean relative to the anchor, and the block mask (the conservative
// bounding-box test above). The record's w holds the skip threshold
// t2 = -log2(255 o).
template <int TS, int NT, int BATCH, int NL = NT / 32>
__device__ __forceinline__ void stage_batch(Stage<BATCH, NL>& st, const uint32_t* __restrict__ pair_face, uint32_t lo,
                                            int count, uint32_t rec_base, const float4* __restrict__ rec_uq,
                                            const float4* __restrict__ col_src,
                                            bool col_by_rec, float ax, float ay, float tox, float toy,
                                            bool want_ids, bool units = false) {
  for (int i = threadIdx.x; i < count; i += NT) {
    uint32_t f = __ldg(pair_face + lo + i);
    uint32_t rid = rec_base + f;
    float4 u = __ldg(rec_uq + 2 * (size_t)rid);
    float4 q = __ldg(rec_uq + 2 * (size_t)rid + 1);
    float4 col = __ldg(col_src + (col_by_rec ? rid : f));
    float ux = __fadd_rn(__fsub_rn(u.x, ax), u.z);
    float uy = __fadd_rn(__fsub_rn(u.y, ay), u.w);
    const uint32_t m = units ? unit_mask<(TS <= 16 ? TS : 16)>(ux, uy, q.x, q.y, q.z, -q.w, tox, toy)  // (no units at 32)
                             : block_mask<TS>(ux, uy, q.x, q.y, q.z, -q.w, tox, toy);
    st.g[i] = make_float4(ux, uy, q.x, q.y);
    st.h[i] = make_float4(q.z, q.w, col.w, 0.0f);
    st.mask[i] = m;
    st.col[i] = make_float4(col.x, col.y, col.z, 0.0f);
    if (want_ids) {
      st.rid[i] = rid;
      st.face[i] = f;
    }
  }
}

// ---------------------------------------------------------------- forward
// Resident CTAs per SM that the register allocation must allow, per launch
// shape (0: the compiler's choice). Measured on the 8 x 512^2 ring workload:
// one pixel per thread runs best at 40 resident warps (<= 51 registers);
// the other shapes and the backward run best uncapped.
template <int TS, int NT>
struct FwdMinBlocks {
  static constexpr int value = (TS == 16 && NT == 256) ? 5 : 0;
};

// Block sum of one FP32 value per thread: a warp tree in FP32, then the
// warps' sums added in FP64 by thread 0 (FP64 is a slow pipe on this GPU:
// a full-warp FP64 tree per block costs more than the rest of a loss pass).
// Relative error at most (5 + depth of the per-thread sums) u, u = 2^-24.
template <int NT>
__device__ __forceinline__ double block_sum_f32(float v, float* sw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += (double)sw[w];
  return s;  // valid in thread 0
}

// Block sum of one FP64 value per thread (FP64 warp tree).
template <int NT>
__device__ __forceinline__ double block_sum_f64(double v, double* sw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += sw[w];
  return s;  // valid in thread 0
}

// The block's sum bs (valid in thread 0) written to part[1 + blockIdx.x];
// the block that finishes last (ticket counter in part[0]) adds the partials
// in index order into *loss and returns the counter to zero. Called by every
// thread of every block of the grid.
template <int NT>
__device__ __forceinline__ void finish_loss_partial(double bs, double* __restrict__ part,
                                                    double* __restrict__ loss) {
  __shared__ double sw[NT / 32];
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    part[1 + blockIdx.x] = bs;
    __threadfence();
    s_last = atomicAdd(reinterpret_cast<unsigned int*>(part), 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += NT) acc += __ldcg(part + 1 + i);
  __syncthreads();
  const double tot = block_sum_f64<NT>(acc, sw);
  if (threadIdx.x == 0) {
    *loss = tot;
    *reinterpret_cast<unsigned int*>(part) = 0u;
  }
}

template <int NT>
__device__ __forceinline__ void loss_partial_and_finish(float v, double* __restrict__ part,
                                                        double* __restrict__ loss) {
  __shared__ float swf[NT / 32];
  finish_loss_partial<NT>(block_sum_f32<NT>(v, swf), part, loss);
}

// MODE: kFwdPlain; kFwdDebug also records per-pixel contributor counts and
// order hashes (tests); kFwdLoss also computes the squared-error loss
// against fl.target in the epilogue.
constexpr int kFwdPlain = 0, kFwdDebug = 1, kFwdLoss = 2;

// Compositing layouts (see the kernels).
constexpr int kLayoutCta = 0, kLayoutHalf = 1, kLayoutWarp = 2;

// Per-tile arguments of the compositing kernels.
struct RasterArgs {
  const uint32_t* pair_face;
  const float4* rec_uq;  // 32-byte records: [2 r] image mean, [2 r + 1] conic and threshold
  const float4* col;  // (r, g, b, o) per face, or per record when col_by_rec
  int col_by_rec;     // view-dependent colour: colours and their gradients per record
  const ViewInfo* views;
  int32_t F;
  float bg0, bg1, bg2;
  const uint4* tile_desc;
  Counters* counters;
  uint32_t n_pos;   // compositing positions (tiles)
  // deterministic backward: per pair slot its sums (3 float4), the records'
  // tile rectangles and first slots, the slot capacity
  float4* pair_grad;
  const uint2* rec_rect;
  const uint32_t* rec_slot;
  int64_t cap_slots;
};

// The next compositing position of a persistent grid's CTA: one atomic on
// the cursor per tile, broadcast through shared memory (the first barrier
// waits until every thread is done with the last tile and with s_pos).
// Returns false when no position is left.
__device__ __forceinline__ bool next_position(uint32_t* cursor, uint32_t n_pos, uint32_t& pos) {
  __shared__ uint32_t s_pos;
  __syncthreads();
  if (threadIdx.x == 0) s_pos = atomicAdd(cursor, 1u);
  __syncthreads();
  pos = s_pos;
  return pos < n_pos;
}

// One tile of the forward at compositing position pos: image, final T and
// last contributor of every pixel.
template <int TS, int NT, int BATCH, int MODE>
__device__ __forceinline__ void fwd_tile(const RasterArgs& a, uint32_t pos, float* __restrict__ images,
                                         float* __restrict__ pix_T, uint32_t* __restrict__ pix_last,
                                         float* __restrict__ t_out, uint32_t* __restrict__ nc_out,
                                         int64_t n_pix_total, const FwdLoss& fl) {
  constexpr int PPT = PixMap<TS, NT>::PPT;
  constexpr int NW = NT / 32;
  __shared__ Stage<BATCH, NW> st;
  // the tile at this compositing position, its view and its pair range
  const uint4 desc = __ldg(a.tile_desc + pos);
  if (desc.x == kNoTile) return;  // a quadrant beyond the image (split binning)
  const int g = (int)desc.x;
  const int c = (int)desc.y;
  const ViewInfo& v = a.views[c];
  const int lt = g - v.tile_base;
  const int tyi = lt / v.tiles_x, txi = lt - tyi * v.tiles_x;
  const int ox = txi * TS, oy = tyi * TS;
  const int axi = ox & ~31, ayi = oy & ~31;
  const float ax = (float)axi, ay = (float)ayi;
  const float tox = (float)(ox - axi), toy = (float)(oy - ayi);
  const int lane = threadIdx.x & 31;

  float pcx[PPT], pcy[PPT], T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
  // fused loss: each thread's target pixels, copied to shared memory
  // asynchronously at the start and read in the epilogue
  __shared__ float s_tgt[MODE == kFwdLoss ? 3 * PPT * NT : 1];
  uint32_t last[PPT], term[PPT], ncontrib[PPT], chash[PPT];
  bool done[PPT], inside[PPT];
  int px[PPT], py[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int lx, ly;
    PixMap<TS, NT>::local(k, lx, ly);
    px[k] = ox + lx;
    py[k] = oy + ly;
    pcx[k] = (float)(px[k] - axi) + 0.5f;
    pcy[k] = (float)(py[k] - ayi) + 0.5f;
    inside[k] = px[k] < v.W && py[k] < v.H;
    done[k] = !inside[k];
    T[k] = 1.0f;
    Cr[k] = Cg[k] = Cb[k] = 0.0f;
    last[k] = 0;
    term[k] = 0;
    ncontrib[k] = 0;
    chash[k] = 0;
    if (MODE == kFwdLoss && inside[k]) {
      const float* tp = fl.target + 3 * (v.pix_base + (int64_t)py[k] * v.W + px[k]);
      const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&s_tgt[3 * (k * NT + threadIdx.x)]);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + 4u * q), "l"(tp + q) : "memory");
    }
  }
  if (MODE == kFwdLoss) asm volatile("cp.async.commit_group;" ::: "memory");
  const uint2 range = make_uint2(desc.z, desc.w);
  const int n = (int)(range.y - range.x);
  const uint32_t rec_base = (uint32_t)c * (uint32_t)a.F;

  for (int base = 0; base < n; base += BATCH) {
    bool tdone = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) tdone &= done[k];
    if (__syncthreads_and(tdone)) break;
    int cnt = min(BATCH, n - base);
    stage_batch<TS, NT, BATCH>(st, a.pair_face, range.x + base, cnt, rec_base, a.rec_uq, a.col,
                               a.col_by_rec != 0, ax, ay, tox, toy, MODE == kFwdDebug);
    __syncthreads();
    const int nl = warp_list<BATCH, NW>(st, cnt, 0, cnt, PixMap<TS, NT>::warp_bits());
    const int warp = threadIdx.x >> 5;
    for (int jj = 0; jj < nl; ++jj) {
      if ((jj & 3) == 0) {  // the warp's early exit, checked every 4 entries
        bool wd = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) wd &= done[k];
        if (__all_sync(kFull, wd)) break;
      }
      const int j = st.list[warp][jj];
      const float4 hh = st.h[j];
      const float4 gg = st.g[j];
      float p2[PPT];
      bool con[PPT];
      bool anyc = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        float dx, dy;
        p2[k] = gauss_p2(gg, hh.x, pcx[k], pcy[k], dx, dy);
        // (a pixel of a block outside the Gaussian's block mask fails the
        // alpha test by construction of the mask: no block test here)
        con[k] = !done[k] && !(p2[k] < hh.y);
        anyc |= con[k];
      }
      if (!anyc) continue;
      {
        const float4 col = st.col[j];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (!con[k]) continue;
          float graw;
          float alpha = gauss_alpha(p2[k], hh.z, graw);
          float test = __fmul_rn(T[k], __fsub_rn(1.0f, alpha));
          if (test < kTMin) {
            done[k] = true;
            term[k] = (uint32_t)(base + j + 1);
            continue;
          }
          float w = __fmul_rn(alpha, T[k]);
          Cr[k] = __fmaf_rn(col.x, w, Cr[k]);
          Cg[k] = __fmaf_rn(col.y, w, Cg[k]);
          Cb[k] = __fmaf_rn(col.z, w, Cb[k]);
          T[k] = test;
          last[k] = (uint32_t)(base + j + 1);
          ++ncontrib[k];
          if (MODE == kFwdDebug) chash[k] = chash[k] * 0x9E3779B1u + st.face[j] + 1u;  // ordered contributor list
        }
      }
    }
  }
  unsigned long long evals = 0, ncon = 0;
  float lsum = 0.0f;  // fused loss: FP32 over this thread's pixels
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!inside[k]) continue;
    ncon += ncontrib[k];
    int64_t pid = v.pix_base + (int64_t)py[k] * v.W + px[k];
    const float i0 = Cr[k] + T[k] * a.bg0, i1 = Cg[k] + T[k] * a.bg1, i2 = Cb[k] + T[k] * a.bg2;
    images[3 * pid] = i0;
    images[3 * pid + 1] = i1;
    images[3 * pid + 2] = i2;
    if (MODE == kFwdLoss) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      const float* tg = &s_tgt[3 * (k * NT + threadIdx.x)];
      const float d0 = i0 - tg[0], d1 = i1 - tg[1], d2 = i2 - tg[2];
      fl.grad[3 * pid] = 2.0f * d0;
      fl.grad[3 * pid + 1] = 2.0f * d1;
      fl.grad[3 * pid + 2] = 2.0f * d2;
      lsum = fmaf(d0, d0, lsum);
      lsum = fmaf(d1, d1, lsum);
      lsum = fmaf(d2, d2, lsum);
    }
    pix_T[pid] = T[k];
    pix_last[pid] = last[k];
    if (t_out) t_out[pid] = T[k];
    if (MODE == kFwdDebug) {
      nc_out[pid] = ncontrib[k];
      nc_out[n_pix_total + pid] = chash[k];
    }
    evals += term[k] ? term[k] : (uint32_t)n;
  }
  if (MODE == kFwdLoss) asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(kFull, evals, o);
    ncon += __shfl_xor_sync(kFull, ncon, o);
  }
  if (lane == 0 && evals) atomicAdd(&a.counters->evals_fwd, evals);
  if (lane == 0 && ncon) atomicAdd(&a.counters->contribs, ncon);
  if (MODE == kFwdLoss) {  // one FP32 partial per warp, no block barrier
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if (lane == 0) fl.part[(int64_t)g * NW + (threadIdx.x >> 5)] = lsum;
  }
}

// ---------------------------------------------------------------- half-warp layout
// Layout for Gaussians that cover few pixels: a TS x TS tile is cut into
// units of 4x4 pixels (row-major, U = TS/4 per row), and each 16-lane half
// of a warp composites PPT units (one pixel of each per lane) and walks its
// own compacted list of the batch's Gaussians that can reach them. The two
// halves of a warp step through their lists together, each on its own
// entry, so a warp-step serves two Gaussians where the full-warp layout
// serves one when the Gaussians are smaller than a warp block (the lists of
// a 4x4 unit are shorter than those of an 8x4 block). 16x16 tiles with 128
// or 256 threads, 8x8 tiles with 32 or 64.
template <int TS, int NT>
struct HalfMap {
  static constexpr int U = TS / 4;             // units per tile row
  static constexpr int PPT = TS * TS / NT;      // units per half = pixels per lane
  static_assert((TS == 16 || TS == 8) && (PPT == 1 || PPT == 2), "half-warp layout: 1 or 2 units per half");
  // half h owns the units in column h % U, rows (h / U) PPT + k
  __device__ __forceinline__ static int unit_of(int h, int k) { return ((h / U) * PPT + k) * U + (h % U); }
  __device__ __forceinline__ static int half() { return threadIdx.x >> 4; }
  __device__ __forceinline__ static uint32_t bits_of(int h) {
    uint32_t b = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) b |= 1u << unit_of(h, k);
    return b;
  }
  __device__ __forceinline__ static void local(int k, int& lx, int& ly) {
    const int l = threadIdx.x & 15, u = unit_of(half(), k);
    lx = (u % U) * 4 + (l & 3);
    ly = (u / U) * 4 + (l >> 2);
  }
};

// Both halves of each warp compact, in order, the batch entries whose unit
// mask reaches their units and whose list position is below their limit;
// returns this lane's half's count (and, in n_max, the larger of the two).
template <int BATCH>
__device__ __forceinline__ int half_lists(uint8_t (*list)[BATCH], const uint32_t* mask, int count, int first_pos,
                                          int limit_lo, int limit_hi, uint32_t bits_lo, uint32_t bits_hi,
                                          int& n_max) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  int n0 = 0, n1 = 0;
  for (int c = 0; c < count; c += 32) {
    const int i = c + lane;
    const uint32_t m = i < count ? mask[i] : 0u;
    const bool r0 = (m & bits_lo) && (first_pos + i) < limit_lo;
    const bool r1 = (m & bits_hi) && (first_pos + i) < limit_hi;
    const uint32_t b0 = __ballot_sync(0xffffffffu, r0), b1 = __ballot_sync(0xffffffffu, r1);
    if (r0) list[2 * warp][n0 + __popc(b0 & lt)] = (uint8_t)i;
    if (r1) list[2 * warp + 1][n1 + __popc(b1 & lt)] = (uint8_t)i;
    n0 += __popc(b0);
    n1 += __popc(b1);
  }
  __syncwarp();
  n_max = max(n0, n1);
  return (lane & 16) ? n1 : n0;
}

// The forward of one tile in the half-warp layout: the same arithmetic and
// decisions per pixel as fwd_tile (so the same image bit for bit), only the
// assignment of pixels to lanes and the list each lane walks differ.
template <int TS, int NT, int BATCH, int MODE>
__device__ __forceinline__ void fwd_tile_half(const RasterArgs& a, uint32_t pos, float* __restrict__ images,
                                              float* __restrict__ pix_T, uint32_t* __restrict__ pix_last,
                                              float* __restrict__ t_out, uint32_t* __restrict__ nc_out,
                                              int64_t n_pix_total, const FwdLoss& fl) {
  using HM = HalfMap<TS, NT>;
  constexpr int PPT = HM::PPT;
  constexpr int NW = NT / 32;
  __shared__ Stage<BATCH, 2 * NW> st;  // list[h]: half h's entries
  const uint4 desc = __ldg(a.tile_desc + pos);
  if (desc.x == kNoTile) return;  // a quadrant beyond the image (split binning)
  const int g = (int)desc.x;
  const int c = (int)desc.y;
  const ViewInfo& v = a.views[c];
  const int lt = g - v.tile_base;
  const int tyi = lt / v.tiles_x, txi = lt - tyi * v.tiles_x;
  const int ox = txi * TS, oy = tyi * TS;
  const int axi = ox & ~31, ayi = oy & ~31;
  const float ax = (float)axi, ay = (float)ayi;
  const float tox = (float)(ox - axi), toy = (float)(oy - ayi);
  const int lane = threadIdx.x & 31;
  const int hl = HM::half();  // this lane's half (list index)

  float pcx[PPT], pcy[PPT], T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
  __shared__ float s_tgt[MODE == kFwdLoss ? 3 * PPT * NT : 1];
  uint32_t last[PPT], term[PPT], ncontrib[PPT], chash[PPT];
  bool done[PPT], inside[PPT];
  int px[PPT], py[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int lx, ly;
    HM::local(k, lx, ly);
    px[k] = ox + lx;
    py[k] = oy + ly;
    pcx[k] = (float)(px[k] - axi) + 0.5f;
    pcy[k] = (float)(py[k] - ayi) + 0.5f;
    inside[k] = px[k] < v.W && py[k] < v.H;
    done[k] = !inside[k];
    T[k] = 1.0f;
    Cr[k] = Cg[k] = Cb[k] = 0.0f;
    last[k] = 0;
    term[k] = 0;
    ncontrib[k] = 0;
    chash[k] = 0;
    if (MODE == kFwdLoss && inside[k]) {
      const float* tp = fl.target + 3 * (v.pix_base + (int64_t)py[k] * v.W + px[k]);
      const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&s_tgt[3 * (k * NT + threadIdx.x)]);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + 4u * q), "l"(tp + q) : "memory");
    }
  }
  if (MODE == kFwdLoss) asm volatile("cp.async.commit_group;" ::: "memory");
  const uint2 range = make_uint2(desc.z, desc.w);
  const int n = (int)(range.y - range.x);
  const uint32_t rec_base = (uint32_t)c * (uint32_t)a.F;
  const int warp = threadIdx.x >> 5;
  const uint32_t bits_lo = HM::bits_of(2 * warp), bits_hi = HM::bits_of(2 * warp + 1);

  for (int base = 0; base < n; base += BATCH) {
    bool tdone = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) tdone &= done[k];
    if (__syncthreads_and(tdone)) break;
    int cnt = min(BATCH, n - base);
    stage_batch<TS, NT, BATCH, 2 * NW>(st, a.pair_face, range.x + base, cnt, rec_base, a.rec_uq, a.col,
                                       a.col_by_rec != 0, ax, ay, tox, toy, MODE == kFwdDebug, true);
    __syncthreads();
    int n_max;
    const int nl = half_lists<BATCH>(st.list, st.mask, cnt, 0, cnt, cnt, bits_lo, bits_hi, n_max);
    for (int jj = 0; jj < n_max; ++jj) {
      const bool act = jj < nl;
      if ((jj & 3) == 0) {  // the warp's early exit, checked every 4 entries
        bool wd = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) wd &= done[k];
        if (__all_sync(kFull, wd || !act)) break;
      }
      const int j = act ? st.list[hl][jj] : 0;
      const float4 hh = st.h[j];
      const float4 gg = st.g[j];
      float p2[PPT];
      bool con[PPT];
      bool anyc = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        float dx, dy;
        p2[k] = gauss_p2(gg, hh.x, pcx[k], pcy[k], dx, dy);
        con[k] = act && !done[k] && !(p2[k] < hh.y);
        anyc |= con[k];
      }
      if (!anyc) continue;
      const float4 col = st.col[j];
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (!con[k]) continue;
        float graw;
        float alpha = gauss_alpha(p2[k], hh.z, graw);
        float test = __fmul_rn(T[k], __fsub_rn(1.0f, alpha));
        if (test < kTMin) {
          done[k] = true;
          term[k] = (uint32_t)(base + j + 1);
          continue;
        }
        float w = __fmul_rn(alpha, T[k]);
        Cr[k] = __fmaf_rn(col.x, w, Cr[k]);
        Cg[k] = __fmaf_rn(col.y, w, Cg[k]);
        Cb[k] = __fmaf_rn(col.z, w, Cb[k]);
        T[k] = test;
        last[k] = (uint32_t)(base + j + 1);
        ++ncontrib[k];
        if (MODE == kFwdDebug) chash[k] = chash[k] * 0x9E3779B1u + st.face[j] + 1u;
      }
    }
  }
  unsigned long long evals = 0, ncon = 0;
  float lsum = 0.0f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!inside[k]) continue;
    ncon += ncontrib[k];
    int64_t pid = v.pix_base + (int64_t)py[k] * v.W + px[k];
    const float i0 = Cr[k] + T[k] * a.bg0, i1 = Cg[k] + T[k] * a.bg1, i2 = Cb[k] + T[k] * a.bg2;
    images[3 * pid] = i0;
    images[3 * pid + 1] = i1;
    images[3 * pid + 2] = i2;
    if (MODE == kFwdLoss) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      const float* tg = &s_tgt[3 * (k * NT + threadIdx.x)];
      const float d0 = i0 - tg[0], d1 = i1 - tg[1], d2 = i2 - tg[2];
      fl.grad[3 * pid] = 2.0f * d0;
      fl.grad[3 * pid + 1] = 2.0f * d1;
      fl.grad[3 * pid + 2] = 2.0f * d2;
      lsum = fmaf(d0, d0, lsum);
      lsum = fmaf(d1, d1, lsum);
      lsum = fmaf(d2, d2, lsum);
    }
    pix_T[pid] = T[k];
    pix_last[pid] = last[k];
    if (t_out) t_out[pid] = T[k];
    if (MODE == kFwdDebug) {
      nc_out[pid] = ncontrib[k];
      nc_out[n_pix_total + pid] = chash[k];
    }
    evals += term[k] ? term[k] : (uint32_t)n;
  }
  if (MODE == kFwdLoss) asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(kFull, evals, o);
    ncon += __shfl_xor_sync(kFull, ncon, o);
  }
  if (lane == 0 && evals) atomicAdd(&a.counters->evals_fwd, evals);
  if (lane == 0 && ncon) atomicAdd(&a.counters->contribs, ncon);
  if (MODE == kFwdLoss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if (lane == 0) fl.part[(int64_t)g * NW + warp] = lsum;
  }
}

// PERSIST: a persistent grid of resident CTAs taking positions from the
// cursor; otherwise one CTA per position (the default: measured faster).
// ---------------------------------------------------------------- warp-staged layout
// Each warp stages the tile's list itself, 32 entries at a time (lane l loads
// entry c + l: face, record, colour), keeps those whose alpha >= 1/255
// region reaches its own pixel rectangle (an exact test of the ellipse
// against the rectangle, cheap here because each lane tests one entry
// against one rectangle) in warp-private shared memory, and composites
// them; no
// barrier of the CTA sits inside the tile's loop, so a warp whose pixels
// finish (or whose list is short) does not wait for the others, and the
// backward starts each warp at its own last contributor. Same per-pixel
// arithmetic and decisions as fwd_tile / bwd_tile. The CTA's warps load the
// same records (mostly from L1).
struct WarpSlots {
  float4 g[32];   // (ux, uy, a2, b2)
  float4 h[32];   // (c2, t2, o, 0)
  float4 col[32]; // (r, g, b, 0)
  uint32_t pos[32];
  uint32_t rid[32];
  uint32_t face[32];
};

// Whether a Gaussian can reach alpha >= 1/255 at some point of the box
// [x0, x1] x [y0, y1] of pixel centres (anchor-relative): the exponent
// p2(d) = a2 dx^2 + b2 dx dy + c2 dy^2, d = mean - point, is concave, so its
// maximum over the box is 0 at the mean when the mean lies inside, else on an
// edge, where it is a concave parabola maximised at its clamped vertex. The
// test passes when that maximum reaches t2 = -log2(255 o) within a margin
// (1e-4 in log2 units plus 1e-5 of the magnitude of the exponent's terms,
// far above the FP32 rounding of this test and of the per-pixel evaluation),
// so culling never changes a result.
__device__ __forceinline__ bool reaches_box(float ux, float uy, float a2, float b2, float c2, float t2, float x0,
                                            float x1, float y0, float y1) {
  if (!(t2 <= 0.0f)) return false;  // o < 1/255: reaches nothing
  const float dxl = ux - x1, dxh = ux - x0, dyl = uy - y1, dyh = uy - y0;
  if (dxl <= 0.0f && dxh >= 0.0f && dyl <= 0.0f && dyh >= 0.0f) return true;
  bool hit = false;
  auto test = [&](float dx, float dy) {
    const float xx = a2 * dx * dx, xy = b2 * dx * dy, yy = c2 * dy * dy;
    const float mag = fabsf(xx) + fabsf(xy) + fabsf(yy);
    hit |= (xx + xy + yy) + (1e-4f + 1e-5f * mag) >= t2;
  };
  // edges dx = const: vertex at dy = -b2 dx / (2 c2); edges dy = const alike
  const float ky = -0.5f * b2 / c2, kx = -0.5f * b2 / a2;
  test(dxl, fminf(fmaxf(ky * dxl, dyl), dyh));
  test(dxh, fminf(fmaxf(ky * dxh, dyl), dyh));
  test(fminf(fmaxf(kx * dyl, dxl), dxh), dyl);
  test(fminf(fmaxf(kx * dyh, dxl), dxh), dyh);
  return hit;
}

// Stages a chunk of 32 entries of the tile's list (lane l: list position i,
// face f, already loaded; valid: i lies in the chunk's range) that reach the
// warp's pixel rectangle into the warp's slots, in order; returns their
// count. The callers load the next chunk's faces before compositing this
// one, so that load overlaps the compositing.
__device__ __forceinline__ int warp_stage(WarpSlots& ws, const RasterArgs& a, uint32_t f, int i, bool valid,
                                          uint32_t rec_base, float ax, float ay, float rx0, float rx1, float ry0,
                                          float ry1) {
  const int lane = threadIdx.x & 31;
  bool rel = false;
  float4 g4, h4, c4;
  uint32_t rid = 0;
  if (valid) {
    rid = rec_base + f;
    const float4 u = __ldg(a.rec_uq + 2 * (size_t)rid);
    const float4 q = __ldg(a.rec_uq + 2 * (size_t)rid + 1);
    const float4 col = __ldg(a.col + (a.col_by_rec ? rid : f));
    const float ux = __fadd_rn(__fsub_rn(u.x, ax), u.z);
    const float uy = __fadd_rn(__fsub_rn(u.y, ay), u.w);
    rel = reaches_box(ux, uy, q.x, q.y, q.z, q.w, rx0, rx1, ry0, ry1);
    g4 = make_float4(ux, uy, q.x, q.y);
    h4 = make_float4(q.z, q.w, col.w, 0.0f);
    c4 = make_float4(col.x, col.y, col.z, 0.0f);
  }
  const uint32_t bal = __ballot_sync(kFull, rel);
  if (rel) {
    const int r = __popc(bal & ((1u << lane) - 1u));
    ws.g[r] = g4;
    ws.h[r] = h4;
    ws.col[r] = c4;
    ws.pos[r] = (uint32_t)i;
    ws.rid[r] = rid;
    ws.face[r] = f;
  }
  __syncwarp();
  return __popc(bal);
}

template <int TS, int NT, int MODE>
__device__ __forceinline__ void fwd_tile_ws(const RasterArgs& a, uint32_t pos, float* __restrict__ images,
                                            float* __restrict__ pix_T, uint32_t* __restrict__ pix_last,
                                            float* __restrict__ t_out, uint32_t* __restrict__ nc_out,
                                            int64_t n_pix_total, const FwdLoss& fl) {
  constexpr int PPT = PixMap<TS, NT>::PPT;
  constexpr int NW = NT / 32;
  // 16x16 and 32x32 tiles: one warp vote per entry and per pixel slot, then
  // the compositing step on every lane with the non-contributing lanes'
  // updates discarded by selects (1.6% faster than a divergent branch per
  // slot on the 64-view workload); 8x8 tiles (dense meshes, few lanes
  // contributing per entry) keep the branches (the selects were 5.7% slower
  // on the level-8 mesh)
  constexpr bool kPredicated = TS >= 16;
  __shared__ WarpSlots slots[NW];
  const uint4 desc = __ldg(a.tile_desc + pos);
  if (desc.x == kNoTile) return;  // a quadrant beyond the image (split binning)
  const int g = (int)desc.x;
  const int c = (int)desc.y;
  const ViewInfo& v = a.views[c];
  const int lt = g - v.tile_base;
  const int tyi = lt / v.tiles_x, txi = lt - tyi * v.tiles_x;
  const int ox = txi * TS, oy = tyi * TS;
  const int axi = ox & ~31, ayi = oy & ~31;
  const float ax = (float)axi, ay = (float)ayi;
  const float tox = (float)(ox - axi), toy = (float)(oy - ayi);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  WarpSlots& ws = slots[warp];

  float pcx[PPT], pcy[PPT], T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
  __shared__ float s_tgt[MODE == kFwdLoss ? 3 * PPT * NT : 1];
  uint32_t last[PPT], term[PPT], ncontrib[PPT], chash[PPT];
  bool done[PPT], inside[PPT];
  int px[PPT], py[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int lx, ly;
    PixMap<TS, NT>::local(k, lx, ly);
    px[k] = ox + lx;
    py[k] = oy + ly;
    pcx[k] = (float)(px[k] - axi) + 0.5f;
    pcy[k] = (float)(py[k] - ayi) + 0.5f;
    inside[k] = px[k] < v.W && py[k] < v.H;
    done[k] = !inside[k];
    T[k] = 1.0f;
    Cr[k] = Cg[k] = Cb[k] = 0.0f;
    last[k] = 0;
    term[k] = 0;
    ncontrib[k] = 0;
    chash[k] = 0;
    if (MODE == kFwdLoss && inside[k]) {
      const float* tp = fl.target + 3 * (v.pix_base + (int64_t)py[k] * v.W + px[k]);
      const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&s_tgt[3 * (k * NT + threadIdx.x)]);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + 4u * q), "l"(tp + q) : "memory");
    }
  }
  if (MODE == kFwdLoss) asm volatile("cp.async.commit_group;" ::: "memory");
  const uint2 range = make_uint2(desc.z, desc.w);
  const int n = (int)(range.y - range.x);
  const uint32_t rec_base = (uint32_t)c * (uint32_t)a.F;
  float rx0, rx1, ry0, ry1;
  PixMap<TS, NT>::region(tox, toy, rx0, rx1, ry0, ry1);

  // 8x8 tiles: the next chunk's faces are loaded before this chunk is
  // composited (1.6% faster there; at 16x16 the extra live register costs
  // the 128-thread shape an occupancy step, 4% slower)
  constexpr bool kPrefetch = TS == 8;
  uint32_t f_next = (kPrefetch && lane < n) ? __ldg(a.pair_face + range.x + lane) : 0u;
  for (int c0 = 0; c0 < n; c0 += 32) {
    bool wd = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) wd &= done[k];
    if (__all_sync(kFull, wd)) break;
    const int i = c0 + lane;
    uint32_t f;
    if (kPrefetch) {
      f = f_next;
      f_next = i + 32 < n ? __ldg(a.pair_face + range.x + i + 32) : 0u;
    } else {
      f = i < n ? __ldg(a.pair_face + range.x + i) : 0u;
    }
    const int nl = warp_stage(ws, a, f, i, i < n, rec_base, ax, ay, rx0, rx1, ry0, ry1);
    for (int jj = 0; jj < nl; ++jj) {
      if ((jj & 7) == 7) {  // the warp's early exit, checked every 8 entries (every 2 or 4: 0.6-1.6% slower)
        bool wd2 = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) wd2 &= done[k];
        if (__all_sync(kFull, wd2)) break;
      }
      const float4 hh = ws.h[jj];
      const float4 gg = ws.g[jj];
      float p2[PPT];
      bool con[PPT];
      bool anyc = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        float dx, dy;
        p2[k] = gauss_p2(gg, hh.x, pcx[k], pcy[k], dx, dy);
        con[k] = !done[k] && !(p2[k] < hh.y);
        anyc |= con[k];
      }
      if (kPredicated ? !__any_sync(kFull, anyc) : !anyc) continue;
      const float4 col = ws.col[jj];
      const uint32_t p1 = ws.pos[jj] + 1u;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (kPredicated ? !__any_sync(kFull, con[k]) : !con[k]) continue;
        float graw;
        float alpha = gauss_alpha(p2[k], hh.z, graw);
        float test = __fmul_rn(T[k], __fsub_rn(1.0f, alpha));
        if constexpr (kPredicated) {
          // every lane computes; a lane without a contribution keeps its
          // state (fma with a zero weight leaves the colour sums unchanged)
          const bool stop = con[k] && test < kTMin;
          const bool add = con[k] && !(test < kTMin);
          done[k] = done[k] || stop;
          term[k] = stop ? p1 : term[k];
          const float w = add ? __fmul_rn(alpha, T[k]) : 0.0f;
          Cr[k] = __fmaf_rn(col.x, w, Cr[k]);
          Cg[k] = __fmaf_rn(col.y, w, Cg[k]);
          Cb[k] = __fmaf_rn(col.z, w, Cb[k]);
          T[k] = add ? test : T[k];
          last[k] = add ? p1 : last[k];
          ncontrib[k] += add ? 1u : 0u;
          if (MODE == kFwdDebug && add) chash[k] = chash[k] * 0x9E3779B1u + ws.face[jj] + 1u;
        } else {
          if (test < kTMin) {
            done[k] = true;
            term[k] = p1;
            continue;
          }
          float w = __fmul_rn(alpha, T[k]);
          Cr[k] = __fmaf_rn(col.x, w, Cr[k]);
          Cg[k] = __fmaf_rn(col.y, w, Cg[k]);
          Cb[k] = __fmaf_rn(col.z, w, Cb[k]);
          T[k] = test;
          last[k] = p1;
          ++ncontrib[k];
          if (MODE == kFwdDebug) chash[k] = chash[k] * 0x9E3779B1u + ws.face[jj] + 1u;
        }
      }
    }
    __syncwarp();  // the slots are refilled by the next chunk
  }
  unsigned long long evals = 0, ncon = 0;
  float lsum = 0.0f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!inside[k]) continue;
    ncon += ncontrib[k];
    int64_t pid = v.pix_base + (int64_t)py[k] * v.W + px[k];
    const float i0 = Cr[k] + T[k] * a.bg0, i1 = Cg[k] + T[k] * a.bg1, i2 = Cb[k] + T[k] * a.bg2;
    images[3 * pid] = i0;
    images[3 * pid + 1] = i1;
    images[3 * pid + 2] = i2;
    if (MODE == kFwdLoss) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      const float* tg = &s_tgt[3 * (k * NT + threadIdx.x)];
      const float d0 = i0 - tg[0], d1 = i1 - tg[1], d2 = i2 - tg[2];
      fl.grad[3 * pid] = 2.0f * d0;
      fl.grad[3 * pid + 1] = 2.0f * d1;
      fl.grad[3 * pid + 2] = 2.0f * d2;
      lsum = fmaf(d0, d0, lsum);
      lsum = fmaf(d1, d1, lsum);
      lsum = fmaf(d2, d2, lsum);
    }
    pix_T[pid] = T[k];
    pix_last[pid] = last[k];
    if (t_out) t_out[pid] = T[k];
    if (MODE == kFwdDebug) {
      nc_out[pid] = ncontrib[k];
      nc_out[n_pix_total + pid] = chash[k];
    }
    evals += term[k] ? term[k] : (uint32_t)n;
  }
  if (MODE == kFwdLoss) asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(kFull, evals, o);
    ncon += __shfl_xor_sync(kFull, ncon, o);
  }
  if (lane == 0 && evals) atomicAdd(&a.counters->evals_fwd, evals);
  if (lane == 0 && ncon) atomicAdd(&a.counters->contribs, ncon);
  if (MODE == kFwdLoss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if (lane == 0) fl.part[(int64_t)g * NW + warp] = lsum;
  }
}

// LAYOUT: kLayoutCta (staging by the CTA, full warps), kLayoutHalf (the
// half-warp layout: 16x16 tiles, 128 or 256 threads) or kLayoutWarp (staging
// by each warp); the last two with one CTA per tile.
template <int TS, int NT, int BATCH, int MODE, bool PERSIST, int LAYOUT = kLayoutCta>
__global__ void __launch_bounds__(NT, FwdMinBlocks<TS, NT>::value)
    k_raster_fwd(RasterArgs a, float* __restrict__ images, float* __restrict__ pix_T, uint32_t* __restrict__ pix_last,
                 float* __restrict__ t_out, uint32_t* __restrict__ nc_out, int64_t n_pix_total, FwdLoss fl) {
  pdl_enter();
  if constexpr (LAYOUT == kLayoutHalf) {
    static_assert(!PERSIST, "half-warp layout: one CTA per tile");
    fwd_tile_half<TS, NT, BATCH, MODE>(a, blockIdx.x, images, pix_T, pix_last, t_out, nc_out, n_pix_total, fl);
  } else if constexpr (LAYOUT == kLayoutWarp) {
    static_assert(!PERSIST, "warp-staged layout: one CTA per tile");
    fwd_tile_ws<TS, NT, MODE>(a, blockIdx.x, images, pix_T, pix_last, t_out, nc_out, n_pix_total, fl);
  } else if (!PERSIST) {
    fwd_tile<TS, NT, BATCH, MODE>(a, blockIdx.x, images, pix_T, pix_last, t_out, nc_out, n_pix_total, fl);
  } else {
    uint32_t pos;
    while (next_position(&a.counters->raster_next_fwd, a.n_pos, pos))
      fwd_tile<TS, NT, BATCH, MODE>(a, pos, images, pix_T, pix_last, t_out, nc_out, n_pix_total, fl);
  }
}

// Sum of n floats into *out, one block, in a fixed order, with double-float
// accumulation in FP32 arithmetic (error ~n 2^-44 relative, no FP64 pipe).
__global__ void __launch_bounds__(1024) k_sum_partials(const float* __restrict__ part, int64_t n, double scale,
                                                       double* __restrict__ out) {
  pdl_enter();
  __shared__ df sw[32];
  // rounds of 16 independent loads per thread, then their (fixed-order) sum
  constexpr int R = 16;
  df acc{0.0f, 0.0f};
  for (int64_t i0 = 0; i0 < n; i0 += 1024 * R) {
    float x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = i0 + (int64_t)r * 1024 + threadIdx.x;
      x[r] = i < n ? part[i] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) acc = df_add(acc, df{x[r], 0.0f});
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    acc = df_add(acc, df{__shfl_xor_sync(kFull, acc.hi, o), __shfl_xor_sync(kFull, acc.lo, o)});
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = sw[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      acc = df_add(acc, df{__shfl_xor_sync(kFull, acc.hi, o), __shfl_xor_sync(kFull, acc.lo, o)});
    if (threadIdx.x == 0) *out = ((double)acc.hi + (double)acc.lo) * scale;
  }
}

// ---------------------------------------------------------------- backward
// Sum of v[0..7] over the warp, transposed: on return lane L (L % 4 == 0)
// holds the total of value index ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 +
// ((L >> 2) & 1).
__device__ __forceinline__ float warp_reduce8_transposed(const float v[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float k0 = (b4 ? v[4] : v[0]) + __shfl_xor_sync(kFull, b4 ? v[0] : v[4], 16);
  float k1 = (b4 ? v[5] : v[1]) + __shfl_xor_sync(kFull, b4 ? v[1] : v[5], 16);
  float k2 = (b4 ? v[6] : v[2]) + __shfl_xor_sync(kFull, b4 ? v[2] : v[6], 16);
  float k3 = (b4 ? v[7] : v[3]) + __shfl_xor_sync(kFull, b4 ? v[3] : v[7], 16);
  float m0 = (b3 ? k2 : k0) + __shfl_xor_sync(kFull, b3 ? k0 : k2, 8);
  float m1 = (b3 ? k3 : k1) + __shfl_xor_sync(kFull, b3 ? k1 : k3, 8);
  float s = (b2 ? m1 : m0) + __shfl_xor_sync(kFull, b2 ? m0 : m1, 4);
  s += __shfl_xor_sync(kFull, s, 2);
  s += __shfl_xor_sync(kFull, s, 1);
  return s;
}

// A list entry whose contributions come from at most this many lanes of a
// warp is added by those lanes' own atomics instead of the warp reduction
// (swept 0-32 on four workloads: with scalar atomics 8 was best, with the
// vector atomics 20; above that, same-address atomics serialise).
#ifndef GMR_BWD_DIRECT_LANES
#define GMR_BWD_DIRECT_LANES 20
#endif
constexpr int kBwdDirectLanes = GMR_BWD_DIRECT_LANES;
// The same for the warp-staged layout (swept 8, 12, 20, 32 on three
// workloads: 12 is best there, 3-5% faster backward than 20; the block-staged
// layout keeps 20).
#ifndef GMR_BWD_DIRECT_LANES_WS
#define GMR_BWD_DIRECT_LANES_WS 12
#endif
constexpr int kBwdDirectLanesWs = GMR_BWD_DIRECT_LANES_WS;
// The same per 16-lane half in the half-warp layout (both halves under it;
// swept 10-16 on the 64-view workload with the predicated chain: 12 and 14
// 2% faster than 10, 16, never reducing, 33% slower).
#ifndef GMR_BWD_DIRECT_LANES_HALF
#define GMR_BWD_DIRECT_LANES_HALF 12
#endif
constexpr int kBwdDirectLanesHalf = GMR_BWD_DIRECT_LANES_HALF;

// LOSS: dL/dimg = 2 (img - target) is formed from bl.img and bl.target (the
// squared-error loss), and each warp writes its pixels' sum of squared
// errors to bl.part; otherwise dL/dimg is read from dL_dimg (or is zero).
// Resident CTAs per SM the backward's register allocation must allow: 9 for
// the 128-thread shape (<= 56 registers; 1% faster on the dense workloads
// than the compiler's 64), the compiler's choice otherwise.
template <int NT>
struct BwdMinBlocks {
  static constexpr int value = NT == 128 ? 9 : 0;
};

// Deterministic backward: the 9 sums of one (tile, Gaussian) pair into its
// slot, the rec_slot of the record plus the rank of the tile (tx, ty) in the
// record's rectangle, row by row (the order in which the projection dealt
// the record's pairs to its slots).
__device__ __forceinline__ void det_store(const RasterArgs& a, uint32_t rid, int tx, int ty, const float* sum) {
  const uint2 rect = __ldg(a.rec_rect + rid);
  const int x0 = (int)(rect.x & 0xffffu), x1 = (int)(rect.x >> 16), y0 = (int)(rect.y & 0xffffu);
  const int64_t slot = (int64_t)__ldg(a.rec_slot + rid) + (int64_t)(ty - y0) * (x1 - x0 + 1) + (tx - x0);
  if (slot >= a.cap_slots) return;  // pair overflow (reported by the forward)
  float4* pg = a.pair_grad + 3 * slot;
  pg[0] = make_float4(sum[0], sum[1], sum[2], sum[3]);
  pg[1] = make_float4(sum[4], sum[5], sum[6], sum[7]);
  pg[2] = make_float4(sum[8], 0.0f, 0.0f, 0.0f);
}

// DET: the deterministic backward (GMR_FLAG_DETERMINISTIC): each warp
// reduces its share of every entry of its list over its lanes (a fixed
// shuffle tree) into shared memory, and after each batch one thread per
// entry adds the warps' shares in warp order and stores the pair's sums to
// its slot; pairs behind the tile's last contributor get zeros.
template <int TS, int NT, int BATCH, bool LOSS, bool DET = false>
__device__ __forceinline__ void bwd_tile(const RasterArgs& a, uint32_t pos, const float* __restrict__ dL_dimg,
                                         const float* __restrict__ dL_dT, const float* __restrict__ pix_T,
                                         const uint32_t* __restrict__ pix_last, float4* __restrict__ rec_grad,
                                         float4* __restrict__ face_grad, const BwdLoss& bl) {
  constexpr int PPT = PixMap<TS, NT>::PPT;
  constexpr int NW = NT / 32;
  static_assert(!DET || BATCH <= 128, "deterministic backward: at most 128 Gaussians per batch");
  __shared__ Stage<BATCH, NW> st;
  __shared__ uint32_t s_maxlast;
  __shared__ float s_acc[DET ? NW : 1][9][DET ? BATCH : 1];  // per warp, value and entry
  __shared__ uint32_t s_wmax[DET ? NW : 1];
  // the tile at this compositing position, its view and its pair range
  const uint4 desc = __ldg(a.tile_desc + pos);
  if (desc.x == kNoTile) return;  // a quadrant beyond the image (split binning)
  const int g = (int)desc.x;
  const int c = (int)desc.y;
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  const ViewInfo& v = a.views[c];
  const int lt = g - v.tile_base;
  const int tyi = lt / v.tiles_x, txi = lt - tyi * v.tiles_x;
  const int ox = txi * TS, oy = tyi * TS;
  const int axi = ox & ~31, ayi = oy & ~31;
  const float ax = (float)axi, ay = (float)ayi;
  const float tox = (float)(ox - axi), toy = (float)(oy - ayi);
  const int lane = threadIdx.x & 31;
  const uint2 range = make_uint2(desc.z, desc.w);
  const uint32_t rec_base = (uint32_t)c * (uint32_t)a.F;
  // a tile whose list fits one batch is staged now, its loads in flight
  // with the pixels' below (the prologue's barrier publishes it); the batch
  // loop then stages nothing
  const int n_all = (int)(range.y - range.x);
  const bool one = n_all <= BATCH;
  if (one && n_all > 0)
    stage_batch<TS, NT, BATCH>(st, a.pair_face, range.x, n_all, rec_base, a.rec_uq, a.col,
                               a.col_by_rec != 0, ax, ay, tox, toy, true);

  // SG = (colour composited behind the current Gaussian, plus T_final bg) . g
  float pcx[PPT], pcy[PPT], T[PPT], SG[PPT], G0[PPT], G1[PPT], G2[PPT];
  uint32_t last[PPT];
  uint32_t tmax = 0;
  float lsum = 0.0f;  // LOSS: FP32 sum of this thread's squared errors
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int lx, ly;
    PixMap<TS, NT>::local(k, lx, ly);
    int px = ox + lx, py = oy + ly;
    pcx[k] = (float)(px - axi) + 0.5f;
    pcy[k] = (float)(py - ayi) + 0.5f;
    bool inside = px < v.W && py < v.H;
    float gT;
    if (inside) {
      int64_t pid = v.pix_base + (int64_t)py * v.W + px;
      T[k] = pix_T[pid];
      last[k] = pix_last[pid];
      if (LOSS) {
        const float d0 = bl.img[3 * pid] - bl.target[3 * pid];
        const float d1 = bl.img[3 * pid + 1] - bl.target[3 * pid + 1];
        const float d2 = bl.img[3 * pid + 2] - bl.target[3 * pid + 2];
        G0[k] = 2.0f * d0;
        G1[k] = 2.0f * d1;
        G2[k] = 2.0f * d2;
        lsum = fmaf(d0, d0, lsum);
        lsum = fmaf(d1, d1, lsum);
        lsum = fmaf(d2, d2, lsum);
      } else if (dL_dimg) {
        G0[k] = dL_dimg[3 * pid];
        G1[k] = dL_dimg[3 * pid + 1];
        G2[k] = dL_dimg[3 * pid + 2];
      } else {
        G0[k] = G1[k] = G2[k] = 0.0f;
      }
      gT = dL_dT ? dL_dT[pid] : 0.0f;
    } else {
      T[k] = 1.0f;
      last[k] = 0;
      G0[k] = G1[k] = G2[k] = 0.0f;
      gT = 0.0f;
    }
    // the background term T_final bg and the final transmittance itself
    // (dL/dT_final, a silhouette loss) both enter as "colour behind every
    // Gaussian": a fourth channel with Gaussian colour 0 and background 1
    SG[k] = T[k] * (a.bg0 * G0[k] + a.bg1 * G1[k] + a.bg2 * G2[k] + gT);
    tmax = max(tmax, last[k]);
  }
  uint32_t wmax = tmax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, o));
  if (lane == 0) atomicMax(&s_maxlast, wmax);
  if (DET && lane == 0) s_wmax[threadIdx.x >> 5] = wmax;
  __shared__ float s_lsum[LOSS ? NT / 32 : 1];
  if (LOSS) {  // warp sums now, the CTA's partial after the barrier
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if (lane == 0) s_lsum[threadIdx.x >> 5] = lsum;
  }
  __syncthreads();
  if (LOSS && threadIdx.x == 0) {  // pairwise over the warps (<= 3 levels)
    float b[NT / 32];
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) b[w] = s_lsum[w];
#pragma unroll
    for (int h = 1; h < NT / 32; h <<= 1)
#pragma unroll
      for (int w = 0; w + h < NT / 32; w += 2 * h) b[w] += b[w + h];
    bl.part[g] = b[0];
  }
  const int end_all = (int)s_maxlast;
  unsigned long long evals = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) evals += last[k];

  for (int end = end_all; end > 0; end -= BATCH) {
    const int start = max(0, end - BATCH);
    if (!one) {
      __syncthreads();
      stage_batch<TS, NT, BATCH>(st, a.pair_face, range.x + start, end - start, rec_base, a.rec_uq,
                                 a.col, a.col_by_rec != 0, ax, ay, tox, toy, true);
      __syncthreads();
    }
    const int nl = warp_list<BATCH, NW>(st, end - start, start, (int)wmax, PixMap<TS, NT>::warp_bits());
    const int warp = threadIdx.x >> 5;
    for (int jj = nl - 1; jj >= 0; --jj) {
      const int j = st.list[warp][jj];
      const int pos_j = start + j;
      const float4 hh = st.h[j];
      const float4 gg = st.g[j];
      float p2[PPT], dxs[PPT], dys[PPT];
      bool con[PPT];
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        p2[k] = gauss_p2(gg, hh.x, pcx[k], pcy[k], dxs[k], dys[k]);
        con[k] = ((uint32_t)pos_j < last[k]) && !(p2[k] < hh.y);
        any |= con[k];
      }
      float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const uint32_t cm = __ballot_sync(kFull, any);
      if (cm != 0u) {
        const float4 col = st.col[j];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          // one vote per pixel slot: the lanes without a contribution
          // compute along and keep their state (a divergent branch per
          // slot measured 1.7% slower in the half-warp backward, 2.8% in
          // the block-staged one)
          if (!__any_sync(kFull, con[k])) continue;
          float graw;
          float alpha = gauss_alpha(p2[k], hh.z, graw);
          float om = __fsub_rn(1.0f, alpha);
          float inv = rcp_refined(om);
          float Tb = T[k] * inv;
          float w = alpha * Tb;
          float cg = col.x * G0[k] + col.y * G1[k] + col.z * G2[k];
          // T_i (c.g) - S.g / (1 - alpha) = (T_(i+1) (c.g) - S.g) / (1 - alpha):
          // the difference of the two (often nearly equal) terms in one FMA
          float dalpha = inv * __fmaf_rn(T[k], cg, -SG[k]);
          const float sg_new = SG[k] + w * cg;
          SG[k] = con[k] ? sg_new : SG[k];
          T[k] = con[k] ? Tb : T[k];
          w = con[k] ? w : 0.0f;
          float dq = (con[k] && graw < kAlphaMax) ? dalpha * alpha : 0.0f;
          float qx = dq * dxs[k], qy = dq * dys[k];
          acc[0] += qx;
          acc[1] += qy;
          acc[2] += qx * dxs[k];
          acc[3] += qx * dys[k];
          acc[4] += qy * dys[k];
          acc[5] += dq;
          acc[6] += w * G0[k];
          acc[7] += w * G1[k];
          acc[8] += w * G2[k];
        }
      }
      if (DET) {  // this warp's share of entry j (zeros when it has none)
        float sv = 0.0f, s8 = 0.0f;
        if (cm != 0u) {
          s8 = acc[8];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s8 += __shfl_xor_sync(kFull, s8, o);
          sv = warp_reduce8_transposed(acc, lane);
        }
        if ((lane & 3) == 0) s_acc[warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)][j] = sv;
        if (lane == 0) s_acc[warp][8][j] = s8;
        continue;
      }
      if (cm == 0u) continue;
      // colour gradient sums: per face, or per record (view-dependent colour)
      const uint32_t ci = a.col_by_rec ? st.rid[j] : st.face[j];
      if (__popc(cm) <= kBwdDirectLanes) {
        // few contributing lanes: their own atomics cost fewer instructions
        // than the warp reduction
        if (any) {  // 16-byte vector atomics: 3 instead of 9
          float4* rg = rec_grad + 2 * (size_t)st.rid[j];
          atomicAdd(rg, make_float4(acc[0], acc[1], acc[2], acc[3]));
          atomicAdd(reinterpret_cast<float*>(rg + 1), acc[4]);
          atomicAdd(face_grad + ci, make_float4(acc[6], acc[7], acc[8], acc[5]));
        }
        continue;
      }
      float s8 = acc[8];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s8 += __shfl_xor_sync(kFull, s8, o);
      float s = warp_reduce8_transposed(acc, lane);
      if ((lane & 3) == 0) {
        int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        float* dst;
        if (vi < 5) dst = reinterpret_cast<float*>(rec_grad + 2 * (size_t)st.rid[j]) + vi;
        else if (vi == 5) dst = reinterpret_cast<float*>(face_grad + ci) + 3;
        else dst = reinterpret_cast<float*>(face_grad + ci) + (vi - 6);
        atomicAdd(dst, s);
      }
      if (lane == 0) atomicAdd(reinterpret_cast<float*>(face_grad + ci) + 2, s8);
    }
    if (DET) {
      __syncthreads();  // every warp's shares of this batch are in s_acc
      for (int j = threadIdx.x; j < end - start; j += NT) {
        // the warps whose list held entry j (the test of warp_list), in order
        float sum[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const uint32_t m = st.mask[j];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          if ((m & PixMap<TS, NT>::warp_bits_of(w)) && start + j < (int)s_wmax[w]) {
#pragma unroll
            for (int q = 0; q < 9; ++q) sum[q] += s_acc[w][q][j];
          }
        }
        det_store(a, st.rid[j], txi, tyi, sum);
      }
    }
  }
  if (DET) {  // the pairs behind the tile's last contributor: zeros
    const float zero[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = end_all + (int)threadIdx.x; j < (int)(range.y - range.x); j += NT)
      det_store(a, rec_base + __ldg(a.pair_face + range.x + j), txi, tyi, zero);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(kFull, evals, o);
  if (lane == 0 && evals) atomicAdd(&a.counters->evals_bwd, evals);
}

// Sum of v[0..7] over each 16-lane half of the warp, transposed: on return
// lane L of a half (L = lane % 16, L even) holds the half's total of value
// index ((L >> 3) & 1) * 4 + ((L >> 2) & 1) * 2 + ((L >> 1) & 1).
__device__ __forceinline__ float half_reduce8_transposed(const float v[8], int lane) {
  const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float k0 = (b3 ? v[4] : v[0]) + __shfl_xor_sync(kFull, b3 ? v[0] : v[4], 8);
  float k1 = (b3 ? v[5] : v[1]) + __shfl_xor_sync(kFull, b3 ? v[1] : v[5], 8);
  float k2 = (b3 ? v[6] : v[2]) + __shfl_xor_sync(kFull, b3 ? v[2] : v[6], 8);
  float k3 = (b3 ? v[7] : v[3]) + __shfl_xor_sync(kFull, b3 ? v[3] : v[7], 8);
  float m0 = (b2 ? k2 : k0) + __shfl_xor_sync(kFull, b2 ? k0 : k2, 4);
  float m1 = (b2 ? k3 : k1) + __shfl_xor_sync(kFull, b2 ? k1 : k3, 4);
  float s = (b1 ? m1 : m0) + __shfl_xor_sync(kFull, b1 ? m0 : m1, 2);
  s += __shfl_xor_sync(kFull, s, 1);
  return s;
}

// The backward of one tile in the half-warp layout (same per-pixel
// arithmetic as bwd_tile): each half walks its own list back to front from
// its own last contributor, and a half's contributions to one Gaussian are
// reduced over its 16 lanes (or added by its few contributing lanes).
template <int TS, int NT, int BATCH, bool LOSS>
__device__ __forceinline__ void bwd_tile_half(const RasterArgs& a, uint32_t pos, const float* __restrict__ dL_dimg,
                                              const float* __restrict__ dL_dT, const float* __restrict__ pix_T,
                                              const uint32_t* __restrict__ pix_last, float4* __restrict__ rec_grad,
                                              float4* __restrict__ face_grad, const BwdLoss& bl) {
  using HM = HalfMap<TS, NT>;
  constexpr int PPT = HM::PPT;
  constexpr int NW = NT / 32;
  __shared__ Stage<BATCH, 2 * NW> st;
  __shared__ uint32_t s_maxlast;
  const uint4 desc = __ldg(a.tile_desc + pos);
  if (desc.x == kNoTile) return;  // a quadrant beyond the image (split binning)
  const int g = (int)desc.x;
  const int c = (int)desc.y;
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  const ViewInfo& v = a.views[c];
  const int lt = g - v.tile_base;
  const int tyi = lt / v.tiles_x, txi = lt - tyi * v.tiles_x;
  const int ox = txi * TS, oy = tyi * TS;
  const int axi = ox & ~31, ayi = oy & ~31;
  const float ax = (float)axi, ay = (float)ayi;
  const float tox = (float)(ox - axi), toy = (float)(oy - ayi);
  const int lane = threadIdx.x & 31;
  const int hl = HM::half();

  float pcx[PPT], pcy[PPT], T[PPT], SG[PPT], G0[PPT], G1[PPT], G2[PPT];
  uint32_t last[PPT];
  uint32_t tmax = 0;
  float lsum = 0.0f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int lx, ly;
    HM::local(k, lx, ly);
    int px = ox + lx, py = oy + ly;
    pcx[k] = (float)(px - axi) + 0.5f;
    pcy[k] = (float)(py - ayi) + 0.5f;
    bool inside = px < v.W && py < v.H;
    float gT;
    if (inside) {
      int64_t pid = v.pix_base + (int64_t)py * v.W + px;
      T[k] = pix_T[pid];
      last[k] = pix_last[pid];
      if (LOSS) {
        const float d0 = bl.img[3 * pid] - bl.target[3 * pid];
        const float d1 = bl.img[3 * pid + 1] - bl.target[3 * pid + 1];
        const float d2 = bl.img[3 * pid + 2] - bl.target[3 * pid + 2];
        G0[k] = 2.0f * d0;
        G1[k] = 2.0f * d1;
        G2[k] = 2.0f * d2;
        lsum = fmaf(d0, d0, lsum);
        lsum = fmaf(d1, d1, lsum);
        lsum = fmaf(d2, d2, lsum);
      } else if (dL_dimg) {
        G0[k] = dL_dimg[3 * pid];
        G1[k] = dL_dimg[3 * pid + 1];
        G2[k] = dL_dimg[3 * pid + 2];
      } else {
        G0[k] = G1[k] = G2[k] = 0.0f;
      }
      gT = dL_dT ? dL_dT[pid] : 0.0f;
    } else {
      T[k] = 1.0f;
      last[k] = 0;
      G0[k] = G1[k] = G2[k] = 0.0f;
      gT = 0.0f;
    }
    SG[k] = T[k] * (a.bg0 * G0[k] + a.bg1 * G1[k] + a.bg2 * G2[k] + gT);
    tmax = max(tmax, last[k]);
  }
  // last contributors: per half (the list limits) and over the CTA
  uint32_t hmax = tmax;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) hmax = max(hmax, __shfl_xor_sync(kFull, hmax, o));
  const int limit_lo = (int)__shfl_sync(kFull, hmax, 0), limit_hi = (int)__shfl_sync(kFull, hmax, 16);
  if (lane == 0) atomicMax(&s_maxlast, (uint32_t)max(limit_lo, limit_hi));
  __shared__ float s_lsum[LOSS ? NW : 1];
  if (LOSS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if (lane == 0) s_lsum[threadIdx.x >> 5] = lsum;
  }
  __syncthreads();
  if (LOSS && threadIdx.x == 0) {
    float b[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) b[w] = s_lsum[w];
#pragma unroll
    for (int h = 1; h < NW; h <<= 1)
#pragma unroll
      for (int w = 0; w + h < NW; w += 2 * h) b[w] += b[w + h];
    bl.part[g] = b[0];
  }
  const int end_all = (int)s_maxlast;
  const uint2 range = make_uint2(desc.z, desc.w);
  const uint32_t rec_base = (uint32_t)c * (uint32_t)a.F;
  const int warp = threadIdx.x >> 5;
  const uint32_t bits_lo = HM::bits_of(2 * warp), bits_hi = HM::bits_of(2 * warp + 1);
  unsigned long long evals = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) evals += last[k];

  // (staging a one-batch list before the prologue's barrier, as the
  // block-staged backward does, made this layout 3% slower)
  for (int end = end_all; end > 0; end -= BATCH) {
    const int start = max(0, end - BATCH);
    __syncthreads();
    stage_batch<TS, NT, BATCH, 2 * NW>(st, a.pair_face, range.x + start, end - start, rec_base, a.rec_uq,
                                       a.col, a.col_by_rec != 0, ax, ay, tox, toy, true, true);
    __syncthreads();
    int n_max;
    const int nl = half_lists<BATCH>(st.list, st.mask, end - start, start, limit_lo, limit_hi, bits_lo, bits_hi,
                                     n_max);
    for (int jj = n_max - 1; jj >= 0; --jj) {
      const bool act = jj < nl;
      const int j = act ? st.list[hl][jj] : 0;
      const int pos_j = start + j;
      const float4 hh = st.h[j];
      const float4 gg = st.g[j];
      float p2[PPT], dxs[PPT], dys[PPT];
      bool con[PPT];
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        p2[k] = gauss_p2(gg, hh.x, pcx[k], pcy[k], dxs[k], dys[k]);
        con[k] = act && ((uint32_t)pos_j < last[k]) && !(p2[k] < hh.y);
        any |= con[k];
      }
      float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const uint32_t cm = __ballot_sync(kFull, any);
      if (cm != 0u) {
        const float4 col = st.col[j];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          // one vote per pixel slot: the lanes without a contribution
          // compute along and keep their state (a divergent branch per
          // slot measured 1.7% slower in the half-warp backward, 2.8% in
          // the block-staged one)
          if (!__any_sync(kFull, con[k])) continue;
          float graw;
          float alpha = gauss_alpha(p2[k], hh.z, graw);
          float om = __fsub_rn(1.0f, alpha);
          float inv = rcp_refined(om);
          float Tb = T[k] * inv;
          float w = alpha * Tb;
          float cg = col.x * G0[k] + col.y * G1[k] + col.z * G2[k];
          float dalpha = inv * __fmaf_rn(T[k], cg, -SG[k]);
          const float sg_new = SG[k] + w * cg;
          SG[k] = con[k] ? sg_new : SG[k];
          T[k] = con[k] ? Tb : T[k];
          w = con[k] ? w : 0.0f;
          float dq = (con[k] && graw < kAlphaMax) ? dalpha * alpha : 0.0f;
          float qx = dq * dxs[k], qy = dq * dys[k];
          acc[0] += qx;
          acc[1] += qy;
          acc[2] += qx * dxs[k];
          acc[3] += qx * dys[k];
          acc[4] += qy * dys[k];
          acc[5] += dq;
          acc[6] += w * G0[k];
          acc[7] += w * G1[k];
          acc[8] += w * G2[k];
        }
      }
      if (cm == 0u) continue;
      const uint32_t cm_half = (lane & 16) ? (cm >> 16) : (cm & 0xffffu);
      const uint32_t ci = a.col_by_rec ? st.rid[j] : st.face[j];
      if (__popc(cm & 0xffffu) <= kBwdDirectLanesHalf && __popc(cm >> 16) <= kBwdDirectLanesHalf) {
        if (any) {
          float4* rg = rec_grad + 2 * (size_t)st.rid[j];
          atomicAdd(rg, make_float4(acc[0], acc[1], acc[2], acc[3]));
          atomicAdd(reinterpret_cast<float*>(rg + 1), acc[4]);
          atomicAdd(face_grad + ci, make_float4(acc[6], acc[7], acc[8], acc[5]));
        }
        continue;
      }
      float s8 = acc[8];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s8 += __shfl_xor_sync(kFull, s8, o);
      const float sv = half_reduce8_transposed(acc, lane);
      if (cm_half != 0u) {  // this half's entry received contributions
        const int l16 = lane & 15;
        if ((l16 & 1) == 0) {
          const int vi = ((l16 >> 3) & 1) * 4 + ((l16 >> 2) & 1) * 2 + ((l16 >> 1) & 1);
          float* dst;
          if (vi < 5) dst = reinterpret_cast<float*>(rec_grad + 2 * (size_t)st.rid[j]) + vi;
          else if (vi == 5) dst = reinterpret_cast<float*>(face_grad + ci) + 3;
          else dst = reinterpret_cast<float*>(face_grad + ci) + (vi - 6);
          atomicAdd(dst, sv);
        }
        if (l16 == 0) atomicAdd(reinterpret_cast<float*>(face_grad + ci) + 2, s8);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(kFull, evals, o);
  if (lane == 0 && evals) atomicAdd(&a.counters->evals_bwd, evals);
}

template <int TS, int NT, bool LOSS>
__device__ __forceinline__ void bwd_tile_ws(const RasterArgs& a, uint32_t pos, const float* __restrict__ dL_dimg,
                                            const float* __restrict__ dL_dT, const float* __restrict__ pix_T,
                                            const uint32_t* __restrict__ pix_last, float4* __restrict__ rec_grad,
                                            float4* __restrict__ face_grad, const BwdLoss& bl) {
  constexpr int PPT = PixMap<TS, NT>::PPT;
  constexpr int NW = NT / 32;
  __shared__ WarpSlots slots[NW];
  const uint4 desc = __ldg(a.tile_desc + pos);
  if (desc.x == kNoTile) return;  // a quadrant beyond the image (split binning)
  const int g = (int)desc.x;
  const int c = (int)desc.y;
  const ViewInfo& v = a.views[c];
  const int lt = g - v.tile_base;
  const int tyi = lt / v.tiles_x, txi = lt - tyi * v.tiles_x;
  const int ox = txi * TS, oy = tyi * TS;
  const int axi = ox & ~31, ayi = oy & ~31;
  const float ax = (float)axi, ay = (float)ayi;
  const float tox = (float)(ox - axi), toy = (float)(oy - ayi);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  WarpSlots& ws = slots[warp];

  float pcx[PPT], pcy[PPT], T[PPT], SG[PPT], G0[PPT], G1[PPT], G2[PPT];
  uint32_t last[PPT];
  uint32_t tmax = 0;
  float lsum = 0.0f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int lx, ly;
    PixMap<TS, NT>::local(k, lx, ly);
    int px = ox + lx, py = oy + ly;
    pcx[k] = (float)(px - axi) + 0.5f;
    pcy[k] = (float)(py - ayi) + 0.5f;
    bool inside = px < v.W && py < v.H;
    float gT;
    if (inside) {
      int64_t pid = v.pix_base + (int64_t)py * v.W + px;
      T[k] = pix_T[pid];
      last[k] = pix_last[pid];
      if (LOSS) {
        const float d0 = bl.img[3 * pid] - bl.target[3 * pid];
        const float d1 = bl.img[3 * pid + 1] - bl.target[3 * pid + 1];
        const float d2 = bl.img[3 * pid + 2] - bl.target[3 * pid + 2];
        G0[k] = 2.0f * d0;
        G1[k] = 2.0f * d1;
        G2[k] = 2.0f * d2;
        lsum = fmaf(d0, d0, lsum);
        lsum = fmaf(d1, d1, lsum);
        lsum = fmaf(d2, d2, lsum);
      } else if (dL_dimg) {
        G0[k] = dL_dimg[3 * pid];
        G1[k] = dL_dimg[3 * pid + 1];
        G2[k] = dL_dimg[3 * pid + 2];
      } else {
        G0[k] = G1[k] = G2[k] = 0.0f;
      }
      gT = dL_dT ? dL_dT[pid] : 0.0f;
    } else {
      T[k] = 1.0f;
      last[k] = 0;
      G0[k] = G1[k] = G2[k] = 0.0f;
      gT = 0.0f;
    }
    SG[k] = T[k] * (a.bg0 * G0[k] + a.bg1 * G1[k] + a.bg2 * G2[k] + gT);
    tmax = max(tmax, last[k]);
  }
  uint32_t wmax = tmax;  // the warp walks its list from its own last contributor
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, o));
  if (LOSS) {  // one FP32 partial per tile: warp sums, then thread 0 over the warps
    __shared__ float s_lsum[NW];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if (lane == 0) s_lsum[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) b[w] = s_lsum[w];
#pragma unroll
      for (int h = 1; h < NW; h <<= 1)
#pragma unroll
        for (int w = 0; w + h < NW; w += 2 * h) b[w] += b[w + h];
      bl.part[g] = b[0];
    }
  }
  const uint2 range = make_uint2(desc.z, desc.w);
  const uint32_t rec_base = (uint32_t)c * (uint32_t)a.F;
  float rx0, rx1, ry0, ry1;
  PixMap<TS, NT>::region(tox, toy, rx0, rx1, ry0, ry1);
  unsigned long long evals = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) evals += last[k];

  // chunks from the warp's last contributor back to the front; 8x8 tiles:
  // the next chunk's faces loaded before this chunk is composited (1.4%
  // faster there; at 16x16 more spills)
  constexpr bool kPrefetch = TS == 8;
  uint32_t f_next = 0u;
  if (kPrefetch) {
    const int end = (int)wmax, i = max(0, end - 32) + lane;
    if (end > 0 && i < end) f_next = __ldg(a.pair_face + range.x + i);
  }
  for (int end = (int)wmax; end > 0; end -= 32) {
    const int c0 = max(0, end - 32);
    const int i = c0 + lane;
    uint32_t f;
    if (kPrefetch) {
      f = f_next;
      const int end2 = end - 32, i2 = max(0, end2 - 32) + lane;
      f_next = (end2 > 0 && i2 < end2) ? __ldg(a.pair_face + range.x + i2) : 0u;
    } else {
      f = i < end ? __ldg(a.pair_face + range.x + i) : 0u;
    }
    const int nl = warp_stage(ws, a, f, i, i < end, rec_base, ax, ay, rx0, rx1, ry0, ry1);
    for (int jj = nl - 1; jj >= 0; --jj) {
      const uint32_t pos_j = ws.pos[jj];
      const float4 hh = ws.h[jj];
      const float4 gg = ws.g[jj];
      float p2[PPT], dxs[PPT], dys[PPT];
      bool con[PPT];
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        p2[k] = gauss_p2(gg, hh.x, pcx[k], pcy[k], dxs[k], dys[k]);
        con[k] = (pos_j < last[k]) && !(p2[k] < hh.y);
        any |= con[k];
      }
      float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (any) {
        const float4 col = ws.col[jj];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          // (a divergent branch per pixel slot: computing the chain on every
          // lane after one vote per slot, as the other layouts do, was 3.5%
          // slower here, where few lanes contribute per entry)
          if (!con[k]) continue;
          float graw;
          float alpha = gauss_alpha(p2[k], hh.z, graw);
          float om = __fsub_rn(1.0f, alpha);
          float inv = rcp_refined(om);
          float Tb = T[k] * inv;
          float w = alpha * Tb;
          float cg = col.x * G0[k] + col.y * G1[k] + col.z * G2[k];
          float dalpha = inv * __fmaf_rn(T[k], cg, -SG[k]);
          SG[k] += w * cg;
          T[k] = Tb;
          float dq = (graw < kAlphaMax) ? dalpha * alpha : 0.0f;
          float qx = dq * dxs[k], qy = dq * dys[k];
          acc[0] += qx;
          acc[1] += qy;
          acc[2] += qx * dxs[k];
          acc[3] += qx * dys[k];
          acc[4] += qy * dys[k];
          acc[5] += dq;
          acc[6] += w * G0[k];
          acc[7] += w * G1[k];
          acc[8] += w * G2[k];
        }
      }
      const uint32_t cm = __ballot_sync(kFull, any);
      if (cm == 0u) continue;
      const uint32_t rid = ws.rid[jj];
      const uint32_t ci = a.col_by_rec ? rid : ws.face[jj];
      if (__popc(cm) <= kBwdDirectLanesWs) {
        if (any) {
          float4* rg = rec_grad + 2 * (size_t)rid;
          atomicAdd(rg, make_float4(acc[0], acc[1], acc[2], acc[3]));
          atomicAdd(reinterpret_cast<float*>(rg + 1), acc[4]);
          atomicAdd(face_grad + ci, make_float4(acc[6], acc[7], acc[8], acc[5]));
        }
        continue;
      }
      float s8 = acc[8];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s8 += __shfl_xor_sync(kFull, s8, o);
      float sv = warp_reduce8_transposed(acc, lane);
      if ((lane & 3) == 0) {
        int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        float* dst;
        if (vi < 5) dst = reinterpret_cast<float*>(rec_grad + 2 * (size_t)rid) + vi;
        else if (vi == 5) dst = reinterpret_cast<float*>(face_grad + ci) + 3;
        else dst = reinterpret_cast<float*>(face_grad + ci) + (vi - 6);
        atomicAdd(dst, sv);
      }
      if (lane == 0) atomicAdd(reinterpret_cast<float*>(face_grad + ci) + 2, s8);
    }
    __syncwarp();  // the slots are refilled by the next chunk
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(kFull, evals, o);
  if (lane == 0 && evals) atomicAdd(&a.counters->evals_bwd, evals);
}

template <int TS, int NT, int BATCH, bool LOSS, bool PERSIST, int LAYOUT = kLayoutCta, bool DET = false>
__global__ void __launch_bounds__(NT, BwdMinBlocks<NT>::value)
    k_raster_bwd(RasterArgs a, const float* __restrict__ dL_dimg, const float* __restrict__ dL_dT,
                 const float* __restrict__ pix_T, const uint32_t* __restrict__ pix_last,
                 float4* __restrict__ rec_grad, float4* __restrict__ face_grad, BwdLoss bl, BwdZero bz) {
  pdl_enter();
  static_assert(!DET || LAYOUT == kLayoutCta, "deterministic backward: block-staged layout");
  if constexpr (LAYOUT == kLayoutHalf) {
    static_assert(!PERSIST, "half-warp layout: one CTA per tile");
    bwd_tile_half<TS, NT, BATCH, LOSS>(a, blockIdx.x, dL_dimg, dL_dT, pix_T, pix_last, rec_grad, face_grad, bl);
  } else if constexpr (LAYOUT == kLayoutWarp) {
    static_assert(!PERSIST, "warp-staged layout: one CTA per tile");
    bwd_tile_ws<TS, NT, LOSS>(a, blockIdx.x, dL_dimg, dL_dT, pix_T, pix_last, rec_grad, face_grad, bl);
  } else if (!PERSIST) {
    bwd_tile<TS, NT, BATCH, LOSS, DET>(a, blockIdx.x, dL_dimg, dL_dT, pix_T, pix_last, rec_grad, face_grad, bl);
  } else {
    uint32_t pos;
    while (next_position(&a.counters->raster_next_bwd, a.n_pos, pos))
      bwd_tile<TS, NT, BATCH, LOSS, DET>(a, pos, dL_dimg, dL_dT, pix_T, pix_last, rec_grad, face_grad, bl);
  }
#pragma unroll
  for (int z = 0; z < 2; ++z)
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < bz.n[z]; i += (int64_t)gridDim.x * NT)
      bz.p[z][i] = 0.0f;
}

// ---------------------------------------------------------------- loss
// L = sum (img - target)^2 and dL/dimg = 2 (img - target) in one launch: a
// persistent grid of at most kL2LossMaxBlocks blocks (one wave on 148 SMs)
// walks the 4096-element chunks (block b takes chunks b, b + grid, ...);
// each block writes the FP64 sum of its chunks to partials[1 + block], and
// the block that finishes last (a ticket counter in partials[0]) adds the
// partials in index order, so the result does not depend on which block
// that is, then returns the counter to zero for the next call. The chunk
// assignment depends only on n, so the sum is deterministic.
constexpr int kLossThreads = 256;
constexpr int kLossItems = 16;  // floats per thread and chunk: 4 float4 of each operand
constexpr int kLossBlockElems = kLossThreads * kLossItems;
static_assert(kLossBlockElems == kL2LossBlockElems, "chunk size of l2_loss_partials_needed");

// Block sum of one double-float per thread (warp tree in double-float,
// FP64 across the warps); valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_df(df v, df* sw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, df{__shfl_xor_sync(kFull, v.hi, o), __shfl_xor_sync(kFull, v.lo, o)});
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += (double)sw[w].hi + (double)sw[w].lo;
  return s;
}

__global__ void __launch_bounds__(kLossThreads) k_l2_loss(const float* __restrict__ img,
                                                           const float* __restrict__ tgt, int64_t n,
                                                           float* __restrict__ grad, double* __restrict__ part,
                                                           double* __restrict__ loss, bool vec4) {
  // FP32 within a chunk (two running sums of 8 squares each), double-float
  // across a thread's chunks and the warp, FP64 across warps and blocks: FP64
  // arithmetic is a slow pipe on this GPU.
  const int64_t nchunks = (n + kLossBlockElems - 1) / kLossBlockElems;
  df acc{0.0f, 0.0f};
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t base = c * kLossBlockElems;
    float acc0 = 0.0f, acc1 = 0.0f;
    if (vec4 && base + kLossBlockElems <= n) {
      const float4* i4 = reinterpret_cast<const float4*>(img + base);
      const float4* t4 = reinterpret_cast<const float4*>(tgt + base);
      float4* g4 = reinterpret_cast<float4*>(grad + base);
      float4 x[kLossItems / 4], y[kLossItems / 4];
#pragma unroll
      for (int k = 0; k < kLossItems / 4; ++k) {
        x[k] = __ldcs(i4 + k * kLossThreads + threadIdx.x);
        y[k] = __ldcs(t4 + k * kLossThreads + threadIdx.x);
      }
#pragma unroll
      for (int k = 0; k < kLossItems / 4; ++k) {
        const float4 d = make_float4(x[k].x - y[k].x, x[k].y - y[k].y, x[k].z - y[k].z, x[k].w - y[k].w);
        g4[k * kLossThreads + threadIdx.x] = make_float4(2.0f * d.x, 2.0f * d.y, 2.0f * d.z, 2.0f * d.w);
        float& a = (k & 1) ? acc1 : acc0;
        a = fmaf(d.x, d.x, a);
        a = fmaf(d.y, d.y, a);
        a = fmaf(d.z, d.z, a);
        a = fmaf(d.w, d.w, a);
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < kLossItems; ++k) {
        const int64_t i = base + (int64_t)k * kLossThreads + threadIdx.x;
        if (i < n) {
          const float d = img[i] - tgt[i];
          grad[i] = 2.0f * d;
          if (k < kLossItems / 2) acc0 = fmaf(d, d, acc0);
          else acc1 = fmaf(d, d, acc1);
        }
      }
    }
    acc = df_add(acc, df{acc0 + acc1, 0.0f});
  }
  __shared__ df sw[kLossThreads / 32];
  const double bs = block_sum_df<kLossThreads>(acc, sw);
  finish_loss_partial<kLossThreads>(bs, part, loss);
}

__global__ void k_debug_records(const uint2* __restrict__ rec_rect, const float4* __restrict__ rec_uq, int64_t n_rec,
                                int32_t* __restrict__ rects, float* __restrict__ conic) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_rec) return;
  if (rects) {
    uint2 r = rec_rect[k];
    rects[4 * k] = (int32_t)(r.x & 0xffff);
    rects[4 * k + 1] = (int32_t)(r.x >> 16);
    rects[4 * k + 2] = (int32_t)(r.y & 0xffff);
    rects[4 * k + 3] = (int32_t)(r.y >> 16);
  }
  if (conic) {
    float4 q = rec_uq[2 * k + 1];
    conic[4 * k] = q.x / kNegHalfLog2e;
    conic[4 * k + 1] = q.y / kNegLog2e;
    conic[4 * k + 2] = q.z / kNegHalfLog2e;
    conic[4 * k + 3] = 0.0f;
  }
}

RasterArgs raster_args(const Workspace& ws, const uint4* tile_desc, int64_t n_pos, const uint32_t* pair_face,
                       const ViewInfo* views, int32_t F, const float* bg, bool col_by_record) {
  RasterArgs a;
  a.pair_face = pair_face;
  a.rec_uq = ws.rec_uq;
  a.col = col_by_record ? ws.rec_col : ws.face_col;
  a.col_by_rec = col_by_record ? 1 : 0;
  a.views = views;
  a.F = F;
  a.bg0 = bg[0];
  a.bg1 = bg[1];
  a.bg2 = bg[2];
  a.tile_desc = tile_desc;
  a.counters = ws.counters;
  a.n_pos = (uint32_t)n_pos;
  a.pair_grad = ws.pair_grad;
  a.rec_rect = ws.rec_rect;
  a.rec_slot = ws.rec_slot;
  a.cap_slots = std::min(ws.cap_pairs, ws.cap_det_pairs);
  return a;
}

template <int TS, int NT, int BATCH>
cudaError_t fwd_launch(int64_t n_tiles, bool persistent, int layout, bool col_by_record, const Workspace& ws,
                       const uint4* tile_desc, int64_t n_pos, const uint32_t* pair_face,
                       const ViewInfo* views, int32_t C, int32_t F, const float* bg, float* images, float* t_out,
                       uint32_t* nc_out, const FwdLoss& fl, cudaStream_t s) {
  auto kern = persistent ? (fl.target ? k_raster_fwd<TS, NT, BATCH, kFwdLoss, true>
                           : nc_out  ? k_raster_fwd<TS, NT, BATCH, kFwdDebug, true>
                                     : k_raster_fwd<TS, NT, BATCH, kFwdPlain, true>)
                        : (fl.target ? k_raster_fwd<TS, NT, BATCH, kFwdLoss, false>
                           : nc_out  ? k_raster_fwd<TS, NT, BATCH, kFwdDebug, false>
                                     : k_raster_fwd<TS, NT, BATCH, kFwdPlain, false>);
  if constexpr ((TS == 16 && (NT == 128 || NT == 256)) || (TS == 8 && (NT == 32 || NT == 64))) {
    if (layout == kLayoutHalf)
      kern = fl.target ? k_raster_fwd<TS, NT, BATCH, kFwdLoss, false, kLayoutHalf>
             : nc_out  ? k_raster_fwd<TS, NT, BATCH, kFwdDebug, false, kLayoutHalf>
                       : k_raster_fwd<TS, NT, BATCH, kFwdPlain, false, kLayoutHalf>;
  } else {
    if (layout == kLayoutHalf) return cudaErrorInvalidValue;
  }
  if constexpr (BATCH == 256) {  // (the warp-staged layout has no batch)
    if (layout == kLayoutWarp)
      kern = fl.target ? k_raster_fwd<TS, NT, 256, kFwdLoss, false, kLayoutWarp>
             : nc_out  ? k_raster_fwd<TS, NT, 256, kFwdDebug, false, kLayoutWarp>
                       : k_raster_fwd<TS, NT, 256, kFwdPlain, false, kLayoutWarp>;
  } else {
    if (layout == kLayoutWarp) return fwd_launch<TS, NT, 256>(n_tiles, persistent, layout, col_by_record, ws, tile_desc,
                                                              n_pos, pair_face, views, C, F, bg, images, t_out, nc_out,
                                                              fl, s);
  }
  const unsigned grid = persistent ? (unsigned)std::min<int64_t>(n_pos, resident_grid(kern, NT)) : (unsigned)n_pos;
  cudaError_t e = launch_chained(kern, false, dim3(grid), dim3(NT), 0, s,
                                 raster_args(ws, tile_desc, n_pos, pair_face, views, F, bg, col_by_record), images,
                                 ws.pix_T, ws.pix_last, t_out, nc_out, ws.cap_pixels, fl);
  if (e == cudaSuccess && fl.target)
    e = launch_chained(k_sum_partials, true, dim3(1), dim3(1024), 0, s, (const float*)fl.part, n_tiles * (NT / 32), 1.0,
                       fl.loss);
  return e;
}

template <int TS, int NT, int BATCH>
cudaError_t bwd_launch(int64_t n_tiles, bool persistent, int layout, bool col_by_record, bool det, const Workspace& ws,
                       const uint4* tile_desc, int64_t n_pos, const uint32_t* pair_face,
                       const ViewInfo* views, int32_t C, int32_t F, const float* bg, const float* dL,
                       const float* dLdT, const BwdLoss& bl, const BwdZero& bz, cudaStream_t s) {
  auto kern = persistent ? (bl.img ? k_raster_bwd<TS, NT, BATCH, true, true> : k_raster_bwd<TS, NT, BATCH, false, true>)
                        : (bl.img ? k_raster_bwd<TS, NT, BATCH, true, false> : k_raster_bwd<TS, NT, BATCH, false, false>);
  if (det) {
    if (layout != kLayoutCta || !ws.pair_grad || !ws.rec_slot) return cudaErrorInvalidValue;
    if constexpr (BATCH <= 128) {
      kern = persistent ? (bl.img ? k_raster_bwd<TS, NT, BATCH, true, true, kLayoutCta, true>
                                  : k_raster_bwd<TS, NT, BATCH, false, true, kLayoutCta, true>)
                        : (bl.img ? k_raster_bwd<TS, NT, BATCH, true, false, kLayoutCta, true>
                                  : k_raster_bwd<TS, NT, BATCH, false, false, kLayoutCta, true>);
    } else {
      return bwd_launch<TS, NT, 128>(n_tiles, persistent, layout, col_by_record, det, ws, tile_desc, n_pos, pair_face,
                                     views, C, F, bg, dL, dLdT, bl, bz, s);
    }
  }
  if constexpr ((TS == 16 && (NT == 128 || NT == 256)) || (TS == 8 && (NT == 32 || NT == 64))) {
    if (layout == kLayoutHalf)
      kern = bl.img ? k_raster_bwd<TS, NT, BATCH, true, false, kLayoutHalf>
                    : k_raster_bwd<TS, NT, BATCH, false, false, kLayoutHalf>;
  } else {
    if (layout == kLayoutHalf) return cudaErrorInvalidValue;
  }
  if constexpr (BATCH == 256) {  // (the warp-staged layout has no batch)
    if (layout == kLayoutWarp)
      kern = bl.img ? k_raster_bwd<TS, NT, 256, true, false, kLayoutWarp>
                    : k_raster_bwd<TS, NT, 256, false, false, kLayoutWarp>;
  } else {
    if (layout == kLayoutWarp) return bwd_launch<TS, NT, 256>(n_tiles, persistent, layout, col_by_record, det, ws,
                                                              tile_desc, n_pos, pair_face, views, C, F, bg, dL, dLdT,
                                                              bl, bz, s);
  }
  const unsigned grid = persistent ? (unsigned)std::min<int64_t>(n_pos, resident_grid(kern, NT)) : (unsigned)n_pos;
  return launch_chained(kern, false, dim3(grid), dim3(NT), 0, s,
                        raster_args(ws, tile_desc, n_pos, pair_face, views, F, bg, col_by_record), dL, dLdT,
                        (const float*)ws.pix_T, (const uint32_t*)ws.pix_last, ws.rec_grad,
                        col_by_record ? ws.rec_cgrad : ws.face_grad, bl, bz);
}

}  // namespace

cudaError_t launch_raster_fwd(int tile, int threads, int batch, bool persistent, int layout, bool col_by_record,
                              const Workspace& ws, const uint4* tile_desc, int64_t n_pos,
                              const uint32_t* pair_face, const ViewInfo* views, int32_t C, int32_t F,
                              int64_t n_tiles, const float* bg, float* images, float* t_final_out,
                              uint32_t* ncontrib_out, const FwdLoss& fl, cudaStream_t s, int64_t* launches) {
  if (n_tiles <= 0) return fl.target ? cudaMemsetAsync(fl.loss, 0, sizeof(double), s) : cudaSuccess;
  if (fl.target) *launches += 1;  // k_sum_partials
  cudaError_t e = cudaSuccess;
#define GMR_FWD(TS_, NT_, B_)                                                                                    \
  if (tile == TS_ && threads == NT_ && batch == B_)                                                              \
  e = fwd_launch<TS_, NT_, B_>(n_tiles, persistent, layout, col_by_record, ws, tile_desc, n_pos, pair_face, views,  \
                               C, F, bg, images,                                                                 \
                               t_final_out,                                                                      \
                               ncontrib_out, fl, s)
  GMR_FWD(16, 256, 64); else GMR_FWD(16, 256, 128); else GMR_FWD(16, 256, 256);
  else GMR_FWD(16, 128, 64); else GMR_FWD(16, 128, 128); else GMR_FWD(16, 128, 256);
  else GMR_FWD(16, 64, 64); else GMR_FWD(16, 64, 128); else GMR_FWD(16, 64, 256);
  else GMR_FWD(32, 256, 64); else GMR_FWD(32, 256, 128); else GMR_FWD(32, 256, 256);
  else GMR_FWD(8, 64, 64); else GMR_FWD(8, 64, 128); else GMR_FWD(8, 64, 256);
  else GMR_FWD(8, 32, 64); else GMR_FWD(8, 32, 128); else GMR_FWD(8, 32, 256);
  else return cudaErrorInvalidValue;
#undef GMR_FWD
  *launches += 1;
  return e;
}

cudaError_t launch_raster_bwd(int tile, int threads, int batch, bool persistent, int layout, bool col_by_record,
                              bool det, const Workspace& ws, const uint4* tile_desc, int64_t n_pos,
                              const uint32_t* pair_face, const ViewInfo* views, int32_t C, int32_t F,
                              int64_t n_tiles, const float* bg, const float* dL_dimages, const float* dL_dT,
                              const BwdLoss& bl, const BwdZero& bz, cudaStream_t s, int64_t* launches) {
  if (n_tiles <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
#define GMR_BWD(TS_, NT_, B_)                                                                                    \
  if (tile == TS_ && threads == NT_ && batch == B_)                                                              \
  e = bwd_launch<TS_, NT_, B_>(n_tiles, persistent, layout, col_by_record, det, ws, tile_desc, n_pos, pair_face,   \
                               views, C, F, bg,                                                                  \
                               dL_dimages,                                                                       \
                               dL_dT, bl, bz, s)
  GMR_BWD(16, 256, 64); else GMR_BWD(16, 256, 128); else GMR_BWD(16, 256, 256);
  else GMR_BWD(16, 128, 64); else GMR_BWD(16, 128, 128); else GMR_BWD(16, 128, 256);
  else GMR_BWD(16, 64, 64); else GMR_BWD(16, 64, 128); else GMR_BWD(16, 64, 256);
  else GMR_BWD(32, 256, 64); else GMR_BWD(32, 256, 128); else GMR_BWD(32, 256, 256);
  else GMR_BWD(8, 64, 64); else GMR_BWD(8, 64, 128); else GMR_BWD(8, 64, 256);
  else GMR_BWD(8, 32, 64); else GMR_BWD(8, 32, 128); else GMR_BWD(8, 32, 256);
  else return cudaErrorInvalidValue;
#undef GMR_BWD
  *launches += 1;
  return e;
}

cudaError_t launch_debug_records(const Workspace& ws, int64_t n_rec, int32_t* rects, float* conic, cudaStream_t s,
                                 int64_t* launches) {
  if (n_rec <= 0) return cudaSuccess;
  k_debug_records<<<(unsigned)((n_rec + 255) / 256), 256, 0, s>>>(ws.rec_rect, ws.rec_uq, n_rec, rects, conic);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_sum_floats(const float* x, int64_t n, double scale, double* out, cudaStream_t s,
                              int64_t* launches) {
  cudaError_t e = launch_chained(k_sum_partials, true, dim3(1), dim3(1024), 0, s, x, n, scale, out);
  *launches += 1;
  return e;
}

// Silhouette loss (Sec. 3.1: binary cross-entropy between the rendered mask
// and the target silhouette), mask M = 1 - T_final clamped to
// [kBceEps, 1 - kBceEps]: L = -(1/n) sum (m log M + (1 - m) log(1 - M)),
// dL/dT_final = (1/n) (m / M - (1 - m) / (1 - M)) where M is not clamped, 0
// where it is, both times a weight. 1 - M is taken as T itself (no
// cancellation).
constexpr float kBceEps = 1e-6f;
constexpr int kBceItems = 16;

__global__ void __launch_bounds__(kLossThreads) k_silhouette_bce(const float* __restrict__ t_final,
                                                                  const float* __restrict__ mask, int64_t n,
                                                                  float inv_n, float weight, float* __restrict__ dL_dT,
                                                                  double* __restrict__ part, double* __restrict__ loss) {
  const int64_t base = (int64_t)blockIdx.x * kLossThreads * kBceItems;
  float acc = 0.0f;
#pragma unroll 4
  for (int k = 0; k < kBceItems; ++k) {
    const int64_t i = base + (int64_t)k * kLossThreads + threadIdx.x;
    if (i < n) {
      const float T = t_final[i], m = mask[i];
      const float Mraw = 1.0f - T;
      const float M = fminf(fmaxf(Mraw, kBceEps), 1.0f - kBceEps);
      const float Tc = fminf(fmaxf(T, kBceEps), 1.0f - kBceEps);  // 1 - M
      acc -= m * logf(M) + (1.0f - m) * logf(Tc);
      const bool inside = Mraw > kBceEps && Mraw < 1.0f - kBceEps;
      dL_dT[i] = inside ? weight * inv_n * (m / M - (1.0f - m) / Tc) : 0.0f;
    }
  }
  // the loss is the mean: scale the FP32 partial here (exact power-of-two
  // scalings aside, one rounding per thread)
  loss_partial_and_finish<kLossThreads>(acc * (weight * inv_n), part, loss);
}

int64_t bce_partials_needed(int64_t n) { return 1 + (n + kLossThreads * kBceItems - 1) / (kLossThreads * kBceItems); }

cudaError_t launch_silhouette_bce(const float* t_final, const float* mask, int64_t n, float weight, float* dL_dT,
                                  double* loss, double* partials, int64_t n_partials, cudaStream_t s,
                                  int64_t* launches) {
  const int64_t nb = bce_partials_needed(n) - 1;
  if (nb + 1 > n_partials) return cudaErrorInvalidValue;
  if (nb == 0) return cudaMemsetAsync(loss, 0, sizeof(double), s);
  k_silhouette_bce<<<(unsigned)nb, kLossThreads, 0, s>>>(t_final, mask, n, 1.0f / (float)n, weight, dL_dT, partials,
                                                          loss);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_l2_loss(const float* img, const float* target, int64_t n, float* grad, double* loss,
                           double* partials, int64_t n_partials, cudaStream_t s, int64_t* launches) {
  const int64_t nb = l2_loss_partials_needed(n) - 1;
  if (nb + 1 > n_partials) return cudaErrorInvalidValue;
  if (nb == 0) return cudaMemsetAsync(loss, 0, sizeof(double), s);
  const bool vec4 = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(target) |
                      reinterpret_cast<uintptr_t>(grad)) & 15u) == 0;
  k_l2_loss<<<(unsigned)nb, kLossThreads, 0, s>>>(img, target, n, grad, partials, loss, vec4);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace gmr
