// Mesh-to-Gaussian conversion (Sec. 2.2) fused with EWA projection
// (Sec. 2.1), its backward, and the standalone conversion.
//
// Closed form used on the device. For a facet with vertices v_a (a = 0, 1,
// 2), centroid mu and d_a = v_a - mu, the uniform density of Eq. 6-8 has
// second moment Sigma_raw = (1/12) sum_a d_a d_a^T, which equals
// R_f blkdiag(Sigma2D, 0) R_f^T of Eq. 15 (the moments of Eq. 9 written
// without the facet frame). Its in-plane eigenvalues satisfy
// lambda1 lambda2 = det Sigma2D = |A|^2 / 108, so the area-matching factor
// of Eq. 12 is the constant kappa = 6 sqrt(3) / pi unless |A|^2 / 108 falls
// below eps = 1e-14, and Eq. 13 (via Eq. 14) becomes
//   Sigma_f = kappa Sigma_raw + s_z^2 n n^T.
// Projected through M = J R (J the EWA Jacobian at the camera-space mean):
//   Sigma' = (kappa/12) sum_a e_a e_a^T + s_z^2 m m^T + 0.3 I,
//   e_a = M d_a, m = M n,
// whose determinant is formed from squared 2D cross products (Cauchy-Binet),
// a sum of non-negative terms, so edge-on facets lose no precision.
// The image-plane mean is evaluated in double-float arithmetic (pairs of
// floats, error-free transformations) and stored as a float pair so that pixel
// offsets keep ~1e-6 px accuracy at any image size; FP64 is not used.

#include <algorithm>

#include "gmr_internal.cuh"

namespace gmr {

namespace {

struct FaceGeom {
  float3 v0, v1, v2;
  float3 e1, e2;      // v1 - v0, v2 - v0
  float3 d[3];        // v_a - centroid
  float3 n;           // unit normal (0 for a degenerate facet)
  float cn;           // |e1 x e2| = 2 |A|
  float w;            // kappa / 12
  float sz2;          // s_z^2
  bool clamped;       // Eq. 12 epsilon clamp active
  float mx, my, mz;   // centroid (rounded)
};

__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 f3add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 f3scale(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// GMR_FLAG_DETERMINISTIC: the compositing backward's sums of each pair are
// in the pair's slot, and a record's pairs sit in consecutive slots from
// rec_slot[rid], in the order of its tiles; record_sums adds them in that
// order. pair_grad == nullptr: not in this mode.
struct DetSums {
  const float4* pair_grad = nullptr;
  const uint32_t* rec_slot = nullptr;
  const uint32_t* rec_ntiles = nullptr;
  int64_t cap_pairs = 0;
  float4* corner_grad = nullptr;  // out: 4 per face (three corners' dL/dv, colour share)
  // r0 = (sum q dx, sum q dy, sum q dx^2, sum q dx dy), r4 = sum q dy^2,
  // cg = (dr, dg, db, sum dq) of record rid
  __device__ __forceinline__ void record_sums(size_t rid, float4& r0, float& r4, float4& cg) const {
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    cg = r0;
    r4 = 0.f;
    const uint32_t n = __ldg(rec_ntiles + rid);
    if (n == 0) return;
    const int64_t s0 = __ldg(rec_slot + rid);
    if (s0 + n > cap_pairs) return;  // pair overflow (reported by the forward): no sums
    for (uint32_t k = 0; k < n; ++k) {
      const float4 a = __ldg(pair_grad + 3 * (s0 + k));
      const float4 b = __ldg(pair_grad + 3 * (s0 + k) + 1);
      const float c = __ldg(pair_grad + 3 * (s0 + k) + 2).x;
      r0 = f4add(r0, a);
      r4 += b.x;
      cg = f4add(cg, make_float4(b.z, b.w, c, b.y));
    }
  }
};
__device__ __forceinline__ float3 f3cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// (a + b + c) / 3 of three floats as a double-float.
__device__ __forceinline__ df df_mean3(float a, float b, float c) {
  df s1 = two_sum(a, b);
  df s = df_add(df{s1.hi, s1.lo}, df{c, 0.0f});
  float q = __fdiv_rn(s.hi, 3.0f);
  float r = __fmaf_rn(-3.0f, q, s.hi);  // exact remainder
  return fast_two_sum(q, __fdiv_rn(__fadd_rn(r, s.lo), 3.0f));
}

__device__ __forceinline__ FaceGeom face_geom(float3 a, float3 b, float3 c, int cov_mode) {
  FaceGeom g;
  g.v0 = a; g.v1 = b; g.v2 = c;
  g.e1 = f3sub(b, a);
  g.e2 = f3sub(c, a);
  g.d[0] = f3scale(-1.0f / 3.0f, f3add(g.e1, g.e2));
  g.d[1] = f3add(g.d[0], g.e1);
  g.d[2] = f3add(g.d[0], g.e2);
  float3 cr = f3cross(g.e1, g.e2);
  g.cn = sqrtf(f3dot(cr, cr));
  g.n = g.cn > 0.0f ? f3scale(1.0f / g.cn, cr) : make_float3(0.f, 0.f, 0.f);
  // The FP32 cross product of nearly parallel edges is cancellation noise,
  // and near the Eq. 12 clamp kappa is proportional to |A|: there, redo it in
  // FP64 from the exact vertex differences (rare, so FP64 costs nothing).
  float scale = sqrtf(f3dot(g.e1, g.e1) * f3dot(g.e2, g.e2));
  if (g.cn < 1e-3f * scale || g.cn < 8e-6f) {
    double ax = a.x, ay = a.y, az = a.z;
    double p1 = (double)b.x - ax, p2 = (double)b.y - ay, p3 = (double)b.z - az;
    double q1 = (double)c.x - ax, q2 = (double)c.y - ay, q3 = (double)c.z - az;
    double r1 = p2 * q3 - p3 * q2, r2 = p3 * q1 - p1 * q3, r3 = p1 * q2 - p2 * q1;
    double rn = sqrt(r1 * r1 + r2 * r2 + r3 * r3);
    g.cn = (float)rn;
    g.n = rn > 0.0 ? make_float3((float)(r1 / rn), (float)(r2 / rn), (float)(r3 / rn)) : make_float3(0.f, 0.f, 0.f);
  }
  if (cov_mode == GMR_COV_AREA) {
    float area = 0.5f * g.cn;
    // Eq. 12 with lambda1 lambda2 = |A|^2 / 108
    g.clamped = (area * area) < 108.0f * kEps;
    float kappa = g.clamped ? area / (kPi * 1e-7f) : kKappa;
    g.w = kappa * (1.0f / 12.0f);
    g.sz2 = kSz * kSz;
  } else {
    g.clamped = false;
    g.w = 1.0f / 12.0f;
    g.sz2 = 0.0f;
  }
  g.mx = (a.x + b.x + c.x) * (1.0f / 3.0f);
  g.my = (a.y + b.y + c.y) * (1.0f / 3.0f);
  g.mz = (a.z + b.z + c.z) * (1.0f / 3.0f);
  return g;
}

struct ProjRec {
  float tx, ty, tz;       // camera-space mean
  float J00, J02, J11, J12;
  float M[6];             // J R, row-major 2x3
  float2 e[3];            // M d_a
  float2 m;               // M n
  float kxx, kxy, kyy;    // Sigma' - 0.3 I
  float qa, qb, qc;       // conic
};

// Image-plane mean u = (fx x/z + cx, fy y/z + cy) of the centroid m (the
// double-float mean of the FP32 vertices, df_mean3) in double-float
// arithmetic.
__device__ __forceinline__ void image_mean(const df m[3], const ViewInfo& v, df& ux, df& uy) {
  df t[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    df acc = {v.t[r], 0.0f};
#pragma unroll
    for (int q = 0; q < 3; ++q) acc = df_add(acc, df_mul_f(m[q], v.R[3 * r + q]));
    t[r] = acc;
  }
  df xz = df_div(t[0], t[2]), yz = df_div(t[1], t[2]);
  ux = df_add(df_mul_f(xz, v.fx), df{v.cx, 0.0f});
  uy = df_add(df_mul_f(yz, v.fy), df{v.cy, 0.0f});
}

__device__ __forceinline__ ProjRec project_rec(const FaceGeom& g, const ViewInfo& v) {
  ProjRec p;
  const float* R = v.R;
  p.tx = R[0] * g.mx + R[1] * g.my + R[2] * g.mz + v.t[0];
  p.ty = R[3] * g.mx + R[4] * g.my + R[5] * g.mz + v.t[1];
  p.tz = R[6] * g.mx + R[7] * g.my + R[8] * g.mz + v.t[2];
  const float iz = 1.0f / p.tz;
  const float xz = p.tx * iz, yz = p.ty * iz;
  p.J00 = v.fx * iz;
  p.J11 = v.fy * iz;
  p.J02 = -v.fx * xz * iz;
  p.J12 = -v.fy * yz * iz;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    p.M[q] = p.J00 * R[q] + p.J02 * R[6 + q];
    p.M[3 + q] = p.J11 * R[3 + q] + p.J12 * R[6 + q];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p.e[a].x = p.M[0] * g.d[a].x + p.M[1] * g.d[a].y + p.M[2] * g.d[a].z;
    p.e[a].y = p.M[3] * g.d[a].x + p.M[4] * g.d[a].y + p.M[5] * g.d[a].z;
  }
  p.m.x = p.M[0] * g.n.x + p.M[1] * g.n.y + p.M[2] * g.n.z;
  p.m.y = p.M[3] * g.n.x + p.M[4] * g.n.y + p.M[5] * g.n.z;
  float sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    sxx += p.e[a].x * p.e[a].x;
    sxy += p.e[a].x * p.e[a].y;
    syy += p.e[a].y * p.e[a].y;
  }
  p.kxx = g.w * sxx + g.sz2 * p.m.x * p.m.x;
  p.kxy = g.w * sxy + g.sz2 * p.m.x * p.m.y;
  p.kyy = g.w * syy + g.sz2 * p.m.y * p.m.y;
  // det(K) by Cauchy-Binet over the four rank-one terms
  float c01 = p.e[0].x * p.e[1].y - p.e[0].y * p.e[1].x;
  float c02 = p.e[0].x * p.e[2].y - p.e[0].y * p.e[2].x;
  float c12 = p.e[1].x * p.e[2].y - p.e[1].y * p.e[2].x;
  float cm = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float t = p.e[a].x * p.m.y - p.e[a].y * p.m.x;
    cm += t * t;
  }
  float detK = g.w * g.w * (c01 * c01 + c02 * c02 + c12 * c12) + g.w * g.sz2 * cm;
  float det = detK + kDilation * (p.kxx + p.kyy) + kDilation * kDilation;
  float inv = 1.0f / det;
  p.qa = (p.kyy + kDilation) * inv;
  p.qb = -p.kxy * inv;
  p.qc = (p.kxx + kDilation) * inv;
  return p;
}

__device__ __forceinline__ bool load_face(const int32_t* faces, int f, int V, int& i0, int& i1, int& i2) {
  i0 = __ldg(faces + 3 * f);
  i1 = __ldg(faces + 3 * f + 1);
  i2 = __ldg(faces + 3 * f + 2);
  return (unsigned)i0 < (unsigned)V && (unsigned)i1 < (unsigned)V && (unsigned)i2 < (unsigned)V;
}

// ---------------------------------------------------------------- kernels

constexpr int kProjThreads = 128;
constexpr int kPairUnroll = 2;  // swept 1, 2, 4, 8: 2 is best over the workloads (8% faster than 4 on 1.3M faces)

// One thread per (face, view): binning spec, depth key, tile rectangle and
// one count per tile of the rectangle, and the precise record (image mean as
// a float pair, pre-scaled conic). The view-0 threads also write the face's
// colour (Eq. 16 in per-vertex mode) and clamped opacity.
__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// View-dependent colour of the facet with vertices a, b, c in view v
// (GMR_COLOR_SH, degree L): max(0, sum_k a_k Y_k(d) + 1/2), d the unit vector
// from the camera centre to the centroid; coef holds the facet's K x 3
// coefficients.
template <int L>
__device__ __forceinline__ float3 sh_colour(const float* __restrict__ coef, float3 a, float3 b, float3 c,
                                            const ViewInfo& v) {
  constexpr int K = (L + 1) * (L + 1);
  const float wx = (a.x + b.x + c.x) * (1.0f / 3.0f) - v.o[0];
  const float wy = (a.y + b.y + c.y) * (1.0f / 3.0f) - v.o[1];
  const float wz = (a.z + b.z + c.z) * (1.0f / 3.0f) - v.o[2];
  const float rinv = 1.0f / sqrtf(wx * wx + wy * wy + wz * wz);
  float Y[K];
  sh_eval<L>(wx * rinv, wy * rinv, wz * rinv, Y);
  float r = 0.5f, g = 0.5f, bl = 0.5f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    r += __ldg(coef + 3 * k) * Y[k];
    g += __ldg(coef + 3 * k + 1) * Y[k];
    bl += __ldg(coef + 3 * k + 2) * Y[k];
  }
  return make_float3(fmaxf(r, 0.0f), fmaxf(g, 0.0f), fmaxf(bl, 0.0f));
}

__device__ __forceinline__ float3 sh_colour_any(int L, const float* __restrict__ coef, float3 a, float3 b, float3 c,
                                                const ViewInfo& v) {
  switch (L) {
    case 0: return sh_colour<0>(coef, a, b, c, v);
    case 1: return sh_colour<1>(coef, a, b, c, v);
    case 2: return sh_colour<2>(coef, a, b, c, v);
    default: return sh_colour<3>(coef, a, b, c, v);
  }
}

// One thread per face and view block: grid.y splits the views into blocks
// of up to kProjMaxVpt (vpt views per block, so that there are enough threads
// for small meshes), and a thread loads its face and vertices and forms the
// centroids and the facet geometry once for all views of its block (64-view
// workload: projection 0.63 -> 0.30 ms; 1.31M faces x 16 views: 1.31 -> 0.84
// ms). Per (view, face) record: binning spec,
// depth key, tile rectangle and one count per tile of the rectangle, and the
// precise record (image mean as a float pair, pre-scaled conic, skip
// threshold). The first view block also writes the face's colour (Eq. 16 in
// per-vertex mode) and clamped opacity.
constexpr int kProjMaxVpt = 32;

// (8 resident CTAs per SM: at most 64 registers; the compiler's 80 allowed 6,
// and the latency of the tile-rank atomics wants the extra warps: 6% faster
// on the 64-view and ring workloads)
__global__ void __launch_bounds__(kProjThreads, 8) k_project(
    const float4* __restrict__ verts, int32_t V, const int32_t* __restrict__ faces, int32_t F, int32_t C, int vpt,
    const float* __restrict__ rgb, const float* __restrict__ opacity, int color_mode, int sh_degree,
    float4* __restrict__ rec_col, float4* __restrict__ rec_cgrad,
    const ViewInfo* __restrict__ views, int tile, float inv_tile, int bshift, int cov_mode, float4* __restrict__ rec_uq,
    uint2* __restrict__ rec_rect, uint32_t* __restrict__ rec_ntiles,
    uint32_t* __restrict__ rec_key, uint32_t* __restrict__ tile_count, float4* __restrict__ face_col,
    int64_t cap_pairs, unsigned long long* __restrict__ pair_tr, uint32_t* __restrict__ pair_rec,
    uint8_t* __restrict__ pair_quad, uint32_t* __restrict__ rec_slot, float4* __restrict__ rec_grad,
    float4* __restrict__ face_grad, Counters* __restrict__ counters) {
  pdl_enter();
  __shared__ ViewInfo sv[kProjMaxVpt];
  __shared__ uint32_t s_off[kProjThreads / 32][32];
  __shared__ uint2 s_first[kProjThreads / 32][32];  // (first tile, rectangle width)
  __shared__ uint2 s_rect[kProjThreads / 32][32];   // split binning: the rectangle on the 8x8 grid
  const int c0 = blockIdx.y * vpt;
  const int nv = min(vpt, C - c0);
  for (int i = threadIdx.x; i < nv; i += kProjThreads) sv[i] = views[c0 + i];
  __syncthreads();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = f < F;
  int i0 = 0, i1 = 0, i2 = 0;
  const bool ok = live && load_face(faces, f, V, i0, i1, i2);
  const bool sh_col = color_mode == GMR_COLOR_SH;
  if (live && c0 == 0 && !sh_col) {
    face_grad[f] = make_float4(0.f, 0.f, 0.f, 0.f);  // the backward's sums start at zero
    float r = 0.f, g = 0.f, b = 0.f;
    if (color_mode == GMR_COLOR_PER_FACE) {
      r = __ldg(rgb + 3 * f); g = __ldg(rgb + 3 * f + 1); b = __ldg(rgb + 3 * f + 2);
    } else if (ok) {
      r = (__ldg(rgb + 3 * i0) + __ldg(rgb + 3 * i1) + __ldg(rgb + 3 * i2)) * (1.0f / 3.0f);
      g = (__ldg(rgb + 3 * i0 + 1) + __ldg(rgb + 3 * i1 + 1) + __ldg(rgb + 3 * i2 + 1)) * (1.0f / 3.0f);
      b = (__ldg(rgb + 3 * i0 + 2) + __ldg(rgb + 3 * i1 + 2) + __ldg(rgb + 3 * i2 + 2)) * (1.0f / 3.0f);
    }
    float o = opacity ? __ldg(opacity + f) : 1.0f;
    o = fminf(fmaxf(o, 0.0f), 1.0f);
    face_col[f] = make_float4(r, g, b, o);
  }
  if (live && !ok && c0 == 0) atomicOr(&counters->status, kDevBadFace);
  // the face's view-independent quantities, once for all views
  float3 a = make_float3(0.f, 0.f, 0.f), b = a, cc = a;
  if (ok) {
    a = ld_vert4(verts, i0);
    b = ld_vert4(verts, i1);
    cc = ld_vert4(verts, i2);
  }
  const BinFace bf = bin_face(a, b, cc);
  const df m[3] = {df_mean3(a.x, b.x, cc.x), df_mean3(a.y, b.y, cc.y), df_mean3(a.z, b.z, cc.z)};
  const FaceGeom gm = face_geom(a, b, cc, cov_mode);
  // w of the record: the compositing's skip threshold t2 = -log2(255 o)
  // (o G < 1/255 iff log2 G < t2; +inf for o = 0)
  const float o = fminf(fmaxf(opacity && live ? __ldg(opacity + f) : 1.0f, 0.0f), 1.0f);
  const float t2 = -(kLog2_255 + log2f(o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;

  for (int vi = 0; vi < nv; ++vi) {
    const int c = c0 + vi;
    const ViewInfo& v = sv[vi];
    const uint32_t rid = (uint32_t)c * (uint32_t)F + (uint32_t)f;
    if (live) {  // the backward's gradient sums of every record start at zero
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      rec_grad[2 * (size_t)rid] = z;
      rec_grad[2 * (size_t)rid + 1] = z;
      if (sh_col) rec_cgrad[rid] = z;
    }
    BinResult br;
    br.visible = false;
    br.depth = 0.f;
    br.x0 = 1; br.x1 = 0; br.y0 = 1; br.y1 = 0;
    if (ok) br = bin_view(bf, v, tile, inv_tile);
    uint32_t nt = 0;
    uint2 rect = make_uint2(1u, 1u);  // x0 = 1 > x1 = 0: empty
    int bx0 = 0, bx1 = 0, by0 = 0;  // the rectangle on the binning grid
    if (br.visible && br.x0 <= br.x1) {
      rect = make_uint2((uint32_t)br.x0 | ((uint32_t)br.x1 << 16), (uint32_t)br.y0 | ((uint32_t)br.y1 << 16));
      // (floor(a / 2t) = floor(floor(a / t) / 2), also clamped: the binning
      // tiles hold every compositing tile of the rectangle)
      bx0 = br.x0 >> bshift;
      bx1 = br.x1 >> bshift;
      by0 = br.y0 >> bshift;
      nt = (uint32_t)(bx1 - bx0 + 1) * (uint32_t)((br.y1 >> bshift) - by0 + 1);
    }
    // (record, tile) pairs: the warp takes a run of pair slots from a global
    // counter and deals its records' pairs out evenly over its lanes (pair p
    // to lane p % 32, its record found by binary search over the exclusive
    // pair offsets). Each pair's rank within its tile comes from the tile's
    // counter (lanes that hit the same tile in the same step combine into one
    // atomic; kPairUnroll steps are issued before their results are used, so
    // that the round trips overlap); slot, tile, rank and record go to the
    // pair scratch (slots beyond its capacity are dropped; the binning
    // reports that).
    {
      const uint32_t incl = warp_incl_scan_u32(nt, lane);
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      if (total > 0) {
        s_off[warp][lane] = incl - nt;
        s_first[warp][lane] = make_uint2((uint32_t)v.btile_base + (uint32_t)by0 * (uint32_t)v.btiles_x + (uint32_t)bx0,
                                         (uint32_t)(bx1 - bx0 + 1));
        if (pair_quad) s_rect[warp][lane] = rect;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&counters->pair_alloc, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (rec_slot && live && nt > 0) rec_slot[rid] = base + (incl - nt);  // this record's first slot
        __syncwarp();
        const uint32_t tx = (uint32_t)v.btiles_x;
        const uint32_t rid0 = rid - (uint32_t)lane;
        for (uint32_t p0 = 0; p0 < total; p0 += 32 * kPairUnroll) {
          uint32_t t[kPairUnroll], peers[kPairUnroll], old[kPairUnroll], own[kPairUnroll], quad[kPairUnroll];
#pragma unroll
          for (int u = 0; u < kPairUnroll; ++u) {
            const uint32_t p = p0 + 32u * u + lane;
            t[u] = 0xffffffffu - (uint32_t)lane;  // distinct dummies for idle lanes
            own[u] = 0;
            quad[u] = 0;
            if (p < total) {
              int q = 0;
#pragma unroll
              for (int st = 16; st > 0; st >>= 1)
                if (s_off[warp][q + st] <= p) q += st;
              const uint2 fr = s_first[warp][q];
              const uint32_t k = p - s_off[warp][q];
              const uint32_t row = k / fr.y;
              t[u] = fr.x + row * tx + (k - row * fr.y);
              own[u] = (uint32_t)q;
              if (pair_quad) {
                // which quadrants (8x8 tiles) of this binning tile the
                // record's 8x8 rectangle holds: bit qy * 2 + qx
                const uint2 r = s_rect[warp][q];
                const int x0 = (int)(r.x & 0xffffu), x1 = (int)(r.x >> 16);
                const int y0 = (int)(r.y & 0xffffu), y1 = (int)(r.y >> 16);
                const int X = 2 * ((x0 >> 1) + (int)(k - row * fr.y)), Y = 2 * ((y0 >> 1) + (int)row);
                const bool cx0 = X >= x0 && X <= x1, cx1 = X + 1 >= x0 && X + 1 <= x1;
                const bool cy0 = Y >= y0 && Y <= y1, cy1 = Y + 1 >= y0 && Y + 1 <= y1;
                quad[u] = (uint32_t)(cx0 && cy0) | (uint32_t)(cx1 && cy0) << 1 | (uint32_t)(cx0 && cy1) << 2 |
                          (uint32_t)(cx1 && cy1) << 3;
              }
            }
            peers[u] = __match_any_sync(0xffffffffu, t[u]);
          }
#pragma unroll
          for (int u = 0; u < kPairUnroll; ++u) {
            old[u] = 0;
            if (p0 + 32u * u + lane < total && (peers[u] & lt) == 0)
              old[u] = atomicAdd(&tile_count[t[u]], (uint32_t)__popc(peers[u]));
          }
#pragma unroll
          for (int u = 0; u < kPairUnroll; ++u) {
            const uint32_t p = p0 + 32u * u + lane;
            const uint32_t rank = __shfl_sync(0xffffffffu, old[u], __ffs(peers[u]) - 1) + __popc(peers[u] & lt);
            const int64_t slot = (int64_t)base + p;
            if (p < total && slot < cap_pairs) {
              pair_tr[slot] = ((unsigned long long)t[u] << 32) | rank;
              pair_rec[slot] = rid0 + own[u];
              if (pair_quad) pair_quad[slot] = (uint8_t)quad[u];
            }
          }
        }
      }
    }
    if (live) {
      if (!ok) {
        rec_key[rid] = 0xffffffffu;
        rec_ntiles[rid] = 0;
        rec_rect[rid] = make_uint2(1u, 1u);
      } else {
        rec_key[rid] = br.visible ? __float_as_uint(br.depth) : 0xffffffffu;
        rec_ntiles[rid] = nt;
        rec_rect[rid] = rect;
        if (nt > 0) {
          // (the facet geometry is recomputed per record: keeping it across the
          // views costs more registers than it saves)
          ProjRec p = project_rec(gm, v);
          df ux, uy;
          image_mean(m, v, ux, uy);
          rec_uq[2 * (size_t)rid] = make_float4(ux.hi, uy.hi, ux.lo, uy.lo);
          rec_uq[2 * (size_t)rid + 1] = make_float4(p.qa * kNegHalfLog2e, p.qb * kNegLog2e, p.qc * kNegHalfLog2e, t2);
          if (sh_col) {
            const float3 col = sh_colour_any(sh_degree, rgb + (size_t)f * 3 * (sh_degree + 1) * (sh_degree + 1), a,
                                             b, cc, v);
            rec_col[rid] = make_float4(col.x, col.y, col.z, o);
          }
        }
      }
    }
    __syncwarp();  // s_off / s_first are refilled for the next view
  }
}

// Backward of conversion + projection. A face's gradient sums over its
// views, per view: the record's sums R0..R4 from the compositing backward
// chained through the conic inverse, Sigma' = M Sigma M^T + 0.3 I, M = J R,
// J(t) and u(t), to dL/dmu, dL/dd_a (d_a = v_a - mu), dL/dn and
// dL/d(kappa/12).
struct FaceAcc {
  float3 dmu;
  float3 dd[3];
  float3 dn;
  float dw;
};

__device__ __forceinline__ void record_bwd(const FaceGeom& g, const ViewInfo& v, float4 r0, float r4, float4 cq,
                                           FaceAcc& acc) {
  const ProjRec p = project_rec(g, v);
  // p2 = a2 dx^2 + b2 dx dy + c2 dy^2 with dx = pixel - u: the mean gradient
  // is ln2 (2 a2 sum q dx + b2 sum q dy, b2 sum q dx + 2 c2 sum q dy), taken
  // with the conic the forward used
  const float dux = kLn2 * (2.0f * cq.x * r0.x + cq.y * r0.y);
  const float duy = kLn2 * (cq.y * r0.x + 2.0f * cq.z * r0.y);
  const float dqa = -0.5f * r0.z, dqb = -r0.w, dqc = -0.5f * r4;
  // dL/dSigma' = -Q G_Q Q with G_Q = [[dqa, dqb/2], [dqb/2, dqc]]
  const float g00 = dqa, g01 = 0.5f * dqb, g11 = dqc;
  const float t00 = p.qa * g00 + p.qb * g01, t01 = p.qa * g01 + p.qb * g11;
  const float t10 = p.qb * g00 + p.qc * g01, t11 = p.qb * g01 + p.qc * g11;
  const float s00 = -(t00 * p.qa + t01 * p.qb);
  const float s01 = -(t00 * p.qb + t01 * p.qc);
  const float s11 = -(t10 * p.qb + t11 * p.qc);
  // Sigma' = w sum e e^T + sz2 m m^T + 0.3 I
  float2 de[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    de[k].x = 2.f * g.w * (s00 * p.e[k].x + s01 * p.e[k].y);
    de[k].y = 2.f * g.w * (s01 * p.e[k].x + s11 * p.e[k].y);
    acc.dw += s00 * p.e[k].x * p.e[k].x + 2.f * s01 * p.e[k].x * p.e[k].y + s11 * p.e[k].y * p.e[k].y;
  }
  float2 dm;
  dm.x = 2.f * g.sz2 * (s00 * p.m.x + s01 * p.m.y);
  dm.y = 2.f * g.sz2 * (s01 * p.m.x + s11 * p.m.y);
  // e_a = M d_a, m = M n
  float dM[6];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float dq0 = dm.x * (&g.n.x)[q], dq1 = dm.y * (&g.n.x)[q];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dq0 += de[k].x * (&g.d[k].x)[q];
      dq1 += de[k].y * (&g.d[k].x)[q];
    }
    dM[q] = dq0;
    dM[3 + q] = dq1;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    acc.dd[k].x += p.M[0] * de[k].x + p.M[3] * de[k].y;
    acc.dd[k].y += p.M[1] * de[k].x + p.M[4] * de[k].y;
    acc.dd[k].z += p.M[2] * de[k].x + p.M[5] * de[k].y;
  }
  acc.dn.x += p.M[0] * dm.x + p.M[3] * dm.y;
  acc.dn.y += p.M[1] * dm.x + p.M[4] * dm.y;
  acc.dn.z += p.M[2] * dm.x + p.M[5] * dm.y;
  // M = J R: dJ = dM R^T (only the non-zero entries of J)
  const float* R = v.R;
  const float dJ00 = dM[0] * R[0] + dM[1] * R[1] + dM[2] * R[2];
  const float dJ02 = dM[0] * R[6] + dM[1] * R[7] + dM[2] * R[8];
  const float dJ11 = dM[3] * R[3] + dM[4] * R[4] + dM[5] * R[5];
  const float dJ12 = dM[3] * R[6] + dM[4] * R[7] + dM[5] * R[8];
  // J(t), u(t) -> dL/dt
  const float iz = 1.0f / p.tz;
  const float x = p.tx, y = p.ty;
  const float fxz2 = v.fx * iz * iz, fyz2 = v.fy * iz * iz;
  const float dtx = dJ02 * (-fxz2) + dux * v.fx * iz;
  const float dty = dJ12 * (-fyz2) + duy * v.fy * iz;
  const float dtz = dJ00 * (-fxz2) + dJ02 * (2.f * v.fx * x * iz * iz * iz) + dJ11 * (-fyz2) +
                    dJ12 * (2.f * v.fy * y * iz * iz * iz) - dux * v.fx * x * iz * iz - duy * v.fy * y * iz * iz;
  // t = R mu + t_cam
  acc.dmu.x += R[0] * dtx + R[3] * dty + R[6] * dtz;
  acc.dmu.y += R[1] * dtx + R[4] * dty + R[7] * dtz;
  acc.dmu.z += R[2] * dtx + R[5] * dty + R[8] * dtz;
}

// Sum over the G lanes of a group (butterfly: every lane ends with the same,
// order-independent total, so the result is deterministic).
template <int G>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// One group of G lanes per face (G a power of two <= 8): lane k of the group
// takes views k, k + G, ... (records with no gradient are skipped), the
// group sums its lanes, and its first lane maps the sums to the three
// vertices (d_a = v_a - mu with mu the vertex mean, n = e1 x e2 / |e1 x e2|,
// kappa = |A| / (pi 1e-7) when clamped) and scatters them; colour and
// opacity gradients are per face. No per-record intermediate goes through
// memory.
constexpr int kProjBwdThreads = 64;  // swept 64, 128, 256: 64 is best (13% faster than 128 on the ring workload)

// Colour chain of one record (GMR_COLOR_SH, degree L): colour = max(0, raw),
// raw = sum_k a_k Y_k(d) + 1/2 per channel, d = w / |w|, w = centroid - o.
// Adds g_ch Y_k to dcoef[k][ch] for the unclamped channels, and the
// direction's share (dL/dd projected on the tangent plane, over |w|) to
// dL/dmu.
template <int L>
__device__ __forceinline__ void sh_colour_bwd(const float* __restrict__ coef, const FaceGeom& g, const ViewInfo& v,
                                              float3 gc, float* dcoef, float3& dmu) {
  constexpr int K = (L + 1) * (L + 1);
  const float wx = g.mx - v.o[0], wy = g.my - v.o[1], wz = g.mz - v.o[2];
  const float rinv = 1.0f / sqrtf(wx * wx + wy * wy + wz * wz);
  const float dx = wx * rinv, dy = wy * rinv, dz = wz * rinv;
  float Y[K];
  sh_eval<L>(dx, dy, dz, Y);
  float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) raw[ch] += __ldg(coef + 3 * k + ch) * Y[k];
  const float gch[3] = {raw[0] > 0.0f ? gc.x : 0.0f, raw[1] > 0.0f ? gc.y : 0.0f, raw[2] > 0.0f ? gc.z : 0.0f};
  float sY[K];  // dL/dY_k
#pragma unroll
  for (int k = 0; k < K; ++k) {
    sY[k] = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      dcoef[3 * k + ch] += gch[ch] * Y[k];
      sY[k] += gch[ch] * __ldg(coef + 3 * k + ch);
    }
  }
  if (L == 0) return;
  const float3 dd = sh_grad_dot<L>(dx, dy, dz, sY);
  const float dot = dd.x * dx + dd.y * dy + dd.z * dz;
  dmu.x += (dd.x - dot * dx) * rinv;
  dmu.y += (dd.y - dot * dy) * rinv;
  dmu.z += (dd.z - dot * dz) * rinv;
}

// L: degree of the view-dependent colour (GMR_COLOR_SH), or -1 for a colour
// per face or per vertex.
template <int G, int L>
__global__ void __launch_bounds__(kProjBwdThreads) k_proj_bwd(
    const float4* __restrict__ verts, int32_t V, const int32_t* __restrict__ faces, int32_t F, int32_t C,
    const ViewInfo* __restrict__ views, int cov_mode, int color_mode, const float* __restrict__ rgb,
    const float* __restrict__ opacity, const float4* __restrict__ rec_grad, const float4* __restrict__ rec_uq,
    const float4* __restrict__ face_grad, const float4* __restrict__ rec_cgrad, float* __restrict__ dverts,
    float* __restrict__ drgb, float* __restrict__ dop, int accumulate, DetSums det) {
  pdl_enter();
  constexpr int K = L >= 0 ? (L + 1) * (L + 1) : 1;
  float dcoef[L >= 0 ? 3 * K : 1];
#pragma unroll
  for (int k = 0; k < (L >= 0 ? 3 * K : 1); ++k) dcoef[k] = 0.0f;
  float dq_sum = 0.0f;  // view-dependent colour: sum over the views of sum dq
  float4 fg_det = make_float4(0.f, 0.f, 0.f, 0.f);  // det: this lane's views' colour sums (dr, dg, db, dq)
  const int64_t gid = (int64_t)blockIdx.x * kProjBwdThreads + threadIdx.x;
  const int f = (int)(gid / G);
  const int sub = (int)(gid % G);
  // the first view's sums and conic are loaded before the face and its
  // vertices, the next view's before this view's arithmetic (the conic
  // too: 4-6% faster, though invisible records then load it for nothing)
  float4 r0n = make_float4(0.f, 0.f, 0.f, 0.f);
  float r4n = 0.f;
  float4 qn = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!det.pair_grad && f < F && sub < C) {
    r0n = rec_grad[2 * ((size_t)sub * F + f)];
    r4n = rec_grad[2 * ((size_t)sub * F + f) + 1].x;
    qn = rec_uq[2 * ((size_t)sub * F + f) + 1];
  }
  int i0 = 0, i1 = 0, i2 = 0;
  const bool ok = f < F && load_face(faces, f, V, i0, i1, i2);
  FaceAcc acc;
  acc.dmu = make_float3(0.f, 0.f, 0.f);
  acc.dd[0] = acc.dd[1] = acc.dd[2] = acc.dn = acc.dmu;
  acc.dw = 0.f;
  float3 a = acc.dmu, b = acc.dmu, cc = acc.dmu;
  FaceGeom g;
  if (ok) {
    a = ld_vert4(verts, i0);
    b = ld_vert4(verts, i1);
    cc = ld_vert4(verts, i2);
    g = face_geom(a, b, cc, cov_mode);
    for (int c = sub; c < C; c += G) {
      const size_t rid = (size_t)c * F + f;
      float4 r0 = r0n;
      float r4 = r4n;
      float4 qc = qn;
      float4 cgd;  // det: the record's colour sums
      if (det.pair_grad) {
        det.record_sums(rid, r0, r4, cgd);
        fg_det = f4add(fg_det, cgd);
        qc = rec_uq[2 * (size_t)rid + 1];
      } else if (c + G < C) {
        r0n = rec_grad[2 * (rid + (size_t)G * F)];
        r4n = rec_grad[2 * (rid + (size_t)G * F) + 1].x;
        qn = rec_uq[2 * (rid + (size_t)G * F) + 1];
      }
      const bool geo = !(r0.x == 0.f && r0.y == 0.f && r0.z == 0.f && r0.w == 0.f && r4 == 0.f);
      if (L >= 0) {
        const float4 cg = det.pair_grad ? cgd : rec_cgrad[rid];
        dq_sum += cg.w;
        if (cg.x != 0.f || cg.y != 0.f || cg.z != 0.f)
          sh_colour_bwd<L >= 0 ? L : 0>(rgb + (size_t)f * 3 * K, g, views[c], make_float3(cg.x, cg.y, cg.z), dcoef,
                                        acc.dmu);
      }
      if (geo) record_bwd(g, views[c], r0, r4, qc, acc);
    }
  }
  if (G > 1) {  // every lane of the warp takes part in the shuffles
    acc.dmu = make_float3(group_sum<G>(acc.dmu.x), group_sum<G>(acc.dmu.y), group_sum<G>(acc.dmu.z));
#pragma unroll
    for (int k = 0; k < 3; ++k)
      acc.dd[k] = make_float3(group_sum<G>(acc.dd[k].x), group_sum<G>(acc.dd[k].y), group_sum<G>(acc.dd[k].z));
    acc.dn = make_float3(group_sum<G>(acc.dn.x), group_sum<G>(acc.dn.y), group_sum<G>(acc.dn.z));
    acc.dw = group_sum<G>(acc.dw);
    if (L >= 0) {
#pragma unroll
      for (int k = 0; k < 3 * K; ++k) dcoef[k] = group_sum<G>(dcoef[k]);
      dq_sum = group_sum<G>(dq_sum);
    } else if (det.pair_grad) {
      fg_det = make_float4(group_sum<G>(fg_det.x), group_sum<G>(fg_det.y), group_sum<G>(fg_det.z),
                           group_sum<G>(fg_det.w));
    }
  }
  if (f >= F || sub != 0) return;
  if (!ok) {  // a face with an index outside [0, V): no gradient (written, unless accumulating)
    if (!accumulate) {
      if (drgb && L >= 0)
        for (int k = 0; k < 3 * K; ++k) drgb[(size_t)f * 3 * K + k] = 0.0f;
      else if (drgb && color_mode == GMR_COLOR_PER_FACE)
        drgb[3 * f] = drgb[3 * f + 1] = drgb[3 * f + 2] = 0.0f;
      if (dop && opacity) dop[f] = 0.0f;
    }
    return;
  }
  // to vertices: d_a = v_a - mu (mu = mean of v), n from e1 x e2
  const float3 sdd = f3add(f3add(acc.dd[0], acc.dd[1]), acc.dd[2]);
  float3 dv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dv[k] = f3add(f3scale(1.0f / 3.0f, f3sub(acc.dmu, sdd)), acc.dd[k]);
  if (g.cn > 0.f) {
    float3 dcr = f3scale(1.0f / g.cn, f3sub(acc.dn, f3scale(f3dot(g.n, acc.dn), g.n)));
    if (g.clamped) {
      // kappa = |A| / (pi 1e-7), |A| = cn / 2, w = kappa / 12
      const float dcn = acc.dw * (1.0f / 12.0f) * (0.5f / (kPi * 1e-7f));
      dcr = f3add(dcr, f3scale(dcn, g.n));
    }
    const float3 de1 = f3cross(g.e2, dcr);
    const float3 de2 = f3cross(dcr, g.e1);
    dv[0] = f3sub(dv[0], f3add(de1, de2));
    dv[1] = f3add(dv[1], de1);
    dv[2] = f3add(dv[2], de2);
  }
  const int idx[3] = {i0, i1, i2};
  const float4 fg = L >= 0 ? make_float4(0.f, 0.f, 0.f, dq_sum) : det.pair_grad ? fg_det : face_grad[f];
  if (det.pair_grad) {
    // the vertices' shares, gathered per vertex in face order afterwards
#pragma unroll
    for (int k = 0; k < 3; ++k) det.corner_grad[4 * (size_t)f + k] = make_float4(dv[k].x, dv[k].y, dv[k].z, 0.f);
    det.corner_grad[4 * (size_t)f + 3] =
        make_float4(fg.x * (1.0f / 3.0f), fg.y * (1.0f / 3.0f), fg.z * (1.0f / 3.0f), 0.f);
  } else if (dverts) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(dverts + 3 * idx[k], dv[k].x);
      atomicAdd(dverts + 3 * idx[k] + 1, dv[k].y);
      atomicAdd(dverts + 3 * idx[k] + 2, dv[k].z);
    }
  }
  if (drgb && L >= 0) {  // the coefficients' gradient, summed over the views (no atomics)
    float* dst = drgb + (size_t)f * 3 * K;
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) dst[k] = accumulate ? dst[k] + dcoef[k] : dcoef[k];
  } else if (drgb) {
    if (color_mode == GMR_COLOR_PER_FACE) {
      if (accumulate) {
        drgb[3 * f] += fg.x; drgb[3 * f + 1] += fg.y; drgb[3 * f + 2] += fg.z;
      } else {
        drgb[3 * f] = fg.x; drgb[3 * f + 1] = fg.y; drgb[3 * f + 2] = fg.z;
      }
    } else if (!det.pair_grad) {  // (det: gathered per vertex afterwards)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        atomicAdd(drgb + 3 * idx[k], fg.x * (1.0f / 3.0f));
        atomicAdd(drgb + 3 * idx[k] + 1, fg.y * (1.0f / 3.0f));
        atomicAdd(drgb + 3 * idx[k] + 2, fg.z * (1.0f / 3.0f));
      }
    }
  }
  if (dop && opacity) {
    const float o = opacity[f];
    // alpha = o G: dL/do = sum dalpha G = (sum dalpha alpha) / o; clamp to [0, 1]
    const float go = (o > 0.f && o <= 1.f) ? fg.w / o : 0.f;
    if (accumulate) dop[f] += go; else dop[f] = go;
  }
}

// Standalone conversion: means, 6 covariance entries, colour, opacity.
__global__ void k_convert(const float* __restrict__ verts, int32_t V, const int32_t* __restrict__ faces, int32_t F,
                          const float* __restrict__ rgb, const float* __restrict__ opacity, int cov_mode,
                          int color_mode, float* __restrict__ means, float* __restrict__ cov,
                          float* __restrict__ face_rgb, float* __restrict__ face_o, Counters* counters) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  int i0, i1, i2;
  if (!load_face(faces, f, V, i0, i1, i2)) {
    atomicOr(&counters->status, kDevBadFace);
    for (int k = 0; k < 3; ++k) {
      if (means) means[3 * f + k] = 0.f;
      if (face_rgb) face_rgb[3 * f + k] = 0.f;
    }
    if (cov) for (int k = 0; k < 6; ++k) cov[6 * f + k] = 0.f;
    if (face_o) face_o[f] = 0.f;
    return;
  }
  float3 a = ld_vert(verts, i0), b = ld_vert(verts, i1), c = ld_vert(verts, i2);
  FaceGeom g = face_geom(a, b, c, cov_mode);
  if (means) {
    // correctly rounded (to ~1e-14) centroid from its double-float value
    df mx = df_mean3(a.x, b.x, c.x), my = df_mean3(a.y, b.y, c.y), mz = df_mean3(a.z, b.z, c.z);
    means[3 * f] = mx.hi + mx.lo; means[3 * f + 1] = my.hi + my.lo; means[3 * f + 2] = mz.hi + mz.lo;
  }
  if (cov) {
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // degenerate facets (|A| = 0) get zero covariance (kappa = 0)
    float w = (g.cn > 0.f) ? g.w : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float3 d = g.d[k];
      s[0] += d.x * d.x; s[1] += d.x * d.y; s[2] += d.x * d.z;
      s[3] += d.y * d.y; s[4] += d.y * d.z; s[5] += d.z * d.z;
    }
    float3 n = g.n;
    cov[6 * f + 0] = w * s[0] + g.sz2 * n.x * n.x;
    cov[6 * f + 1] = w * s[1] + g.sz2 * n.x * n.y;
    cov[6 * f + 2] = w * s[2] + g.sz2 * n.x * n.z;
    cov[6 * f + 3] = w * s[3] + g.sz2 * n.y * n.y;
    cov[6 * f + 4] = w * s[4] + g.sz2 * n.y * n.z;
    cov[6 * f + 5] = w * s[5] + g.sz2 * n.z * n.z;
  }
  if (face_rgb) {
    for (int k = 0; k < 3; ++k) {
      float v = (color_mode == GMR_COLOR_PER_FACE)
                    ? rgb[3 * f + k]
                    : (rgb[3 * i0 + k] + rgb[3 * i1 + k] + rgb[3 * i2 + k]) * (1.0f / 3.0f);
      face_rgb[3 * f + k] = v;
    }
  }
  if (face_o) face_o[f] = fminf(fmaxf(opacity ? opacity[f] : 1.0f, 0.0f), 1.0f);
}

// The vertices padded to 16 bytes: one thread per vertex (a warp reads 384
// contiguous bytes and writes 512).
constexpr int kPadThreads = 256;
__global__ void __launch_bounds__(kPadThreads) k_pad_verts(const float* __restrict__ verts, int32_t V,
                                                           float4* __restrict__ verts4) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * kPadThreads + threadIdx.x;
  if (i < V) verts4[i] = make_float4(__ldg(verts + 3 * i), __ldg(verts + 3 * i + 1), __ldg(verts + 3 * i + 2), 0.0f);
}

}  // namespace

cudaError_t launch_project(const float* verts, int32_t V, const int32_t* faces, int32_t F, const float* rgb,
                           const float* opacity, int color_mode, int sh_degree, const ViewInfo* views, int32_t C,
                           int tile, int bshift, int cov_mode, bool det, Workspace& ws, cudaStream_t s,
                           int64_t* launches) {
  if (F <= 0 || C <= 0) return cudaSuccess;
  // views per thread: as many as keep about two threads per SM slot (148 SMs
  // x 2048) busy, at most kProjMaxVpt, spread evenly over the view blocks
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>((int64_t)F * C / (148 * 2048 * 2), kProjMaxVpt));
  const int n_blocks_y = (int)((C + want - 1) / want);
  const int vpt = (C + n_blocks_y - 1) / n_blocks_y;
  dim3 grid((F + kProjThreads - 1) / kProjThreads, n_blocks_y);
  if (ws.cap_verts4 < V) return cudaErrorInvalidValue;
  if (V > 0) {
    cudaError_t e = launch_chained(k_pad_verts, true, dim3((unsigned)((V + kPadThreads - 1) / kPadThreads)),
                                   dim3(kPadThreads), 0, s, verts, V, ws.verts4);
    *launches += 1;
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch_chained(k_project, true, grid, dim3(kProjThreads), 0, s, (const float4*)ws.verts4, V, faces,
                                 F, C, vpt, rgb,
                                 opacity,
                                 color_mode, sh_degree, ws.rec_col, ws.rec_cgrad, views, tile, 1.0f / (float)tile,
                                 bshift, cov_mode, ws.rec_uq,
                                 ws.rec_rect, ws.rec_ntiles, ws.rec_key, ws.tile_count, ws.face_col, ws.cap_pairs,
                                 ws.pair_key[1], ws.pair_face, bshift ? ws.pair_quad : nullptr,
                                 det ? ws.rec_slot : nullptr, ws.rec_grad, ws.face_grad, ws.counters);
  *launches += 1;
  return e;
}

cudaError_t launch_project_bwd(const float* verts, int32_t V, const int32_t* faces, int32_t F,
                               const ViewInfo* views, int32_t C, int cov_mode, int color_mode, int sh_degree,
                               const float* rgb, const float* opacity, bool det, const Workspace& ws,
                               float* dverts, float* drgb, float* dop, int accumulate, cudaStream_t s,
                               int64_t* launches) {
  if (F <= 0) return cudaSuccess;
  // lanes per face: enough threads to fill the GPU when faces are few, no
  // more lanes than views (more lanes than that repeat the per-face work and
  // measured slower: 1.8x on 1.3M faces x 16 views with G = 8 instead of 1)
  int G = 1;
  while (G < 8 && G < C && (int64_t)F * G < 148 * 2048) G <<= 1;
  const int64_t threads = (int64_t)F * G;
  const unsigned blocks = (unsigned)((threads + kProjBwdThreads - 1) / kProjBwdThreads);
  const int L = color_mode == GMR_COLOR_SH ? sh_degree : -1;
#define GMR_PB(G_) (L < 0 ? k_proj_bwd<G_, -1> : L == 0 ? k_proj_bwd<G_, 0> : L == 1 ? k_proj_bwd<G_, 1> \
                    : L == 2 ? k_proj_bwd<G_, 2> : k_proj_bwd<G_, 3>)
  auto kern = G == 1 ? GMR_PB(1) : G == 2 ? GMR_PB(2) : G == 4 ? GMR_PB(4) : GMR_PB(8);
#undef GMR_PB
  DetSums ds;
  if (det) {
    ds.pair_grad = ws.pair_grad;
    ds.rec_slot = ws.rec_slot;
    ds.rec_ntiles = ws.rec_ntiles;
    ds.cap_pairs = std::min(ws.cap_pairs, ws.cap_det_pairs);
    ds.corner_grad = ws.corner_grad;
  }
  cudaError_t e = launch_chained(kern, true, dim3(blocks), dim3(kProjBwdThreads), 0, s, (const float4*)ws.verts4, V,
                                 faces, F, C, views,
                                 cov_mode, color_mode, rgb, opacity, (const float4*)ws.rec_grad,
                                 (const float4*)ws.rec_uq, (const float4*)ws.face_grad, (const float4*)ws.rec_cgrad,
                                 dverts, drgb, dop, accumulate, ds);
  *launches += 1;
  if (e != cudaSuccess || !det) return e;
  // per-vertex sums over the incidence list (vertex gradients, and colour
  // gradients of a per-vertex colour)
  return launch_vertex_gather(faces, F, V, ws, dverts, color_mode == GMR_COLOR_PER_VERTEX ? drgb : nullptr,
                              accumulate, s, launches);
}

cudaError_t launch_convert(const float* verts, int32_t V, const int32_t* faces, int32_t F, const float* rgb,
                           const float* opacity, int cov_mode, int color_mode, float* means, float* cov,
                           float* face_rgb, float* face_o, Counters* counters, cudaStream_t s, int64_t* launches) {
  if (F <= 0) return cudaSuccess;
  k_convert<<<(F + 255) / 256, 256, 0, s>>>(verts, V, faces, F, rgb, opacity, cov_mode, color_mode, means, cov,
                                            face_rgb, face_o, counters);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace gmr
