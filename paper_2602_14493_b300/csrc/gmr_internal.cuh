// Internal declarations of the Gaussian Mesh Renderer CUDA library.
// Device helpers shared by the kernels, the per-view table, the workspace
// and the launchers' prototypes. Not part of the public ABI (include/gmr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "gmr.h"

namespace gmr {

// ---------------------------------------------------------------- constants
// 3DGS compositing constants (Sec. 2.1 renders with the standard 3DGS
// rasterizer; the values are that rasterizer's).
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;
// Eq. 12: epsilon clamp of lambda1 lambda2, and s_z.
constexpr float kEps = 1e-14f;
constexpr float kSz = 1e-6f;
constexpr float kPi = 3.14159265358979f;
// kappa = 6 sqrt(3) / pi when lambda1 lambda2 = |A|^2/108 >= eps.
constexpr float kKappa = 3.30797337f;
// Binning spec constants, FP32: 2 ln 255 and kappa / 18.
constexpr float kTwoLn255 = 11.0825271606445312f;
constexpr float kKappaOver18 = 0.18377630412578583f;
// -log2(e)/2, -log2(e), ln 2: the conic is stored pre-scaled so that
// o * 2^(a2 dx^2 + b2 dx dy + c2 dy^2) = o * exp(-1/2 d^T Q d).
constexpr float kNegHalfLog2e = -0.72134752044448170f;
constexpr float kNegLog2e = -1.44269504088896340f;
constexpr float kLn2 = 0.69314718055994531f;

constexpr int kMaxViews = 65535;

// ---------------------------------------------------------------- launch chain
// Programmatic dependent launch. The step's kernels are launched with
// launch_chained(kern, chained = true, ...): such a kernel may be scheduled
// while the kernel before it on the stream is still running, and its CTAs
// then block in pdl_enter() until that kernel has completed and its writes
// are visible. So pdl_enter() is the first statement of every kernel of the
// step (before any global access, and before any early return: a kernel's
// completion then implies that of every kernel before it). The kernel also
// releases its own dependent at once: the dependent's CTAs take SM slots
// only as this kernel's CTAs retire (all of them have started by then),
// which hides the launch latency and the tail between two kernels. Without
// the launch attribute both instructions do nothing.
// Kernels whose CTAs take tiles heaviest first (the per-tile sort and the
// two compositing kernels) are launched with chained = false: an early
// launch places their first, heaviest CTAs on whichever SMs free up first,
// several to one SM, and their tail grows (the level-8 mesh step: +10%).
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Whether launch_chained() sets the attribute (GMR_PDL=0 in the environment
// turns it off; read once).
bool chained_launch_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kern)(KArgs...), bool chained, dim3 grid, dim3 block, size_t smem,
                           cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained && chained_launch_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- view table
struct ViewInfo {
  float R[9];
  float t[3];
  float fx, fy, cx, cy, znear;
  float o[3];  // camera centre in world coordinates, -R^T t
  int32_t W, H, tiles_x, tiles_y;
  int32_t tile_base;  // first global tile id of this view
  // the binning grid: the compositing tiles themselves, or (8x8 compositing
  // tiles, split binning) 16x16 tiles whose sorted lists are split into
  // their four 8x8 quadrants
  int32_t btiles_x, btiles_y, btile_base;
  int64_t pix_base;   // first packed pixel of this view
};
// Descriptor of a compositing position with no tile (a quadrant of a 16x16
// binning tile beyond the image's last 8x8 tile).
constexpr uint32_t kNoTile = 0xffffffffu;

// Device status bits (mirrors GMR_DEV_*).
constexpr uint32_t kDevBadFace = GMR_DEV_BAD_FACE_INDEX;
constexpr uint32_t kDevOverflow = GMR_DEV_PAIR_OVERFLOW;

// Device counters block.
struct Counters {
  // cleared together at the start of every forward (kFwdCountersBytes;
  // evals_bwd too, kStepCountersBytes, when the backward follows in order)
  uint32_t n_pairs;     // total pairs of the current forward (scan total)
  uint32_t pair_alloc;  // pair slots handed out by the projection
  uint32_t n_long;      // tiles whose segment is too long for a warp sort
  uint32_t long_next;   // k_long_sort's work cursor into the long-segment list
  unsigned long long evals_fwd;
  unsigned long long contribs;
  uint32_t n_class[16];  // tiles per work class (see tile_of_block); 16-byte aligned
  uint32_t raster_next_fwd;  // next compositing position of the persistent forward grid
  uint32_t pad0;
  // cleared at the start of every backward (kBwdCountersBytes from here)
  unsigned long long evals_bwd;
  uint32_t raster_next_bwd;  // next compositing position of the persistent backward grid
  uint32_t pad2;
  // GMR_DEV_* bits, sticky until gmr_get_device_status reads them
  uint32_t status;
  uint32_t pad1;
};
constexpr size_t kFwdCountersBytes = offsetof(Counters, evals_bwd);
constexpr size_t kStepCountersBytes = offsetof(Counters, status);
constexpr size_t kBwdCountersBytes = offsetof(Counters, status) - offsetof(Counters, evals_bwd);
static_assert(offsetof(Counters, n_class) % 16 == 0, "n_class is read with 16-byte loads");

// Compositing order of the tiles, heaviest first (a longest-job-first
// schedule: a heavy tile started late is what leaves SMs idle at the end of
// a compositing launch). The binning puts every tile in the work class of
// its pair count L, class 15 - bit_length(L) clamped to [0, 15] (so one
// class per power of two, empty tiles last), at an atomically taken
// position of that class's region of tile_order (regions of n_tiles
// entries; filed by the scan of the tile counts). The per-tile sort's warp
// w takes the w-th tile in class order and writes, at position w, the
// descriptor (tile, view, pair range) that compositing CTA w reads as its
// first load.
constexpr int kTileClasses = 16;
__device__ __forceinline__ int tile_class(uint32_t L) {
  const int bits = 32 - __clz((int)L);
  return kTileClasses - 1 - min(bits, kTileClasses - 1);
}
// Binary search of the view owning binning tile g.
__device__ __forceinline__ int find_view(const ViewInfo* views, int C, int g) {
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (views[mid].btile_base <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int tile_of_block(const uint32_t* __restrict__ tile_order,
                                             const uint32_t* __restrict__ n_class, int64_t n_tiles, int64_t b) {
  // the 16 class counts in four 16-byte loads issued together (n_class is
  // 16-byte aligned in the counters block)
  static_assert(kTileClasses == 16, "class counts are read as four uint4");
  const uint4* q = reinterpret_cast<const uint4*>(n_class);
  const uint4 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
  const uint32_t n[kTileClasses] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                                    q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
  int c = 0;
#pragma unroll
  for (int k = 0; k < kTileClasses - 1; ++k) {
    if (c == k && b >= (int64_t)n[k]) {
      b -= n[k];
      c = k + 1;
    }
  }
  return (int)tile_order[c * n_tiles + b];
}

// ---------------------------------------------------------------- helpers
// ---- double-float arithmetic (an unevaluated sum hi + lo of two floats) with
// the error-free transformations TwoSum (Knuth) and TwoProduct (by FMA); every
// operation is an explicit rounded intrinsic so that none is contracted or
// reassociated. Used for the image-plane mean, which must stay accurate to
// ~1e-6 px at any image size, and for the loss sums, while FP64 is a slow
// pipe on this GPU.
struct df {
  float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df qb = df_mul_f(b, q1);
  df r = df_add(a, df{-qb.hi, -qb.lo});
  float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 / a for a in [0.01, 1] (the 1 - alpha of compositing): the hardware
// approximation refined by one Newton-Raphson step for f(x) = 1/x - a,
// x1 = x0 + x0 (1 - a x0), which squares the relative error of x0 (to well
// under one ulp of FP32). The backward reconstructs the transmittance of
// every layer by repeated division, so the error per step compounds.
__device__ __forceinline__ float rcp_refined(float a) {
  float x0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x0) : "f"(a));
  const float e = __fmaf_rn(-a, x0, 1.0f);
  return __fmaf_rn(x0, e, x0);
}

__device__ __forceinline__ float3 ld_vert(const float* v, int i) {
  return make_float3(__ldg(v + 3 * i), __ldg(v + 3 * i + 1), __ldg(v + 3 * i + 2));
}
// A vertex of the forward's padded copy (one 16-byte load).
__device__ __forceinline__ float3 ld_vert4(const float4* v, int i) {
  const float4 p = __ldg(v + i);
  return make_float3(p.x, p.y, p.z);
}

// FP32 binning specification. Every operation is a separately rounded
// IEEE-754 single operation in a fixed order (the _rn intrinsics are never
// contracted), so the depth key and the tile rectangle are reproducible bit
// for bit by any IEEE implementation of the same sequence. The rectangle is
// conservative: it covers the bounding box (half-widths
// sqrt(2 ln 255 Sigma'_xx) + 0.25 px and sqrt(2 ln 255 Sigma'_yy) + 0.25 px,
// with the area scale kappa = 6 sqrt(3)/pi, the largest it takes) of the
// pixel centres where o * G can reach 1/255 for o <= 1, so the image does not
// depend on it.
struct BinResult {
  bool visible;
  float depth;
  int x0, x1, y0, y1;
};

__device__ __forceinline__ float dot3_rn(const float* r, float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fmul_rn(r[0], x), __fmul_rn(r[1], y)), __fmul_rn(r[2], z));
}

// The view-independent part of the specification: centroid and edges.
struct BinFace {
  float mx, my, mz;
  float e1x, e1y, e1z, e2x, e2y, e2z;
};
__device__ __forceinline__ BinFace bin_face(float3 a, float3 b, float3 c) {
  BinFace q;
  q.mx = __fdiv_rn(__fadd_rn(__fadd_rn(a.x, b.x), c.x), 3.0f);
  q.my = __fdiv_rn(__fadd_rn(__fadd_rn(a.y, b.y), c.y), 3.0f);
  q.mz = __fdiv_rn(__fadd_rn(__fadd_rn(a.z, b.z), c.z), 3.0f);
  q.e1x = __fsub_rn(b.x, a.x); q.e1y = __fsub_rn(b.y, a.y); q.e1z = __fsub_rn(b.z, a.z);
  q.e2x = __fsub_rn(c.x, a.x); q.e2y = __fsub_rn(c.y, a.y); q.e2z = __fsub_rn(c.z, a.z);
  return q;
}

// The per-view part, from bin_face's result (the same operations in the same
// order as if computed from the vertices here).
__device__ __forceinline__ BinResult bin_view(const BinFace& q, const ViewInfo& v, int tile, float inv_tile) {
  BinResult r;
  const float mx = q.mx, my = q.my, mz = q.mz;
  float tx = __fadd_rn(dot3_rn(v.R + 0, mx, my, mz), v.t[0]);
  float ty = __fadd_rn(dot3_rn(v.R + 3, mx, my, mz), v.t[1]);
  float tz = __fadd_rn(dot3_rn(v.R + 6, mx, my, mz), v.t[2]);
  r.depth = tz;
  float fxx = __fmul_rn(v.fx, tx);
  float fyy = __fmul_rn(v.fy, ty);
  float ux = __fadd_rn(__fdiv_rn(fxx, tz), v.cx);
  float uy = __fadd_rn(__fdiv_rn(fyy, tz), v.cy);
  float q1x = dot3_rn(v.R + 0, q.e1x, q.e1y, q.e1z), q1y = dot3_rn(v.R + 3, q.e1x, q.e1y, q.e1z),
        q1z = dot3_rn(v.R + 6, q.e1x, q.e1y, q.e1z);
  float q2x = dot3_rn(v.R + 0, q.e2x, q.e2y, q.e2z), q2y = dot3_rn(v.R + 3, q.e2x, q.e2y, q.e2z),
        q2z = dot3_rn(v.R + 6, q.e2x, q.e2y, q.e2z);
  float zz = __fmul_rn(tz, tz);
  float j00 = __fdiv_rn(v.fx, tz);
  float j11 = __fdiv_rn(v.fy, tz);
  float j02 = -__fdiv_rn(fxx, zz);
  float j12 = -__fdiv_rn(fyy, zz);
  float p1x = __fadd_rn(__fmul_rn(j00, q1x), __fmul_rn(j02, q1z));
  float p1y = __fadd_rn(__fmul_rn(j11, q1y), __fmul_rn(j12, q1z));
  float p2x = __fadd_rn(__fmul_rn(j00, q2x), __fmul_rn(j02, q2z));
  float p2y = __fadd_rn(__fmul_rn(j11, q2y), __fmul_rn(j12, q2z));
  float kxx = __fmul_rn(kKappaOver18, __fsub_rn(__fadd_rn(__fmul_rn(p1x, p1x), __fmul_rn(p2x, p2x)), __fmul_rn(p1x, p2x)));
  float kyy = __fmul_rn(kKappaOver18, __fsub_rn(__fadd_rn(__fmul_rn(p1y, p1y), __fmul_rn(p2y, p2y)), __fmul_rn(p1y, p2y)));
  float rx = __fadd_rn(__fsqrt_rn(__fmul_rn(kTwoLn255, __fadd_rn(kxx, 0.3f))), 0.25f);
  float ry = __fadd_rn(__fsqrt_rn(__fmul_rn(kTwoLn255, __fadd_rn(kyy, 0.3f))), 0.25f);
  r.visible = (tz > v.znear) && isfinite(ux) && isfinite(uy) && isfinite(rx) && isfinite(ry);
  r.x0 = 1; r.x1 = 0; r.y0 = 1; r.y1 = 0;
  if (!r.visible) return r;
  float bx0 = floorf(__fmul_rn(__fsub_rn(__fsub_rn(ux, rx), 0.5f), inv_tile));
  float bx1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(ux, rx), 0.5f), inv_tile));
  float by0 = floorf(__fmul_rn(__fsub_rn(__fsub_rn(uy, ry), 0.5f), inv_tile));
  float by1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(uy, ry), 0.5f), inv_tile));
  bx0 = fmaxf(bx0, 0.0f);
  by0 = fmaxf(by0, 0.0f);
  bx1 = fminf(bx1, (float)(v.tiles_x - 1));
  by1 = fminf(by1, (float)(v.tiles_y - 1));
  if (bx0 > bx1 || by0 > by1) return r;
  r.x0 = (int)bx0; r.x1 = (int)bx1; r.y0 = (int)by0; r.y1 = (int)by1;
  return r;
}

__device__ __forceinline__ BinResult bin_spec(float3 a, float3 b, float3 c, const ViewInfo& v, int tile,
                                              float inv_tile) {
  return bin_view(bin_face(a, b, c), v, tile, inv_tile);
}

// Exponent of one staged Gaussian at one pixel, in log2 units:
// p2 = a2 dx^2 + b2 dx dy + c2 dy^2 = -1/2 d^T Q d / ln 2, so that
// G = 2^p2. g = (ux, uy, a2, b2) with (ux, uy) the mean relative to the
// 32-pixel-aligned anchor of the pixel's block, (pcx, pcy) the pixel centre
// relative to the same anchor. A Gaussian is skipped at the pixel when
// p2 < t2 = log2(1 / (255 o)), i.e. when o G < 1/255; otherwise its weight is
// alpha = min(0.99, o 2^p2). Forward and backward use this same sequence of
// explicit single-precision operations, so they take identical decisions.
__device__ __forceinline__ float gauss_p2(float4 g, float c2, float pcx, float pcy, float& dx, float& dy) {
  dx = __fsub_rn(g.x, pcx);
  dy = __fsub_rn(g.y, pcy);
  float t = __fmaf_rn(g.z, dx, __fmul_rn(g.w, dy));
  return __fmaf_rn(t, dx, __fmul_rn(__fmul_rn(c2, dy), dy));
}

__device__ __forceinline__ float gauss_alpha(float p2, float o, float& graw) {
  graw = __fmul_rn(o, ex2_approx(p2));
  return fminf(graw, kAlphaMax);
}

// log2(255)
constexpr float kLog2_255 = 7.99435343685886f;

// ---------------------------------------------------------------- view-dependent colour
// Real spherical harmonics (no Condon-Shortley phase) of degree <= L at the
// unit vector (x, y, z), ordered (l, m) = (0, 0), (1, -1), (1, 0), (1, 1),
// (2, -2), ..., (3, 3), as polynomials in x, y, z; the FP32 constants are the
// normalisations written next to them. The colour of a facet seen along d is
// max(0, sum_k a_k Y_k(d) + 1/2) per channel (the 3DGS offset and clamp).
constexpr int kShMaxCoeffs = 16;
namespace sh {
constexpr float c0 = 0.282094791773878f;   // (1/2) sqrt(1/pi)
constexpr float c1 = 0.488602511902920f;   // sqrt(3/(4 pi))
constexpr float c2a = 1.092548430592079f;  // (1/2) sqrt(15/pi): xy, yz, xz
constexpr float c2b = 0.315391565252520f;  // (1/4) sqrt(5/pi): 3 z^2 - 1
constexpr float c2c = 0.546274215296040f;  // (1/4) sqrt(15/pi): x^2 - y^2
constexpr float c3a = 0.590043589926644f;  // (1/4) sqrt(35/(2 pi)): y (3x^2 - y^2), x (x^2 - 3y^2)
constexpr float c3b = 2.890611442640554f;  // (1/2) sqrt(105/pi): xyz
constexpr float c3c = 0.457045799464466f;  // (1/4) sqrt(21/(2 pi)): y (5z^2 - 1), x (5z^2 - 1)
constexpr float c3d = 0.373176332590115f;  // (1/4) sqrt(7/pi): z (5z^2 - 3)
constexpr float c3e = 1.445305721320277f;  // (1/4) sqrt(105/pi): z (x^2 - y^2)
}  // namespace sh

template <int L>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
  Y[0] = sh::c0;
  if (L < 1) return;
  Y[1] = sh::c1 * y;
  Y[2] = sh::c1 * z;
  Y[3] = sh::c1 * x;
  if (L < 2) return;
  Y[4] = sh::c2a * x * y;
  Y[5] = sh::c2a * y * z;
  Y[6] = sh::c2b * (3.0f * z * z - 1.0f);
  Y[7] = sh::c2a * x * z;
  Y[8] = sh::c2c * (x * x - y * y);
  if (L < 3) return;
  Y[9] = sh::c3a * y * (3.0f * x * x - y * y);
  Y[10] = sh::c3b * x * y * z;
  Y[11] = sh::c3c * y * (5.0f * z * z - 1.0f);
  Y[12] = sh::c3d * z * (5.0f * z * z - 3.0f);
  Y[13] = sh::c3c * x * (5.0f * z * z - 1.0f);
  Y[14] = sh::c3e * z * (x * x - y * y);
  Y[15] = sh::c3a * x * (x * x - 3.0f * y * y);
}

// sum_k s_k grad Y_k at (x, y, z): the gradient of the polynomials above
// (off the sphere as written; callers project onto the tangent plane).
template <int L>
__device__ __forceinline__ float3 sh_grad_dot(float x, float y, float z, const float* s) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (L >= 1) {
    gy += sh::c1 * s[1];
    gz += sh::c1 * s[2];
    gx += sh::c1 * s[3];
  }
  if (L >= 2) {
    gx += sh::c2a * (y * s[4] + z * s[7]) + 2.0f * sh::c2c * x * s[8];
    gy += sh::c2a * (x * s[4] + z * s[5]) - 2.0f * sh::c2c * y * s[8];
    gz += sh::c2a * (y * s[5] + x * s[7]) + 6.0f * sh::c2b * z * s[6];
  }
  if (L >= 3) {
    gx += sh::c3a * (6.0f * x * y * s[9] + (3.0f * x * x - 3.0f * y * y) * s[15]) + sh::c3b * y * z * s[10] +
          sh::c3c * (5.0f * z * z - 1.0f) * s[13] + 2.0f * sh::c3e * x * z * s[14];
    gy += sh::c3a * ((3.0f * x * x - 3.0f * y * y) * s[9] - 6.0f * x * y * s[15]) + sh::c3b * x * z * s[10] +
          sh::c3c * (5.0f * z * z - 1.0f) * s[11] - 2.0f * sh::c3e * y * z * s[14];
    gz += sh::c3b * x * y * s[10] + 10.0f * sh::c3c * z * (y * s[11] + x * s[13]) +
          sh::c3d * (15.0f * z * z - 3.0f) * s[12] + sh::c3e * (x * x - y * y) * s[14];
  }
  return make_float3(gx, gy, gz);
}

// ---------------------------------------------------------------- workspace
struct Workspace {
  // the vertices padded to 16 bytes (x, y, z, 0), written at the start of
  // every forward: the projection and its backward gather one vector per
  // vertex
  int64_t cap_verts4 = 0;
  float4* verts4 = nullptr;
  // records: one per (view, face)
  int64_t cap_records = 0;
  // one 32-byte record per (view, face), so that a gather touches one DRAM
  // sector: [2 r] = (ux_hi, uy_hi, ux_lo, uy_lo) the image mean,
  // [2 r + 1] = (a2, b2, c2, t2) the pre-scaled conic and skip threshold
  float4* rec_uq = nullptr;
  uint2* rec_rect = nullptr;     // packed (x0 | x1 << 16, y0 | y1 << 16)
  uint32_t* rec_ntiles = nullptr;
  uint32_t* rec_key = nullptr;   // FP32 depth bits (0xffffffff when culled)
  // 2 float4 per record: (sum q dx, sum q dy, sum q dx^2, sum q dx dy),
  // (sum q dy^2, 0, 0, 0) with q = alpha dL/dalpha over the record's pixels
  float4* rec_grad = nullptr;
  // view-dependent colour (GMR_COLOR_SH), one per record: colour and
  // opacity (r, g, b, o), and its gradient sums (dr, dg, db, sum dq)
  int64_t cap_sh_records = 0;
  float4* rec_col = nullptr;
  float4* rec_cgrad = nullptr;
  // faces
  int64_t cap_faces = 0;
  float4* face_col = nullptr;    // (r, g, b, o)
  float4* face_grad = nullptr;   // (dr, dg, db, sum dq)
  // pixels
  int64_t cap_pixels = 0;
  float* pix_T = nullptr;
  uint32_t* pix_last = nullptr;
  uint32_t* pix_ncontrib = nullptr;  // 2 x cap_pixels: counts, then order hashes (GMR_FLAG_DEBUG_COUNTS)
  // tiles
  int64_t cap_tiles = 0;
  uint32_t* tile_count = nullptr;  // pairs per tile (zero between forwards)
  uint32_t* tile_start = nullptr;  // exclusive scan of tile_count
  uint2* tile_range = nullptr;     // [start, end) per tile, (0, 0) when empty
  uint32_t* long_tiles = nullptr;  // tiles of more than 512 pairs (sorted by one CTA each)
  uint32_t* tile_order = nullptr;  // kTileClasses regions of cap_tiles: compositing order
  uint4* tile_desc = nullptr;      // per compositing position: (tile, view, range start, range end)
  // pairs
  int64_t cap_pairs = 0;
  // pair_key[0]: (depth bits << 32 | face) per pair in tile segments;
  // pair_key[1]: scratch of the long-segment sort, and before that, per pair
  // slot of the projection, (tile << 32 | rank of the pair in its tile)
  unsigned long long* pair_key[2] = {nullptr, nullptr};
  // face ids in (tile, depth, face) order; before the sort, per pair slot of
  // the projection, the pair's record id
  uint32_t* pair_face = nullptr;
  // split binning: per pair slot of the projection, the quadrants of its
  // 16x16 binning tile that the record's 8x8 rectangle holds (bit 2 qy + qx);
  // the keys then carry them below the face id (face << 4 | quadrants)
  uint8_t* pair_quad = nullptr;
  // scratch for scans
  int64_t cap_scan = 0;
  uint32_t* scan_tmp = nullptr;     // block sums
  // loss partial sums
  int64_t cap_loss = 0;
  double* loss_part = nullptr;
  float* reg_scratch = nullptr;  // mesh regularisers (edge lengths, neighbour sums), 1 double of mean first
  int64_t cap_reg = 0;
  // views
  int32_t cap_views = 0;
  ViewInfo* views = nullptr;
  Counters* counters = nullptr;
  // split binning (8x8 compositing tiles binned as 16x16): per binning
  // tile of n sorted pairs from `start`, its quadrants' lists at 4 start +
  // q n (4 x cap_pairs face ids), the compositing positions' descriptors
  // (4 per binning tile) and the 8x8 tiles' ranges (debug)
  int64_t cap_split_pairs = 0;
  uint32_t* pair_face_c = nullptr;
  int64_t cap_split_tiles = 0;
  uint4* tile_desc_c = nullptr;
  uint2* tile_range_c = nullptr;
  // GMR_FLAG_DETERMINISTIC: per record, the first of its pair slots (the
  // projection deals a record's pairs to consecutive slots, in the order of
  // its tiles in its rectangle, row by row); per pair slot, the compositing
  // backward's sums (3 float4: (sum q dx, sum q dy, sum q dx^2,
  // sum q dx dy), (sum q dy^2, sum dq, dr, dg), (db, 0, 0, 0))
  int64_t cap_det_records = 0;
  uint32_t* rec_slot = nullptr;
  int64_t cap_det_pairs = 0;
  float4* pair_grad = nullptr;
  // the vertex-to-face incidence list: per vertex its count, then (after the
  // scan) its first entry (cap_det_verts + 1), a fill cursor per vertex, the
  // entries 3 f + corner (3 per face), and per face the three corners'
  // vertex gradients and its colour gradient share (4 float4)
  int64_t cap_det_verts = 0;
  uint32_t* v_off = nullptr;
  uint32_t* v_cur = nullptr;
  int64_t cap_det_faces = 0;
  uint32_t* v_inc = nullptr;
  float4* corner_grad = nullptr;
};

// ---------------------------------------------------------------- launchers
// Every launcher returns cudaGetLastError() after enqueueing on stream s and
// increments *launches by the number of kernels it launched.

// gmr_sort.cu: exclusive scan of n u32 values into out, their sum into
// *total; src is set to zero
cudaError_t scan_exclusive(uint32_t* src, int64_t n, uint32_t* out, uint32_t* total, uint32_t* block_sums,
                           uint32_t* tile_order, uint32_t* n_class, cudaStream_t s, int64_t* launches);
int64_t scan_block_sums_needed(int64_t n);
// project.cu
// Conversion + projection of every (view, face) record; also writes the
// per-face colour/opacity and counts the pairs of every tile.
// Projection (S1-S2); it also zeroes the record and face gradient sums
// (ws.rec_grad for all C x F records, ws.face_grad for all F faces).
// With color_mode GMR_COLOR_SH (degree sh_degree) it writes ws.rec_col and
// zeroes ws.rec_cgrad for every record instead of ws.face_col / face_grad.
// det (GMR_FLAG_DETERMINISTIC): it also writes ws.rec_slot. It first pads
// the vertices into ws.verts4 (cap_verts4 >= V), which the projection
// backward reads too.
// tile: the compositing tile (the records' rectangles are in its units);
// bshift: log2 of binning tile / compositing tile (1 with split binning),
// the pairs are counted and emitted per binning tile.
cudaError_t launch_project(const float* verts, int32_t V, const int32_t* faces, int32_t F, const float* rgb,
                           const float* opacity, int color_mode, int sh_degree, const ViewInfo* views, int32_t C,
                           int tile, int bshift, int cov_mode, bool det, Workspace& ws, cudaStream_t s,
                           int64_t* launches);
// det: the record sums come from the pair slots (ws.pair_grad, ws.rec_slot,
// ws.rec_ntiles) instead of ws.rec_grad / face_grad / rec_cgrad, and the
// vertex (and per-vertex colour) gradients are gathered over the
// vertex-to-face incidence list (built here, in ws.v_off / v_cur / v_inc)
// from ws.corner_grad instead of added by atomics.
cudaError_t launch_project_bwd(const float* verts, int32_t V, const int32_t* faces, int32_t F,
                               const ViewInfo* views, int32_t C, int cov_mode, int color_mode, int sh_degree,
                               const float* rgb, const float* opacity, bool det, const Workspace& ws, float* dverts,
                               float* drgb, float* dop, int accumulate, cudaStream_t s, int64_t* launches);
// gmr_det.cu: dverts (V x 3) and dcol (V x 3, per-vertex colours; either
// may be null) from ws.corner_grad, each vertex's incident faces' shares
// added in (face, corner) order over the incidence list built here
// (ws.v_off, v_cur, v_inc: cap_det_verts >= V, cap_det_faces >= F);
// accumulate: add to the outputs instead of writing them.
cudaError_t launch_vertex_gather(const int32_t* faces, int32_t F, int32_t V, const Workspace& ws, float* dverts,
                                 float* dcol, int accumulate, cudaStream_t s, int64_t* launches);
cudaError_t launch_convert(const float* verts, int32_t V, const int32_t* faces, int32_t F, const float* rgb,
                           const float* opacity, int cov_mode, int color_mode, float* means, float* cov,
                           float* face_rgb, float* face_o, Counters* counters, cudaStream_t s, int64_t* launches);

// raster.cu
// bin.cu: scatter keys into tile segments, sort each segment, write ranges.
// split: the keys carry the pairs' quadrants (ws.pair_quad) below the face.
cudaError_t launch_bin_pairs(const Workspace& ws, int64_t n_rec, int32_t F, const ViewInfo* views, int32_t C,
                             int64_t n_tiles, bool split, cudaStream_t s, int64_t* launches);
cudaError_t launch_expand_tiles(const uint2* ranges, int64_t n_tiles, uint32_t* tile_ids, cudaStream_t s,
                                int64_t* launches);
// Split binning: the sorted list of every 16x16 binning tile (ws.tile_desc,
// n_btiles positions; entries face << 4 | quadrants) into the lists of its
// four 8x8 quadrants (the order kept) in ws.pair_face_c, with the
// compositing descriptors ws.tile_desc_c (position 4 w + q; kNoTile beyond
// the image) and the 8x8 ranges ws.tile_range_c.
cudaError_t launch_split_quads(const Workspace& ws, const ViewInfo* views, int64_t n_btiles, cudaStream_t s,
                               int64_t* launches);
// Debug copies of the forward's per-record data: tile rectangle and the
// unscaled conic.
cudaError_t launch_debug_records(const Workspace& ws, int64_t n_rec, int32_t* rects, float* conic, cudaStream_t s,
                                 int64_t* launches);
// Optional squared-error loss fused into the forward's epilogue (target ==
// nullptr: none): grad = 2 (image - target), *loss = sum (image - target)^2;
// part holds one FP32 partial sum per warp (n_tiles * threads / 32 floats),
// added up by a one-block kernel after the compositing.
struct FwdLoss {
  const float* target = nullptr;
  float* grad = nullptr;
  float* part = nullptr;
  double* loss = nullptr;
};
// persistent: a grid of resident CTAs taking compositing positions from a
// cursor (Counters::raster_next_fwd / _bwd, zero at launch) instead of one
// CTA per tile.
// Both compositing kernels read the colour of a record from ws.rec_col when
// col_by_record (GMR_COLOR_SH), else from ws.face_col by face; the backward
// adds colour gradients to ws.rec_cgrad or ws.face_grad likewise.
// layout: 0 staging by the CTA (full warps), 1 the half-warp layout (16x16
// tiles, 128 or 256 threads), 2 staging by each warp; 1 and 2 not with
// persistent.
// n_pos compositing positions (descriptors tile_desc, lists in pair_face:
// ws.tile_desc / ws.pair_face, or the split binning's); n_tiles compositing
// tiles (the loss partials are per tile).
cudaError_t launch_raster_fwd(int tile, int threads, int batch, bool persistent, int layout, bool col_by_record,
                              const Workspace& ws, const uint4* tile_desc, int64_t n_pos,
                              const uint32_t* pair_face, const ViewInfo* views, int32_t C, int32_t F,
                              int64_t n_tiles, const float* bg, float* images, float* t_final_out,
                              uint32_t* ncontrib_out, const FwdLoss& fl, cudaStream_t s, int64_t* launches);
// Optional squared-error loss fused into the backward's prologue (img ==
// nullptr: none): dL/dimg = 2 (img - target) is formed per pixel instead of
// being read, and the loss sum goes to one FP32 partial per CTA (part,
// n_tiles floats), added up by a one-block kernel (launch_sum_floats) after
// the compositing backward.
struct BwdLoss {
  const float* img = nullptr;
  const float* target = nullptr;
  float* part = nullptr;
};
// Up to two caller buffers (n floats each) that the projection backward
// accumulates into: the compositing backward's CTAs zero them (it runs
// before that kernel), which saves their memsets between the two
// compositing kernels.
struct BwdZero {
  float* p[2] = {nullptr, nullptr};
  int64_t n[2] = {0, 0};
};
// det (GMR_FLAG_DETERMINISTIC, layout 0 only; batch capped at 128): every
// pair's sums go to its slot in ws.pair_grad (zeros for the pairs behind the
// tile's last contributor) instead of atomics into rec_grad / face_grad /
// rec_cgrad.
cudaError_t launch_raster_bwd(int tile, int threads, int batch, bool persistent, int layout, bool col_by_record,
                              bool det, const Workspace& ws, const uint4* tile_desc, int64_t n_pos,
                              const uint32_t* pair_face, const ViewInfo* views, int32_t C, int32_t F,
                              int64_t n_tiles, const float* bg, const float* dL_dimages, const float* dL_dT,
                              const BwdLoss& bl, const BwdZero& bz, cudaStream_t s, int64_t* launches);
// The L2 loss kernel: a one-wave grid of at most kL2LossMaxBlocks blocks
// striding over chunks of kL2LossBlockElems floats.
constexpr int kL2LossBlockElems = 256 * 16;
constexpr int kL2LossMaxBlocks = 148 * 4;
// Doubles of partial-sum scratch launch_l2_loss needs for n floats: the
// ticket counter plus one per block; never more than 1 + kL2LossMaxBlocks.
constexpr int64_t l2_loss_partials_needed(int64_t n) {
  return 1 + ((n + kL2LossBlockElems - 1) / kL2LossBlockElems < kL2LossMaxBlocks
                  ? (n + kL2LossBlockElems - 1) / kL2LossBlockElems
                  : kL2LossMaxBlocks);
}
// partials: l2_loss_partials_needed(n) doubles; partials[0] holds a ticket
// counter that must be zero before the first call (every call leaves it zero)
cudaError_t launch_l2_loss(const float* img, const float* target, int64_t n, float* grad, double* loss,
                           double* partials, int64_t n_partials, cudaStream_t s, int64_t* launches);
// weight x the silhouette binary cross-entropy of the mask 1 - T_final
// against a target mask (mean over n pixels), with dL/dT_final; partials as
// for the L2 loss
cudaError_t launch_silhouette_bce(const float* t_final, const float* mask, int64_t n, float weight, float* dL_dT,
                                  double* loss, double* partials, int64_t n_partials, cudaStream_t s,
                                  int64_t* launches);
int64_t bce_partials_needed(int64_t n);
// *out = scale * sum of n floats (one CTA, fixed order, double-float sums)
cudaError_t launch_sum_floats(const float* x, int64_t n, double scale, double* out, cudaStream_t s,
                              int64_t* launches);
// gmr_optim.cu
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int group, float lr, float b1,
                        float b2, float eps, int step, cudaStream_t s, int64_t* launches);
// edge-length and Laplacian regularisers: losses[0..1] (unweighted), vertex
// gradients (weighted) added to dverts (may be null); scratch holds
// regularizer_scratch_floats(V, F) floats, mean_slot one double
int64_t regularizer_scratch_floats(int32_t V, int32_t F);
cudaError_t launch_regularizers(const float* verts, int32_t V, const int32_t* faces, int32_t F, float w_edge,
                                float w_lap, float* dverts, double* losses, float* scratch, double* mean_slot,
                                cudaStream_t s, int64_t* launches);
// out[0] = mean_a min_b |a - b|^2, out[1] = mean_b min_a |b - a|^2; scratch: na + nb floats
cudaError_t launch_chamfer(const float* a, int64_t na, const float* b, int64_t nb, float* scratch, double* out,
                           cudaStream_t s, int64_t* launches);

template <typename K>
inline int resident_grid(K kern, int threads, size_t smem = 0) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  const auto key = std::make_pair(reinterpret_cast<const void*>(kern), dev);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 148;
  }
  const int n = std::max(1, per_sm) * std::max(1, sms);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = n;
  return n;
}


}  // namespace gmr
