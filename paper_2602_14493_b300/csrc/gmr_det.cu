// Per-vertex gradient sums in a fixed order (GMR_FLAG_DETERMINISTIC): the
// chain rule of the conversion (Eq. 4-16) gives every face a share of the
// gradient of each of its three vertices (and, with per-vertex colours,
// Eq. 16, a third of its colour gradient); a vertex's gradient is the sum
// of its incident faces' shares. Instead of float atomics (whose order, and
// so whose rounding, varies from run to run) the shares are gathered per
// vertex over a vertex-to-face incidence list, in increasing (face, corner)
// order:
//
//  1. count the corners of every vertex (faces with an index outside [0, V)
//     are left out, as the projection leaves them out);
//  2. exclusive scan of the counts (one CTA, chunks of 8192 with a carry):
//     the first entry of every vertex, and a fill cursor;
//  3. each corner takes an entry from its vertex's cursor (in any order);
//  4. one thread per vertex sorts its entries (3 f + corner; unique keys, so
//     the sorted order is unique) and adds the shares in that order.

#include "gmr_internal.cuh"

namespace gmr {
namespace {

constexpr int kDetThreads = 256;
constexpr int kScanChunkThreads = 1024;
constexpr int kScanPerThread = 8;

__device__ __forceinline__ bool corner_vertex(const int32_t* __restrict__ faces, int64_t i, int32_t V, int& v) {
  const int64_t f = i / 3;
  const int i0 = __ldg(faces + 3 * f), i1 = __ldg(faces + 3 * f + 1), i2 = __ldg(faces + 3 * f + 2);
  if ((unsigned)i0 >= (unsigned)V || (unsigned)i1 >= (unsigned)V || (unsigned)i2 >= (unsigned)V) return false;
  const int k = (int)(i - 3 * f);
  v = k == 0 ? i0 : k == 1 ? i1 : i2;
  return true;
}

__global__ void __launch_bounds__(kDetThreads) k_vert_count(const int32_t* __restrict__ faces, int32_t F, int32_t V,
                                                            uint32_t* __restrict__ v_cnt) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * kDetThreads + threadIdx.x;
  int v;
  if (i < 3 * (int64_t)F && corner_vertex(faces, i, V, v)) atomicAdd(v_cnt + v, 1u);
}

// In place: v_off[0, V) counts -> first entries, v_off[V] = total; v_cur =
// first entries.
__global__ void __launch_bounds__(kScanChunkThreads) k_vert_scan(uint32_t* __restrict__ v_off, int32_t V,
                                                                 uint32_t* __restrict__ v_cur) {
  pdl_enter();
  __shared__ uint32_t s_warp[kScanChunkThreads / 32];
  __shared__ uint32_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  constexpr int64_t kChunk = (int64_t)kScanChunkThreads * kScanPerThread;
  for (int64_t base = 0; base < V; base += kChunk) {
    uint32_t x[kScanPerThread];
    uint32_t sum = 0;
#pragma unroll
    for (int r = 0; r < kScanPerThread; ++r) {
      const int64_t i = base + (int64_t)threadIdx.x * kScanPerThread + r;
      x[r] = i < V ? v_off[i] : 0u;
      sum += x[r];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = s_warp[lane];
      uint32_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      s_warp[lane] = ti - t;  // exclusive prefix of the warps' sums
    }
    __syncthreads();
    uint32_t pre = s_carry + s_warp[warp] + incl - sum;
#pragma unroll
    for (int r = 0; r < kScanPerThread; ++r) {
      const int64_t i = base + (int64_t)threadIdx.x * kScanPerThread + r;
      if (i < V) {
        v_off[i] = pre;
        v_cur[i] = pre;
      }
      pre += x[r];
    }
    __syncthreads();  // every thread has read s_carry and s_warp
    if (threadIdx.x == kScanChunkThreads - 1) s_carry = pre;
    __syncthreads();
  }
  if (threadIdx.x == 0) v_off[V] = s_carry;
}

__global__ void __launch_bounds__(kDetThreads) k_vert_fill(const int32_t* __restrict__ faces, int32_t F, int32_t V,
                                                           uint32_t* __restrict__ v_cur, uint32_t* __restrict__ v_inc) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * kDetThreads + threadIdx.x;
  int v;
  if (i < 3 * (int64_t)F && corner_vertex(faces, i, V, v)) v_inc[atomicAdd(v_cur + v, 1u)] = (uint32_t)i;
}

// Ascending sort of a[0, n) in place (a vertex's few entries): Shell's
// method with Ciura's gaps, extended by x2.25, for the rare long list.
__device__ void sort_entries(uint32_t* a, uint32_t n) {
  constexpr uint32_t kGaps[] = {1,     4,     10,    23,     57,     132,    301,     701,     1577,   3548,
                                7983,  17961, 40412, 90927,  204585, 460316, 1035711, 2330349, 5243285};
  constexpr int kNumGaps = (int)(sizeof(kGaps) / sizeof(kGaps[0]));
  int gi = 0;
  while (gi + 1 < kNumGaps && kGaps[gi + 1] < n) ++gi;
  for (; gi >= 0; --gi) {
    const uint32_t gap = kGaps[gi];
    for (uint32_t i = gap; i < n; ++i) {
      const uint32_t key = a[i];
      uint32_t j = i;
      while (j >= gap && a[j - gap] > key) {
        a[j] = a[j - gap];
        j -= gap;
      }
      a[j] = key;
    }
  }
}

__global__ void __launch_bounds__(kDetThreads) k_vert_gather(const uint32_t* __restrict__ v_off,
                                                             uint32_t* __restrict__ v_inc,
                                                             const float4* __restrict__ corner_grad, int32_t V,
                                                             float* __restrict__ dverts, float* __restrict__ dcol,
                                                             int accumulate) {
  pdl_enter();
  const int64_t v = (int64_t)blockIdx.x * kDetThreads + threadIdx.x;
  if (v >= V) return;
  const uint32_t b = v_off[v], e = v_off[v + 1];
  sort_entries(v_inc + b, e - b);
  float3 s = make_float3(0.f, 0.f, 0.f), sc = s;
  for (uint32_t k = b; k < e; ++k) {
    const uint32_t c = v_inc[k];
    const uint32_t f = c / 3;
    const float4 g = corner_grad[4 * (size_t)f + (c - 3 * f)];
    s.x += g.x;
    s.y += g.y;
    s.z += g.z;
    if (dcol) {
      const float4 h = corner_grad[4 * (size_t)f + 3];
      sc.x += h.x;
      sc.y += h.y;
      sc.z += h.z;
    }
  }
  if (dverts) {
    float* d = dverts + 3 * v;
    if (accumulate) {
      d[0] += s.x; d[1] += s.y; d[2] += s.z;
    } else {
      d[0] = s.x; d[1] = s.y; d[2] = s.z;
    }
  }
  if (dcol) {
    float* d = dcol + 3 * v;
    if (accumulate) {
      d[0] += sc.x; d[1] += sc.y; d[2] += sc.z;
    } else {
      d[0] = sc.x; d[1] = sc.y; d[2] = sc.z;
    }
  }
}

}  // namespace

cudaError_t launch_vertex_gather(const int32_t* faces, int32_t F, int32_t V, const Workspace& ws, float* dverts,
                                 float* dcol, int accumulate, cudaStream_t s, int64_t* launches) {
  if (V <= 0 || (!dverts && !dcol)) return cudaSuccess;
  if (ws.cap_det_verts < V || ws.cap_det_faces < F) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(ws.v_off, 0, sizeof(uint32_t) * ((size_t)V + 1), s);
  if (e != cudaSuccess) return e;
  const unsigned corner_blocks = (unsigned)((3 * (int64_t)F + kDetThreads - 1) / kDetThreads);
  if (F > 0) k_vert_count<<<corner_blocks, kDetThreads, 0, s>>>(faces, F, V, ws.v_off);
  k_vert_scan<<<1, kScanChunkThreads, 0, s>>>(ws.v_off, V, ws.v_cur);
  if (F > 0) k_vert_fill<<<corner_blocks, kDetThreads, 0, s>>>(faces, F, V, ws.v_cur, ws.v_inc);
  k_vert_gather<<<(unsigned)((V + kDetThreads - 1) / kDetThreads), kDetThreads, 0, s>>>(
      ws.v_off, ws.v_inc, ws.corner_grad, V, dverts, dcol, accumulate);
  *launches += F > 0 ? 4 : 2;
  return cudaGetLastError();
}

}  // namespace gmr
