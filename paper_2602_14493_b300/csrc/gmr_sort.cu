// Device-wide exclusive scan of u32 values. Turns the per-tile pair counts
// into the tile segments of the binning and gives the total pair count; the
// counts are consumed (set back to zero, ready for the next forward).
// Up to kSingleMax values: one CTA walks the array in chunks of 8192 with a
// running carry (one launch); beyond, reduce-then-scan over many CTAs (three
// launches, no block waits on another).
//
// The same pass files every tile under its work class (tile_class of its
// pair count) in the compositing order (tile_of_block): each CTA counts its
// chunk's tiles per class in shared memory (warp-aggregated) and writes them
// into its run of each class's region, the runs in chunk order (so tiles of
// one view stay together within a class): the single CTA takes its runs
// chunk by chunk, the multi-CTA scan from per-block class counts scanned in
// block order.

#include "gmr_internal.cuh"

namespace gmr {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048


__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total (all threads see it).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* smem_warp, uint32_t* total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = warp_incl_scan(v, lane);
  if (lane == 31) smem_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? smem_warp[lane] : 0u;
    uint32_t wi = warp_incl_scan(w, lane);
    if (lane < nw) smem_warp[lane] = wi - w;
    if (lane == nw - 1) smem_warp[32] = wi;
  }
  __syncthreads();
  uint32_t r = incl - v + smem_warp[warp];
  *total = smem_warp[32];
  __syncthreads();
  return r;
}

// Counts the tiles i0 + k (k < NI, i0 + k < n) of the calling thread, with
// pair counts v[k], in the CTA's per-class counters s_hist (warp-aggregated
// shared-memory atomics) and returns each tile's class and rank within the
// CTA's tiles of that class.
template <int NI>
__device__ __forceinline__ void count_classes(const uint32_t (&v)[NI], int64_t i0, int64_t n, uint32_t (&rank)[NI],
                                              int (&cls)[NI], uint32_t* s_hist) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < NI; ++k) {
    const bool ok = i0 + k < n;
    cls[k] = tile_class(v[k]);
    const uint32_t key = ok ? (uint32_t)cls[k] : 0xffffffffu;  // idle lanes in a group of their own
    const uint32_t peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (ok && lane == leader) base = atomicAdd(&s_hist[cls[k]], (uint32_t)__popc(peers));
    rank[k] = __shfl_sync(0xffffffffu, base, leader) + __popc(peers & lt);
  }
}

// Files the tiles i0 + k (k < NI, i0 + k < n) of every thread of the CTA
// under their classes: tile_order[c * n + slot], slot = the CTA's run of
// class c + the tile's rank. The runs come from block_base (kTileClasses
// offsets, when given) or are reserved from n_class by one global atomic per
// class. Every thread of the CTA calls it (it holds barriers); s_hist and
// s_base are kTileClasses words of shared memory each.
template <int NI>
__device__ __forceinline__ void file_tiles(const uint32_t (&v)[NI], int64_t i0, int64_t n,
                                           uint32_t* __restrict__ tile_order, uint32_t* __restrict__ n_class,
                                           const uint32_t* __restrict__ block_base, uint32_t* s_hist,
                                           uint32_t* s_base) {
  if (threadIdx.x < kTileClasses) s_hist[threadIdx.x] = 0u;
  __syncthreads();
  uint32_t rank[NI];
  int cls[NI];
  count_classes<NI>(v, i0, n, rank, cls, s_hist);
  __syncthreads();
  if (threadIdx.x < kTileClasses) {
    const uint32_t cnt = s_hist[threadIdx.x];
    s_base[threadIdx.x] = block_base ? block_base[threadIdx.x] : (cnt ? atomicAdd(&n_class[threadIdx.x], cnt) : 0u);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NI; ++k)
    if (i0 + k < n) tile_order[cls[k] * n + s_base[cls[k]] + rank[k]] = (uint32_t)(i0 + k);
  __syncthreads();
}

// Per block of kScanTile values: their sum, and (block_hist, kTileClasses
// words per block) how many of them fall in each work class.
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ src, int64_t n,
                                                              uint32_t* __restrict__ block_sums,
                                                              uint32_t* __restrict__ block_hist) {
  pdl_enter();
  __shared__ uint32_t sw[33];
  __shared__ uint32_t s_hist[kTileClasses];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (threadIdx.x < kTileClasses) s_hist[threadIdx.x] = 0u;
  __syncthreads();
  uint32_t acc = 0;
  uint32_t v[kScanItems];
  const int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = i0 + k < n ? src[i0 + k] : 0u;
    acc += v[k];
  }
  uint32_t rank[kScanItems];
  int cls[kScanItems];
  count_classes<kScanItems>(v, i0, n, rank, cls, s_hist);
  uint32_t tot;
  block_excl_scan(acc, sw, &tot);  // (barriers inside)
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
  if (threadIdx.x < kTileClasses) block_hist[(int64_t)blockIdx.x * kTileClasses + threadIdx.x] = s_hist[threadIdx.x];
}

// Single block: exclusive scan of the block sums in place, total to *total;
// per class, the blocks' counts turned into their offsets in block order
// (so each class keeps the tiles' order across blocks) and the class
// totals written to n_class.
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* __restrict__ sums, int64_t nb,
                                                   uint32_t* __restrict__ total, uint32_t* __restrict__ block_hist,
                                                   uint32_t* __restrict__ n_class) {
  pdl_enter();
  __shared__ uint32_t sw[33];
  if (threadIdx.x < kTileClasses) {
    uint32_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const uint32_t c = block_hist[b * kTileClasses + threadIdx.x];
      block_hist[b * kTileClasses + threadIdx.x] = run;
      run += c;
    }
    n_class[threadIdx.x] = run;
  }
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < nb ? sums[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_excl_scan(v, sw, &tot);
    if (i < nb) sums[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t* __restrict__ src, int64_t n,
                                                            const uint32_t* __restrict__ block_sums,
                                                            uint32_t* __restrict__ out, uint32_t* __restrict__ tile_order,
                                                            const uint32_t* __restrict__ block_hist) {
  pdl_enter();
  __shared__ uint32_t sw[33];
  __shared__ uint32_t tile[kScanTile];
  __shared__ uint32_t s_hist[kTileClasses], s_base[kTileClasses];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  // coalesced load into shared memory, then each thread scans 8 consecutive
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int j = k * kScanThreads + threadIdx.x;
    int64_t i = base + j;
    tile[j] = i < n ? src[i] : 0u;
    if (i < n) src[i] = 0u;
  }
  __syncthreads();
  uint32_t v[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = tile[threadIdx.x * kScanItems + k];
    acc += v[k];
  }
  file_tiles<kScanItems>(v, base + (int64_t)threadIdx.x * kScanItems, n, tile_order, nullptr,
                         block_hist + (int64_t)blockIdx.x * kTileClasses, s_hist, s_base);
  uint32_t tot;
  uint32_t pre = block_excl_scan(acc, sw, &tot) + block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile[threadIdx.x * kScanItems + k] = pre;
    pre += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int j = k * kScanThreads + threadIdx.x;
    int64_t i = base + j;
    if (i < n) out[i] = tile[j];
  }
}

constexpr int kSingleThreads = 1024;
constexpr int kSingleChunk = kSingleThreads * kScanItems;  // 8192
constexpr int64_t kSingleMax = 4 * kSingleChunk;

// One CTA; each thread owns 8 consecutive values of a chunk, loaded and
// stored as two 16-byte vectors (no shared-memory transpose), with a scalar
// path for the ragged last chunk.
__global__ void __launch_bounds__(kSingleThreads) k_scan_single(uint32_t* __restrict__ src, int64_t n,
                                                                uint32_t* __restrict__ out,
                                                                uint32_t* __restrict__ total,
                                                                uint32_t* __restrict__ tile_order,
                                                                uint32_t* __restrict__ n_class) {
  pdl_enter();
  __shared__ uint32_t sw[33];
  __shared__ uint32_t s_hist[kTileClasses], s_base[kTileClasses];
  uint32_t carry = 0;
  for (int64_t base = 0; base < n; base += kSingleChunk) {
    const int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    const bool full = i0 + kScanItems <= n;
    if (full) {
      const uint4 a = *reinterpret_cast<const uint4*>(src + i0);
      const uint4 b = *reinterpret_cast<const uint4*>(src + i0 + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(src + i0) = z;
      *reinterpret_cast<uint4*>(src + i0 + 4) = z;
    } else {
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) {
        v[k] = i0 + k < n ? src[i0 + k] : 0u;
        if (i0 + k < n) src[i0 + k] = 0u;
      }
    }
    file_tiles<kScanItems>(v, i0, n, tile_order, n_class, nullptr, s_hist, s_base);
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) acc += v[k];
    uint32_t tot;
    uint32_t pre = block_excl_scan(acc, sw, &tot) + carry;
    uint32_t o[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      o[k] = pre;
      pre += v[k];
    }
    if (full) {
      *reinterpret_cast<uint4*>(out + i0) = make_uint4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<uint4*>(out + i0 + 4) = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
      for (int k = 0; k < kScanItems; ++k)
        if (i0 + k < n) out[i0 + k] = o[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

}  // namespace

// block sums, then kTileClasses class counts per block
int64_t scan_block_sums_needed(int64_t n) { return ((n + kScanTile - 1) / kScanTile + 1) * (1 + kTileClasses); }

cudaError_t scan_exclusive(uint32_t* src, int64_t n, uint32_t* out, uint32_t* total, uint32_t* block_sums,
                           uint32_t* tile_order, uint32_t* n_class, cudaStream_t s, int64_t* launches) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
    return cudaGetLastError();
  }
  // the vector path needs 16-byte aligned arrays (workspace allocations are)
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
  if (n <= kSingleMax && aligned) {
    cudaError_t e = launch_chained(k_scan_single, true, dim3(1), dim3(kSingleThreads), 0, s, src, n, out, total,
                                   tile_order, n_class);
    *launches += 1;
    return e;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  uint32_t* block_hist = block_sums + nb + 1;
  cudaError_t e = launch_chained(k_scan_reduce, true, dim3((unsigned)nb), dim3(kScanThreads), 0, s, (const uint32_t*)src,
                                 n, block_sums, block_hist);
  if (e == cudaSuccess)
    e = launch_chained(k_scan_top, true, dim3(1), dim3(1024), 0, s, block_sums, nb, total, block_hist, n_class);
  if (e == cudaSuccess)
    e = launch_chained(k_scan_down, true, dim3((unsigned)nb), dim3(kScanThreads), 0, s, src, n,
                       (const uint32_t*)block_sums, out, tile_order, (const uint32_t*)block_hist);
  *launches += 3;
  return e;
}

}  // namespace gmr
