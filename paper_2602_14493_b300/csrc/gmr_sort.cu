// Device-wide exclusive scan and stable LSD radix sort of (u32 key, u32
// value) pairs. Used to order the per-(view, face) Gaussians by depth key and
// then the (tile, Gaussian) pairs by tile id; stability of both passes gives
// the (tile, depth, face index) order of the 3DGS binning (Sec. 2.1).
//
// Both are reduce-then-scan designs: no block ever waits on another block,
// so nothing can spin. The element count may live in device memory (the
// pair count is produced on the device); grids are sized for the capacity and
// blocks past the count do nothing.

#include "gmr_internal.cuh"

namespace gmr {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                         // per thread
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 per block
constexpr int kRadix = 256;

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

__device__ __forceinline__ uint32_t load_item(const uint32_t* src, const uint32_t* idx, int64_t i) {
  return idx ? src[idx[i]] : src[i];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ src,
                                                              const uint32_t* __restrict__ idx, int64_t n,
                                                              uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t sw[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) acc += load_item(src, idx, i);
  }
  uint32_t tot;
  block_excl_scan(acc, sw, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place, total to *total.
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* __restrict__ sums, int64_t nb,
                                                   uint32_t* __restrict__ total) {
  __shared__ uint32_t sw[33];
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

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ src,
                                                            const uint32_t* __restrict__ idx, int64_t n,
                                                            const uint32_t* __restrict__ block_sums,
                                                            uint32_t* __restrict__ out) {
  __shared__ uint32_t sw[33];
  __shared__ uint32_t tile[kScanTile];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  // coalesced load into shared memory, then each thread scans 8 consecutive
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int j = k * kScanThreads + threadIdx.x;
    int64_t i = base + j;
    tile[j] = i < n ? load_item(src, idx, i) : 0u;
  }
  __syncthreads();
  uint32_t v[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = tile[threadIdx.x * kScanItems + k];
    acc += v[k];
  }
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

// ---- radix sort

__device__ __forceinline__ uint32_t sort_count(const uint32_t* n_dev, int64_t n_cap) {
  if (!n_dev) return (uint32_t)n_cap;
  uint32_t n = *n_dev;
  return n > (uint64_t)n_cap ? (uint32_t)n_cap : n;
}

// Per-block digit histogram, stored digit-major: counts[d * nb + block].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ n_dev, int64_t n_cap,
                                                             int shift, uint32_t* __restrict__ counts) {
  __shared__ uint32_t hist[kRadix];
  hist[threadIdx.x] = 0;
  __syncthreads();
  uint32_t n = sort_count(n_dev, n_cap);
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base < n) {
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
      int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
      if (i < n) atomicAdd(&hist[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter. Warp w of a block owns items [base + w*512, base + w*512 +
// 512), taken 32 at a time in order; equal digits within a 32-item step are
// ranked by lane (match_any), earlier steps and warps come first, so the
// relative order of equal digits is kept.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ n_dev, int64_t n_cap, int shift,
    const uint32_t* __restrict__ offsets) {
  __shared__ uint32_t wcount[kSortWarps][kRadix];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < kRadix; d += 32) wcount[warp][d] = 0;
  __syncwarp();
  uint32_t n = sort_count(n_dev, n_cap);
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) return;  // uniform over the block
  int64_t wbase = base + (int64_t)warp * (32 * kSortItems);
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    int64_t i = wbase + k * 32 + lane;
    bool ok = i < n;
    key[k] = ok ? keys_in[i] : 0u;
    val[k] = ok ? vals_in[i] : 0u;
    uint32_t d = ok ? ((key[k] >> shift) & (kRadix - 1)) : (kRadix + lane);
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = wcount[warp][ok ? d : 0];
    __syncwarp();
    rank[k] = before + __popc(peers & lt_mask);
    if (ok && (peers & lt_mask) == 0) wcount[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, per digit
  {
    int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t c = wcount[w][d];
      wcount[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    int64_t i = wbase + k * 32 + lane;
    if (i < n) {
      uint32_t d = (key[k] >> shift) & (kRadix - 1);
      uint32_t pos = offsets[(int64_t)d * gridDim.x + blockIdx.x] + wcount[warp][d] + rank[k];
      keys_out[pos] = key[k];
      vals_out[pos] = val[k];
    }
  }
}

}  // namespace

int64_t scan_block_sums_needed(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t scan_exclusive(const uint32_t* src, const uint32_t* idx, int64_t n, uint32_t* out, uint32_t* total,
                           uint32_t* block_sums, cudaStream_t s, int64_t* launches) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
    return cudaGetLastError();
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(src, idx, n, block_sums);
  k_scan_top<<<1, 1024, 0, s>>>(block_sums, nb, total);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(src, idx, n, block_sums, out);
  *launches += 3;
  return cudaGetLastError();
}

int64_t radix_counts_needed(int64_t n_cap) { return ((n_cap + kSortTile - 1) / kSortTile) * kRadix; }

int radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], const uint32_t* n_dev, int64_t n_cap, int bits,
                     uint32_t* counts, uint32_t* scan_tmp, cudaStream_t s, int64_t* launches, cudaError_t* err) {
  *err = cudaSuccess;
  if (n_cap <= 0 || bits <= 0) return 0;
  int64_t nb = (n_cap + kSortTile - 1) / kSortTile;
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<(unsigned)nb, kSortThreads, 0, s>>>(keys[cur], n_dev, n_cap, shift, counts);
    *launches += 1;
    cudaError_t e = scan_exclusive(counts, nullptr, nb * kRadix, counts, nullptr, scan_tmp, s, launches);
    if (e != cudaSuccess) { *err = e; return cur; }
    k_radix_scatter<<<(unsigned)nb, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_dev,
                                                          n_cap, shift, counts);
    *launches += 1;
    cur ^= 1;
  }
  *err = cudaGetLastError();
  return cur;
}

}  // namespace gmr
