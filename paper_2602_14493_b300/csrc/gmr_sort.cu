// Device-wide exclusive scan and stable LSD radix sort of (u32 key, u32
// value) pairs. Used to order the per-(view, face) Gaussians by depth key and
// then the (tile, Gaussian) pairs by tile id; stability of both passes gives
// the (tile, depth, face index) order of the 3DGS binning (Sec. 2.1).
//
// The scan is a reduce-then-scan design (no block waits on another). The
// sort uses one kernel per digit with a bounded look-back (below). The element
// count may live in device memory (the pair count is produced on the
// device); grids are sized for the capacity and blocks past the count do
// nothing.

#include <algorithm>

#include "gmr_internal.cuh"

namespace gmr {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
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

// ---- radix sort (one sweep per 8-bit digit)
//
// LSD radix sort in which each digit pass is a single kernel. Tiles of
// kTile items are claimed in order through an atomic ticket; every tile
// ranks its items by digit (stable, warp match_any), publishes its per-digit
// counts, and finds the number of items of each digit in all earlier tiles
// by looking back over the published counts (a predecessor publishes first
// its own count, then its inclusive prefix, flagged so that the look-back
// can stop at the first prefix). Items are then reordered in shared memory
// and written out in runs per digit. The global start of each digit comes
// from one histogram of all passes computed up front.
//
// The look-back waits only on tiles with an earlier ticket, which belong to
// blocks that are already running, so it always ends; it is nevertheless
// bounded, and on expiry the kernel sets GMR_DEV_SORT_TIMEOUT and continues.

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 4;
constexpr uint32_t kSpinLimit = 1u << 20;
constexpr int kLookback = 16;

// A status word carries its flag and its count together, so single-copy
// atomic relaxed accesses at GPU scope suffice (no other data is published
// through it); relaxed loads of a look-back window can be in flight together.
__device__ __forceinline__ void st_status(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_status(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t sort_count(const uint32_t* n_dev, int64_t n_cap) {
  if (!n_dev) return (uint32_t)n_cap;
  uint32_t n = *n_dev;
  return n > (uint64_t)n_cap ? (uint32_t)n_cap : n;
}

// Histogram of every digit pass (warp-aggregated shared-memory counts).
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ n_dev, int64_t n_cap,
                                                            int passes, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[kMaxPasses][kRadix];
  for (int p = 0; p < kMaxPasses; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  const uint32_t n = sort_count(n_dev, n_cap);
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t stride = (int64_t)gridDim.x * kSortThreads;
  const int64_t n_round = ((int64_t)n + 31) & ~(int64_t)31;
  for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n_round; i += stride) {
    const bool ok = i < n;
    const uint32_t k = ok ? keys[i] : 0u;
    for (int p = 0; p < passes; ++p) {
      uint32_t d = ok ? ((k >> (8 * p)) & (kRadix - 1)) : (kRadix + lane);
      uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (ok && (peers & lt) == 0) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    uint32_t v = h[p][threadIdx.x];
    if (v) atomicAdd(&ghist[p * kRadix + threadIdx.x], v);
  }
}

template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ n_dev, int64_t n_cap, int shift,
    const uint32_t* __restrict__ ghist, uint32_t* __restrict__ ticket, uint32_t* __restrict__ status,
    uint32_t* __restrict__ dev_status) {
  constexpr int kTile = kSortThreads * ITEMS;
  __shared__ uint32_t s_keys[kTile];
  __shared__ uint32_t s_vals[kTile];
  __shared__ uint32_t wcount[kSortWarps][kRadix];
  __shared__ uint32_t s_local[kRadix];   // block-local start of each digit
  __shared__ uint32_t s_global[kRadix];  // global start of each digit for this tile
  __shared__ uint32_t sw[33];
  __shared__ uint32_t s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  for (int d = lane; d < kRadix; d += 32) wcount[warp][d] = 0;
  __syncthreads();
  const uint32_t n = sort_count(n_dev, n_cap);
  const uint32_t t = s_tile;
  const uint32_t n_tiles = (n + kTile - 1) / kTile;
  if (t >= n_tiles) return;  // uniform over the block
  const int64_t base = (int64_t)t * kTile;
  const int64_t wbase = base + (int64_t)warp * (32 * ITEMS);
  uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = wbase + k * 32 + lane;
    bool ok = i < n;
    key[k] = ok ? keys_in[i] : 0u;
    val[k] = ok ? vals_in[i] : 0u;
    uint32_t d = ok ? ((key[k] >> shift) & (kRadix - 1)) : (kRadix + lane);
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = wcount[warp][ok ? d : 0];
    __syncwarp();
    rank[k] = before + __popc(peers & lt);
    if (ok && (peers & lt) == 0) wcount[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: warp offsets inside the tile, tile count
  const int d = threadIdx.x;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    uint32_t c = wcount[w][d];
    wcount[w][d] = cnt;
    cnt += c;
  }
  uint32_t tot;
  s_local[d] = block_excl_scan(cnt, sw, &tot);
  // look back over earlier tiles for the count of digit d before this tile
  uint32_t* my = status + (size_t)t * kRadix + d;
  uint32_t excl = 0;
  if (t == 0) {
    st_status(my, kFlagPrefix | cnt);
  } else {
    st_status(my, kFlagAgg | cnt);
    // look back kLookback predecessors per round trip: the loads are
    // independent, so a round costs one memory latency instead of kLookback
    int64_t pred = (int64_t)t - 1;
    uint32_t spins = 0;
    while (true) {
      uint32_t v[kLookback];
#pragma unroll
      for (int i = 0; i < kLookback; ++i)
        v[i] = (pred - i >= 0) ? ld_status(status + (size_t)(pred - i) * kRadix + d) : kFlagPrefix;
      int i = 0;
      bool found = false;
#pragma unroll
      for (int q = 0; q < kLookback; ++q) {
        if (found || i != q) continue;  // stop at the first prefix or unpublished entry
        uint32_t f = v[q] & ~kCountMask;
        if (f == 0u) continue;
        excl += v[q] & kCountMask;
        if (f == kFlagPrefix) found = true;
        else i = q + 1;
      }
      if (found) break;
      pred -= i;
      if (i == 0) {  // predecessor `pred` has not published yet
        if (++spins > kSpinLimit) {
          atomicOr(dev_status, GMR_DEV_SORT_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    st_status(my, kFlagPrefix | (excl + cnt));
  }
  uint32_t gtot;
  const uint32_t gstart = block_excl_scan(ghist[d], sw, &gtot);
  s_global[d] = gstart + excl;
  __syncthreads();
  // reorder inside the tile by digit (stable), then write runs per digit
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = wbase + k * 32 + lane;
    if (i < n) {
      uint32_t dd = (key[k] >> shift) & (kRadix - 1);
      uint32_t lp = s_local[dd] + wcount[warp][dd] + rank[k];
      s_keys[lp] = key[k];
      s_vals[lp] = val[k];
    }
  }
  __syncthreads();
  const int m = (int)min((int64_t)kTile, (int64_t)n - base);
  for (int i = threadIdx.x; i < m; i += kSortThreads) {
    uint32_t k2 = s_keys[i];
    uint32_t dd = (k2 >> shift) & (kRadix - 1);
    uint32_t gpos = s_global[dd] + ((uint32_t)i - s_local[dd]);
    keys_out[gpos] = k2;
    vals_out[gpos] = s_vals[i];
  }
}

constexpr int kPassItems = 8;
constexpr int kPassTile = kSortThreads * kPassItems;  // 2048

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

// Scratch layout (u32): ghist[kMaxPasses][256], tickets[kMaxPasses],
// status[kMaxPasses][tiles][256].
int64_t radix_counts_needed(int64_t n_cap) {
  int64_t tiles = (n_cap + kPassTile - 1) / kPassTile;
  return (int64_t)kMaxPasses * kRadix + kMaxPasses + (int64_t)kMaxPasses * tiles * kRadix + 64;
}

int radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], const uint32_t* n_dev, int64_t n_cap, int bits,
                     uint32_t* scratch, uint32_t* dev_status, cudaStream_t s, int64_t* launches, cudaError_t* err) {
  *err = cudaSuccess;
  if (n_cap <= 0 || bits <= 0) return 0;
  const int passes = (bits + 7) / 8;
  if (passes > kMaxPasses || n_cap >= (int64_t)kCountMask) {
    *err = cudaErrorInvalidValue;
    return 0;
  }
  const int64_t tiles = (n_cap + kPassTile - 1) / kPassTile;
  uint32_t* ghist = scratch;
  uint32_t* tickets = scratch + kMaxPasses * kRadix;
  uint32_t* status = tickets + kMaxPasses;
  const size_t bytes = sizeof(uint32_t) * ((size_t)kMaxPasses * kRadix + kMaxPasses + (size_t)passes * tiles * kRadix);
  cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, s);
  if (e != cudaSuccess) { *err = e; return 0; }
  const int hist_blocks = (int)std::min<int64_t>((n_cap + kSortThreads - 1) / kSortThreads, 4 * 148);
  k_sort_hist<<<hist_blocks, kSortThreads, 0, s>>>(keys[0], n_dev, n_cap, passes, ghist);
  *launches += 1;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    k_sort_pass<kPassItems><<<(unsigned)tiles, kSortThreads, 0, s>>>(
        keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_dev, n_cap, 8 * p, ghist + p * kRadix, tickets + p,
        status + (size_t)p * tiles * kRadix, dev_status);
    *launches += 1;
    cur ^= 1;
  }
  *err = cudaGetLastError();
  return cur;
}

}  // namespace gmr
