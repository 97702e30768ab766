// Binning of the Gaussians into screen tiles, in (tile, depth, face) order
// (the 3DGS binning, Sec. 2.1), as a two-level radix sort:
//
//  1. most significant digit = the global tile id: the projection counts the
//     pairs of every tile and gives each pair its rank among the tile's
//     pairs (atomics on the tile counters, in whatever order the pairs
//     arrive); an exclusive scan of the counts gives each tile's segment,
//     and k_place_keys writes each pair's 64-bit key (depth bits << 32 |
//     face) to segment start + rank, with no atomics;
//  2. the remaining digits, (depth bits, face), within each tile: segments
//     of up to 512 keys (nearly all) are sorted by one warp each: up to 256
//     keys by a bitonic network in registers (shuffles only), 257 to 512 as
//     two such halves merged through shared memory; longer segments are listed and sorted by one CTA
//     each: up to 4096 keys by a merge sort in shared memory (register
//     bitonic chunks, then merge-path rounds), beyond that by LSD radix
//     passes through global memory on the 8-bit digits that differ within
//     the segment (usually not the depth's exponent byte nor the face
//     index's upper bytes).
//
// Keys are unique (face ids are), so the result is the unique (tile, depth,
// face) order whatever order step 1 put the keys of a segment in.

#include <algorithm>
#include <atomic>

#include "gmr_internal.cuh"

namespace gmr {

namespace {

constexpr int kSegThreads = 256;
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegSmem = 4096;  // keys of a long segment sorted in shared memory
constexpr int kRadix = 256;
// the radix pass gives each digit one thread of the CTA (its run offsets)
static_assert(kSegThreads == kRadix, "cta_radix_pass: one thread per digit");

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

constexpr int kPlaceThreads = 256;

// Key of each pair slot of the projection to segment start + rank. The pair
// count is known only on the device, so the grid is one wave (sized by the
// device, not by the pair capacity: a workspace grown by a larger earlier
// forward would otherwise launch many blocks with nothing to do) striding over
// rounds of U slots per thread; the slot loads of a round, then their
// gathers, are issued together, so the dependent gathers overlap (the
// kernel waits on them: more in flight per thread pays once there are
// enough pairs to fill the wave, see launch_bin_pairs).
// With split binning (pair_quad) the key's low word is face << 4 | the
// pair's quadrants: the order by (depth, face) is unchanged.
template <int U>
__global__ void __launch_bounds__(kPlaceThreads) k_place_keys(
    const unsigned long long* __restrict__ pair_tr, const uint32_t* __restrict__ pair_rec,
    const uint8_t* __restrict__ pair_quad, const uint32_t* __restrict__ rec_key, int32_t F,
    const uint32_t* __restrict__ tile_start, int64_t cap, unsigned long long* __restrict__ keys,
    const Counters* __restrict__ counters) {
  pdl_enter();
  const int64_t n = counters->n_pairs;
  if (n > cap) return;  // overflow: the pair scratch is incomplete
  constexpr int64_t kRound = (int64_t)kPlaceThreads * U;
  for (int64_t base = (int64_t)blockIdx.x * kRound; base < n; base += (int64_t)gridDim.x * kRound) {
    unsigned long long tr[U];
    uint32_t rid[U], key[U], start[U], quad[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * kPlaceThreads + threadIdx.x;
      tr[u] = i < n ? pair_tr[i] : 0ull;
      rid[u] = i < n ? pair_rec[i] : 0u;
      quad[u] = (pair_quad && i < n) ? pair_quad[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * kPlaceThreads + threadIdx.x;
      key[u] = i < n ? rec_key[rid[u]] : 0u;
      start[u] = i < n ? tile_start[(uint32_t)(tr[u] >> 32)] : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * kPlaceThreads + threadIdx.x;
      if (i < n) {
        const uint32_t c = rid[u] / (uint32_t)F;
        const uint32_t face = rid[u] - c * (uint32_t)F;
        keys[start[u] + (uint32_t)tr[u]] =
            ((unsigned long long)key[u] << 32) | (pair_quad ? (face << 4 | quad[u]) : face);
      }
    }
  }
}

// Exclusive scan of one value per thread over the CTA (kSegThreads threads).
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t* sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(v, lane);
  if (lane == 31) sw[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kSegWarps ? sw[lane] : 0u;
    uint32_t wi = warp_incl_scan(w, lane);
    if (lane < kSegWarps) sw[lane] = wi - w;
  }
  __syncthreads();
  const uint32_t r = incl - v + sw[warp];
  __syncthreads();
  return r;
}

// Stable LSD counting pass on the 8-bit digit at `shift` of keys src[0, n)
// -> dst (shared or global memory), by the whole CTA with 3 barriers: warp w
// owns the consecutive chunk [w C, (w + 1) C) of the keys (C a multiple of
// 32), so the order of equal digits is chunk order, then round order within
// a chunk, then lane order (`__match_any_sync` ranks equal digits among the
// lanes of a round). hist holds kSegWarps x kRadix counters.
__device__ void cta_radix_pass(const unsigned long long* src, unsigned long long* dst, int n, int shift,
                               uint32_t* hist, uint32_t* sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int C = ((n + kSegWarps * 32 - 1) / (kSegWarps * 32)) * 32;
  const int c0 = min(n, warp * C), c1 = min(n, c0 + C);
  uint32_t* h = hist + warp * kRadix;
  for (int d = lane; d < kRadix; d += 32) h[d] = 0u;
  __syncwarp();
  // A: digit counts of this warp's chunk
  for (int base = c0; base < c1; base += 32) {
    const int i = base + lane;
    const bool ok = i < c1;
    const uint32_t d = ok ? (uint32_t)(src[i] >> shift) & 0xffu : (uint32_t)(kRadix + lane);
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (ok && (peers & lt) == 0) h[d] += (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // B: start of every (digit, warp) run: digits in order, warps in order
  {
    const int d = threadIdx.x;  // kSegThreads == kRadix
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) {
      const uint32_t c = hist[w * kRadix + d];
      hist[w * kRadix + d] = run;
      run += c;
    }
    const uint32_t start = cta_excl_scan(run, sw);  // barriers inside
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) hist[w * kRadix + d] += start;
  }
  __syncthreads();
  // C: scatter, in the same order as A
  for (int base = c0; base < c1; base += 32) {
    const int i = base + lane;
    const bool ok = i < c1;
    const unsigned long long k = ok ? src[i] : 0ull;
    const uint32_t d = ok ? (uint32_t)(k >> shift) & 0xffu : (uint32_t)(kRadix + lane);
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (ok) dst[h[d] + __popc(peers & lt)] = k;
    __syncwarp();
    if (ok && (peers & lt) == 0) h[d] += (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
}

// Ascending bitonic sort of 32*KPL 64-bit keys held by one warp, element
// e = lane * KPL + r in register r of lane `lane`: the stages that compare
// elements less than KPL apart stay inside a thread (two selects, no
// shuffle), the others exchange whole registers between lanes. The stage
// loops are not unrolled (one body per exchange distance class keeps the
// code small enough for the instruction cache); the register loops are, so
// `v` stays in registers.
template <int KPL>
__device__ __forceinline__ void cmp_lanes(unsigned long long (&v)[KPL], int k, int jl, int lane) {
  // partner lane ^ jl (distance j = jl * KPL >= KPL, so k > KPL: the
  // direction depends on the lane only)
  const bool upper = (lane & jl) != 0;
  const bool asc = ((lane * KPL) & k) == 0;
  const bool take_min = asc != upper;
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[r], jl);
    const bool lt = v[r] < o;
    v[r] = (take_min == lt) ? v[r] : o;
  }
}

// partner in register r ^ J of the same lane (distance J < KPL)
template <int KPL, int J>
__device__ __forceinline__ void cmp_regs(unsigned long long (&v)[KPL], int k, int lane) {
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    if (r & J) continue;
    const bool asc = ((lane * KPL + r) & k) == 0;
    const unsigned long long a = v[r], b = v[r | J];
    const bool sw = asc ? (a > b) : (a < b);
    v[r] = sw ? b : a;
    v[r | J] = sw ? a : b;
  }
}

template <int KPL>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[KPL], int lane) {
  constexpr int N = 32 * KPL;
  constexpr int LOG = KPL == 1 ? 0 : KPL == 2 ? 1 : KPL == 4 ? 2 : 3;
  static_assert(KPL == 1 || KPL == 2 || KPL == 4 || KPL == 8, "KPL");
#pragma unroll 1
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= KPL) {
        cmp_lanes<KPL>(v, k, j >> LOG, lane);
      } else {
        if (KPL > 1 && j == 1) cmp_regs<KPL, 1>(v, k, lane);
        if (KPL > 2 && j == 2) cmp_regs<KPL, 2>(v, k, lane);
        if (KPL > 4 && j == 4) cmp_regs<KPL, 4>(v, k, lane);
      }
    }
  }
}

template <int KPL>
__device__ __forceinline__ void warp_sort_segment(const unsigned long long* __restrict__ gk, int L,
                                                  uint32_t* __restrict__ out, int lane) {
  unsigned long long v[KPL];
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int e = r * 32 + lane;  // any input order suits a sort: the coalesced one
    v[r] = e < L ? gk[e] : ~0ull;
  }
  warp_bitonic<KPL>(v, lane);
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int e = lane * KPL + r;
    if (e < L) out[e] = (uint32_t)v[r];
  }
}

// Position of element e (0..255) of a sorted half in shared memory: e with
// its low four bits XORed with the next four. For each register r, the 32
// lanes' elements lane * 8 + r then fall on distinct 8-byte bank pairs two
// by two (two wavefronts, the minimum for 256 bytes).
__device__ __forceinline__ int swz16(int e) { return e ^ ((e >> 4) & 15); }

// Ascending sort of 257 to 512 64-bit keys by one warp (s holds 512 keys):
// each half of 256 is sorted in registers (the second padded with all-ones
// keys) and stored to s in the swizzled order; then lane l merges outputs
// 16 l .. 16 l + 15 of the two sorted halves (merge path: a binary search
// for where that output diagonal crosses them, taking from the first half
// on ties, then 16 sequential steps) and writes their face ids. (A bitonic
// network over the 512 keys in shared memory took 45 exchange stages, each
// lane 8 pairs of loads and stores per stage, and was bound by the
// shared-memory instruction queue.)
__device__ __forceinline__ void warp_sort_512(const unsigned long long* __restrict__ gk, int L,
                                              uint32_t* __restrict__ out, unsigned long long* s, int lane) {
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    unsigned long long v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = h * 256 + r * 32 + lane;
      v[r] = e < L ? gk[e] : ~0ull;
    }
    warp_bitonic<8>(v, lane);
#pragma unroll
    for (int r = 0; r < 8; ++r) s[h * 256 + swz16(lane * 8 + r)] = v[r];
  }
  __syncwarp();
  const unsigned long long* A = s;
  const unsigned long long* B = s + 256;
  const int d = lane * 16;
  int lo = max(0, d - 256), hi = min(d, 256);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (A[swz16(mid)] <= B[swz16(d - 1 - mid)]) lo = mid + 1;
    else hi = mid;
  }
  int i = lo, j = d - lo;
  unsigned long long a = i < 256 ? A[swz16(i)] : ~0ull, b = j < 256 ? B[swz16(j)] : ~0ull;
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    const bool take_a = j >= 256 || (i < 256 && a <= b);
    if (d + k < L) out[d + k] = (uint32_t)(take_a ? a : b);
    if (take_a) {
      ++i;
      a = i < 256 ? A[swz16(i)] : ~0ull;
    } else {
      ++j;
      b = j < 256 ? B[swz16(j)] : ~0ull;
    }
  }
  __syncwarp();
}

constexpr int kWarpSortMax = 512;   // keys sorted by one warp
constexpr int kTileSortThreads = 64;  // small CTAs: tiles of uneven length retire independently
constexpr int kTilesPerCta = kTileSortThreads / 32;

// One warp per global tile, warp w taking the w-th tile of the compositing
// order: write the range and, at position w, the tile's descriptor (tile,
// view, range) for the compositing CTA w; sort segments of up to 256 keys
// in registers (8 per lane at most, which keeps the register count and so
// the occupancy at that of the common case) and of 257 to 512 keys as two
// register-sorted halves merged through shared memory; list longer segments
// for k_long_sort.
__global__ void __launch_bounds__(kTileSortThreads) k_tile_sort(
    const uint32_t* __restrict__ tile_start, int64_t n_tiles, const unsigned long long* __restrict__ keys,
    uint32_t* __restrict__ pair_face, uint2* __restrict__ ranges, uint32_t* __restrict__ long_list,
    const uint32_t* __restrict__ tile_order, const ViewInfo* __restrict__ views, int32_t C,
    uint4* __restrict__ tile_desc, Counters* __restrict__ counters, int64_t cap) {
  pdl_enter();
  __shared__ unsigned long long s_keys[kTilesPerCta][kWarpSortMax];
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kTilesPerCta + (threadIdx.x >> 5);
  if (w >= n_tiles) return;
  // warps take the tiles heaviest first, as the compositing does
  int64_t t = 0;
  if (lane == 0) t = tile_of_block(tile_order, counters->n_class, n_tiles, w);
  t = __shfl_sync(0xffffffffu, t, 0);
  const uint32_t P = counters->n_pairs;
  if ((int64_t)P > cap) {  // overflow: the keys were not written
    if (lane == 0) {
      ranges[t] = make_uint2(0u, 0u);
      tile_desc[w] = make_uint4((uint32_t)t, (uint32_t)find_view(views, C, (int)t), 0u, 0u);
    }
    if (t == 0 && lane == 0) atomicOr(&counters->status, kDevOverflow);
    return;
  }
  const uint32_t start = tile_start[t];
  const uint32_t end = (t + 1 < n_tiles) ? tile_start[t + 1] : P;
  const int L = (int)(end - start);
  if (lane == 0) {
    const uint2 rg = L > 0 ? make_uint2(start, end) : make_uint2(0u, 0u);
    ranges[t] = rg;
    // what the compositing CTA at this position needs first, in one record
    tile_desc[w] = make_uint4((uint32_t)t, (uint32_t)find_view(views, C, (int)t), rg.x, rg.y);
  }
  if (L <= 0) return;
  const unsigned long long* gk = keys + start;
  uint32_t* out = pair_face + start;
  if (L == 1) {
    if (lane == 0) out[0] = (uint32_t)gk[0];
  } else if (L <= 32) {
    warp_sort_segment<1>(gk, L, out, lane);
  } else if (L <= 64) {
    warp_sort_segment<2>(gk, L, out, lane);
  } else if (L <= 128) {
    warp_sort_segment<4>(gk, L, out, lane);
  } else if (L <= 256) {
    warp_sort_segment<8>(gk, L, out, lane);
  } else if (L <= kWarpSortMax) {
    warp_sort_512(gk, L, out, s_keys[threadIdx.x >> 5], lane);
  } else if (lane == 0) {
    long_list[atomicAdd(&counters->n_long, 1u)] = (uint32_t)t;
  }
}

// One merge round of a CTA-wide merge sort: the sorted runs of length R in
// src[0, n) (the last one possibly shorter) are merged pairwise into dst
// (R a power of two, n a multiple of 128). Thread t writes the ipt outputs
// from t ipt on (ipt the power of two >= n / kSegThreads, which divides 2R,
// so no thread's outputs cross a pair of runs): it finds where that output
// diagonal crosses the merge path of its two runs by binary search (taking
// from the first run on ties), then merges its outputs sequentially.
__device__ __forceinline__ void cta_merge_round(const unsigned long long* __restrict__ src,
                                                unsigned long long* __restrict__ dst, int n, int R) {
  int ipt = 1;
  while (ipt * kSegThreads < n) ipt <<= 1;
  const int out0 = threadIdx.x * ipt;
  if (out0 >= n) return;
  const int pair0 = out0 & ~(2 * R - 1);
  const int la = min(R, n - pair0), lb = max(0, min(R, n - pair0 - R));
  const unsigned long long* A = src + pair0;
  const unsigned long long* B = A + R;
  const int diag = out0 - pair0;
  int lo = max(0, diag - lb), hi = min(diag, la);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  int i = lo, j = diag - lo;
  unsigned long long a = i < la ? A[i] : ~0ull, b = j < lb ? B[j] : ~0ull;
  for (int k = 0; k < ipt; ++k) {
    const bool take_a = j >= lb || (i < la && a <= b);
    dst[out0 + k] = take_a ? a : b;
    if (take_a) {
      ++i;
      a = i < la ? A[i] : ~0ull;
    } else {
      ++j;
      b = j < lb ? B[j] : ~0ull;
    }
  }
}

// Each warp sorts the 32 KPL-key chunks warp, warp + kSegWarps, ... of the
// segment gk[0, L) (padded with all-ones keys) in registers and stores them,
// sorted, to s. Any input order suits a sort: the loads take the coalesced
// (and bank-conflict-free) one.
template <int KPL>
__device__ __forceinline__ void cta_sort_chunks(const unsigned long long* __restrict__ gk, int L,
                                                unsigned long long* s, int nchunks, int warp, int lane) {
  for (int c = warp; c < nchunks; c += kSegWarps) {
    unsigned long long v[KPL];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      const int e = c * (32 * KPL) + r * 32 + lane;
      v[r] = e < L ? gk[e] : ~0ull;
    }
    warp_bitonic<KPL>(v, lane);
    ulonglong2* p = reinterpret_cast<ulonglong2*>(s + c * (32 * KPL) + lane * KPL);
#pragma unroll
    for (int r = 0; r < KPL / 2; ++r) p[r] = make_ulonglong2(v[2 * r], v[2 * r + 1]);
  }
}

// Segments longer than kWarpSortMax: one CTA each (a persistent grid over
// the long list). Up to kSegSmem keys: a merge sort in dynamic shared memory
// (register-sorted chunks of 128 keys, or 256 above 1024 keys, the last one
// padded with all-ones keys, then ceil(log2(chunks)) merge rounds). Longer:
// LSD radix passes on the 8-bit digits that differ within the segment,
// through global memory.
__global__ void __launch_bounds__(kSegThreads) k_long_sort(const uint32_t* __restrict__ long_list,
                                                           Counters* __restrict__ counters,
                                                           const uint2* __restrict__ ranges,
                                                           unsigned long long* __restrict__ keys,
                                                           unsigned long long* __restrict__ keys_tmp,
                                                           uint32_t* __restrict__ pair_face) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned long long s_dyn[];
  unsigned long long* sa = s_dyn;                 // kSegSmem keys
  unsigned long long* sb = s_dyn + kSegSmem;      // kSegSmem keys
  uint32_t* hist = reinterpret_cast<uint32_t*>(s_dyn + 2 * kSegSmem);  // kSegWarps x kRadix
  __shared__ uint32_t sw[32];
  __shared__ unsigned long long red_and[kSegWarps], red_or[kSegWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ uint32_t s_next;
  const uint32_t nlong = counters->n_long;
  // segments are taken from a shared cursor, not by CTA index: a CTA that
  // starts late (or shares its SM) takes fewer
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(&counters->long_next, 1u);
    __syncthreads();
    const uint32_t li = s_next;
    __syncthreads();
    if (li >= nlong) break;
    const uint2 rg = ranges[long_list[li]];
    const int L = (int)(rg.y - rg.x);
    unsigned long long* gk = keys + rg.x;
    if (L <= kSegSmem) {
      // chunks of 128 keys (one per warp) up to 1024 keys, of 256 beyond
      const int cs = L <= 1024 ? 128 : 256;
      const int nch = (L + cs - 1) / cs;
      const int n = nch * cs;
      if (cs == 128) cta_sort_chunks<4>(gk, L, sa, nch, warp, lane);
      else cta_sort_chunks<8>(gk, L, sa, nch, warp, lane);
      __syncthreads();
      unsigned long long* src = sa;
      unsigned long long* dst = sb;
      for (int R = cs; R < n; R <<= 1) {
        cta_merge_round(src, dst, n, R);
        __syncthreads();
        unsigned long long* tmp = src;
        src = dst;
        dst = tmp;
      }
      for (int i = threadIdx.x; i < L; i += kSegThreads) pair_face[rg.x + i] = (uint32_t)src[i];
      __syncthreads();
      continue;
    }
    unsigned long long a = ~0ull, o = 0ull;
    for (int i = threadIdx.x; i < L; i += kSegThreads) {
      const unsigned long long k = gk[i];
      a &= k;
      o |= k;
    }
#pragma unroll
    for (int s2 = 16; s2 > 0; s2 >>= 1) {
      a &= __shfl_xor_sync(0xffffffffu, a, s2);
      o |= __shfl_xor_sync(0xffffffffu, o, s2);
    }
    if (lane == 0) {
      red_and[warp] = a;
      red_or[warp] = o;
    }
    __syncthreads();
    unsigned long long diff = 0;
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) diff |= red_and[w] ^ red_or[w];
    unsigned long long* src = gk;
    unsigned long long* dst = keys_tmp + rg.x;
    for (int shift = 0; shift < 64; shift += 8) {
      if (((diff >> shift) & 0xffull) == 0) continue;  // uniform over the CTA
      cta_radix_pass(src, dst, L, shift, hist, sw);
      unsigned long long* tmp = src;
      src = dst;
      dst = tmp;
    }
    for (int i = threadIdx.x; i < L; i += kSegThreads) pair_face[rg.x + i] = (uint32_t)src[i];
    __syncthreads();
  }
}

constexpr size_t kLongSortSmem = (2 * kSegSmem) * sizeof(unsigned long long) + kSegWarps * kRadix * sizeof(uint32_t);

// Split binning: one warp per binning (16x16) tile, at its compositing
// position w: the tile's sorted list, 32 entries at a time (lane l takes
// entry c + l: face << 4 | the quadrants its record's 8x8 rectangle holds,
// from the projection), is dealt to the lists of those quadrants (a ballot
// per quadrant keeps the order), quadrant q's list from 4 start + q n; lanes
// 0-3 then write the quadrants' descriptors at positions 4 w + q (kNoTile
// for a quadrant beyond the image) and their ranges. A record is in the 8x8
// tile (X, Y) exactly when its rectangle holds it, and then also in the
// binning tile (X / 2, Y / 2), so the quadrant lists are the 8x8 binning's,
// in its order.
constexpr int kSplitThreads = 128;
__global__ void __launch_bounds__(kSplitThreads) k_split_quads(const uint4* __restrict__ desc_b, int64_t n_btiles,
                                                               const uint32_t* __restrict__ pair_face,
                                                               const ViewInfo* __restrict__ views,
                                                               uint32_t* __restrict__ pair_face_c,
                                                               uint4* __restrict__ desc_c, uint2* __restrict__ range_c) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (kSplitThreads / 32) + (threadIdx.x >> 5);
  if (w >= n_btiles) return;
  const uint4 d = desc_b[w];  // (binning tile, view, start, end)
  const ViewInfo& v = views[d.y];
  const int lt = (int)d.x - v.btile_base;
  const int by = lt / v.btiles_x, bx = lt - by * v.btiles_x;
  const uint32_t n = d.w - d.z;
  const uint32_t base = 4u * d.z;
  const uint32_t below = (1u << lane) - 1u;
  bool valid[4];
  uint32_t cnt[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    valid[q] = 2 * bx + (q & 1) < v.tiles_x && 2 * by + (q >> 1) < v.tiles_y;
    cnt[q] = 0;
  }
  // the next chunk's entries are loaded before this chunk is dealt
  uint32_t e_next = lane < n ? __ldg(pair_face + d.z + lane) : 0u;
  for (uint32_t c = 0; c < n; c += 32) {
    const uint32_t i = c + lane;
    const uint32_t e = e_next;
    e_next = i + 32 < n ? __ldg(pair_face + d.z + i + 32) : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool in = valid[q] && ((e >> q) & 1u);
      const uint32_t bal = __ballot_sync(0xffffffffu, in);
      if (in) pair_face_c[base + (uint32_t)q * n + cnt[q] + __popc(bal & below)] = e >> 4;
      cnt[q] += __popc(bal);
    }
  }
  if (lane < 4) {
    const int q = lane;
    const uint32_t cq = q == 0 ? cnt[0] : q == 1 ? cnt[1] : q == 2 ? cnt[2] : cnt[3];
    const int Xq = 2 * bx + (q & 1), Yq = 2 * by + (q >> 1);
    if (Xq < v.tiles_x && Yq < v.tiles_y) {
      const uint32_t g = (uint32_t)v.tile_base + (uint32_t)Yq * (uint32_t)v.tiles_x + (uint32_t)Xq;
      const uint32_t lo = base + (uint32_t)q * n;
      const uint2 rg = cq > 0 ? make_uint2(lo, lo + cq) : make_uint2(0u, 0u);
      desc_c[4 * w + q] = make_uint4(g, d.y, rg.x, rg.y);
      range_c[g] = rg;
    } else {
      desc_c[4 * w + q] = make_uint4(kNoTile, d.y, 0u, 0u);
    }
  }
}

// Debug: global tile id of every sorted pair, from the ranges.
__global__ void k_expand_tiles(const uint2* __restrict__ ranges, int64_t n_tiles, uint32_t* __restrict__ tile_ids) {
  const int64_t t = blockIdx.x;
  if (t >= n_tiles) return;
  const uint2 r = ranges[t];
  for (uint32_t i = r.x + threadIdx.x; i < r.y; i += blockDim.x) tile_ids[i] = (uint32_t)t;
}

}  // namespace

cudaError_t launch_bin_pairs(const Workspace& ws, int64_t n_rec, int32_t F, const ViewInfo* views, int32_t C,
                             int64_t n_tiles, bool split, cudaStream_t s, int64_t* launches) {
  if (n_rec > 0 && ws.cap_pairs > 0) {
    // slots per thread and round by the workload's size (the pair count is
    // on the device; the records, 1-3 pairs each, are known here): 4 up to
    // 1M records, 8 up to 10M, 12 beyond (swept 4-12: 8 took the 64-view
    // workload's binning, 5.2M records, 0.509 -> 0.472 ms, 12 the level-8
    // mesh's, 21M records, 2.06 -> 1.78 ms; on 8 views of a 20K-face mesh
    // 4 is 7% faster than 8: fewer, longer threads leave SMs idle)
    const int U = n_rec <= (int64_t(1) << 20) ? 4 : n_rec <= int64_t(10) * (1 << 20) ? 8 : 12;
    auto kern = U == 4 ? k_place_keys<4> : U == 8 ? k_place_keys<8> : k_place_keys<12>;
    // one wave (the blocks that are resident at once), or fewer for a small
    // pair capacity: a grid sized for more blocks per SM than its registers
    // allow runs the rest as a second wave as long as the first
    const int64_t blocks = std::min<int64_t>((ws.cap_pairs + kPlaceThreads * U - 1) / (kPlaceThreads * U),
                                             resident_grid(kern, kPlaceThreads));
    cudaError_t e = launch_chained(kern, true, dim3((unsigned)blocks), dim3(kPlaceThreads), 0, s,
                                   (const unsigned long long*)ws.pair_key[1], (const uint32_t*)ws.pair_face,
                                   split ? (const uint8_t*)ws.pair_quad : nullptr, (const uint32_t*)ws.rec_key, F,
                                   (const uint32_t*)ws.tile_start, ws.cap_pairs, ws.pair_key[0],
                                   (const Counters*)ws.counters);
    *launches += 1;
    if (e != cudaSuccess) return e;
  }
  if (n_tiles > 0) {
    // the dynamic shared memory limit is a per-device attribute of the kernel
    static std::atomic<bool> smem_set[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !smem_set[dev].load()) {
      e = cudaFuncSetAttribute(k_long_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSortSmem);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) smem_set[dev].store(true);
    }
    e = launch_chained(k_tile_sort, false, dim3((unsigned)((n_tiles + kTilesPerCta - 1) / kTilesPerCta)),
                       dim3(kTileSortThreads), 0, s, (const uint32_t*)ws.tile_start, n_tiles,
                       (const unsigned long long*)ws.pair_key[0], ws.pair_face, ws.tile_range, ws.long_tiles,
                       (const uint32_t*)ws.tile_order, views, C, ws.tile_desc, ws.counters, ws.cap_pairs);
    if (e != cudaSuccess) return e;
    e = launch_chained(k_long_sort, true, dim3((unsigned)resident_grid(k_long_sort, kSegThreads, kLongSortSmem)),
                       dim3(kSegThreads), kLongSortSmem, s,
                       (const uint32_t*)ws.long_tiles, ws.counters, (const uint2*)ws.tile_range,
                       ws.pair_key[0], ws.pair_key[1], ws.pair_face);
    *launches += 2;
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_split_quads(const Workspace& ws, const ViewInfo* views, int64_t n_btiles, cudaStream_t s,
                               int64_t* launches) {
  if (n_btiles <= 0) return cudaSuccess;
  if (ws.cap_split_pairs < 4 * ws.cap_pairs || ws.cap_split_tiles < 4 * n_btiles) return cudaErrorInvalidValue;
  constexpr int kPerCta = kSplitThreads / 32;
  cudaError_t e = launch_chained(k_split_quads, true, dim3((unsigned)((n_btiles + kPerCta - 1) / kPerCta)),
                                 dim3(kSplitThreads), 0, s, (const uint4*)ws.tile_desc, n_btiles,
                                 (const uint32_t*)ws.pair_face, views, ws.pair_face_c, ws.tile_desc_c,
                                 ws.tile_range_c);
  *launches += 1;
  return e;
}

cudaError_t launch_expand_tiles(const uint2* ranges, int64_t n_tiles, uint32_t* tile_ids, cudaStream_t s,
                                int64_t* launches) {
  if (n_tiles <= 0) return cudaSuccess;
  k_expand_tiles<<<(unsigned)n_tiles, 128, 0, s>>>(ranges, n_tiles, tile_ids);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace gmr
