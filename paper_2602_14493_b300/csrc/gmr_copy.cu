// gmr_copy_h2d: a host-to-device copy done by a kernel that reads the pinned
// host buffer directly over the bus (zero-copy loads), for the inputs of a
// step that arrive from the host every step (the target images of the
// image loss).
//
// Why a kernel: on the virtualised B300 hosts this library is measured on,
// copy-engine transfers of a few tens of MB reach 15-25 GB/s while a kernel
// with a few hundred KB of loads in flight reaches 25-50 GB/s for the same
// buffer; it runs on any stream, so it overlaps the previous step's compute
// the same way a copy-engine transfer does (it occupies up to kCopyBlocks
// small CTAs while it runs). From kEngineMinBytes up the copy engine is
// faster (the 64-view workload's 329 MB of target images per step: 11.1 ->
// 7.3 ms per end-to-end step) and takes no SM from the compute: such copies
// go to it (one cudaMemcpyAsync).

#include <algorithm>

#include "gmr_internal.cuh"

namespace {

constexpr int kCopyThreads = 256;
// swept 32-1184 CTAs x 4-16 loads in flight with the copies overlapping a
// compute stream: 2 CTAs per SM with 4 loads each is best (20% faster than
// 64 x 8 on a 25 MB input per step)
constexpr int kCopyBlocks = 296;
constexpr int kCopyUnroll = 4;  // 16-byte loads in flight per thread
constexpr int64_t kEngineMinBytes = int64_t(64) << 20;

__global__ void __launch_bounds__(kCopyThreads) k_copy_h2d(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                           int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * kCopyThreads;
  int64_t i = (int64_t)blockIdx.x * kCopyThreads + threadIdx.x;
  for (; i + (kCopyUnroll - 1) * stride < n; i += kCopyUnroll * stride) {
    uint4 v[kCopyUnroll];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; ++u) v[u] = src[i + u * stride];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; ++u) dst[i + u * stride] = v[u];
  }
  for (; i < n; i += stride) dst[i] = src[i];
}

__global__ void k_copy_bytes(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

gmr_status gmr_copy_h2d(void* dst, const void* src, int64_t bytes, gmr_stream stream) {
  if (bytes < 0 || (bytes > 0 && (!dst || !src))) return GMR_ERR_INVALID_ARG;
  if (bytes == 0) return GMR_OK;
  void* dsrc = nullptr;
  if (cudaHostGetDevicePointer(&dsrc, const_cast<void*>(src), 0) != cudaSuccess || !dsrc) {
    cudaGetLastError();  // not page-locked (or not mapped into this device's address space)
    return GMR_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (bytes >= kEngineMinBytes)
    return cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyHostToDevice, s) == cudaSuccess ? GMR_OK : GMR_ERR_CUDA;
  const bool vec = ((reinterpret_cast<uintptr_t>(dsrc) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0;
  const int64_t nvec = vec ? bytes / 16 : 0;
  if (nvec > 0) {
    const int64_t want = (nvec + (int64_t)kCopyThreads * kCopyUnroll - 1) / ((int64_t)kCopyThreads * kCopyUnroll);
    const unsigned blocks = (unsigned)std::min<int64_t>(std::max<int64_t>(want, 1), kCopyBlocks);
    k_copy_h2d<<<blocks, kCopyThreads, 0, s>>>(static_cast<const uint4*>(dsrc), static_cast<uint4*>(dst), nvec);
  }
  const int64_t done = nvec * 16, rest = bytes - done;
  if (rest > 0) {
    const unsigned blocks = (unsigned)std::min<int64_t>((rest + 255) / 256, kCopyBlocks);
    k_copy_bytes<<<blocks, 256, 0, s>>>(static_cast<const uint8_t*>(dsrc) + done, static_cast<uint8_t*>(dst) + done,
                                        rest);
  }
  return cudaGetLastError() == cudaSuccess ? GMR_OK : GMR_ERR_CUDA;
}
