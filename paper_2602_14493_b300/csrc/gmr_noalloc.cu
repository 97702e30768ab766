// gmr_l2_loss_noalloc: the squared-error loss and its gradient without any
// device allocation and without a context.
//
// Who needs this: code that must not call cudaMalloc at the point where it
// computes the loss. cudaMalloc can synchronise the device and take global
// driver locks, so a real-time or latency-critical loop cannot afford it; a
// process whose device memory is entirely managed by its own pool (or by a
// framework's caching allocator that must stay the only owner) is not
// allowed to make side allocations; and code on a path where an allocation
// failure cannot be handled (error recovery, shutdown) must not depend on
// one. Such callers pass their own input and output buffers and
// get the partial sums of the reduction from a fixed array compiled into
// this library.
//
// The scratch array lives in device memory of every GPU that loads the
// library, from load until process exit (593 doubles, 4,744 bytes per GPU:
// the loss kernel's grid never has more than 592 blocks, whatever n). Its
// device address is looked up once per device with cudaGetSymbolAddress,
// during the first call made with that device current; make that first call
// before any stream capture that includes this entry point. The address is
// kept for the life of the process: after cudaDeviceReset() of a device the
// library's device code is loaded again elsewhere, so this entry point must
// not be called on that device afterwards. Each GPU has its own copy, and all
// calls on one GPU share it: two calls whose work can overlap on the same GPU
// (for example on two streams without an ordering between them) race on it,
// so the caller must order them. The array's first slot is the loss
// kernel's completion counter: it starts at zero (static storage) and every
// call leaves it at zero; every call writes all the partial sums it later
// reads, so the previous call's leftovers are never used.

#include <mutex>

#include "gmr_internal.cuh"

namespace {

// Completion counter + partial sums of one call (one double per block of
// the loss kernel's grid), sized for the largest grid it launches.
constexpr int64_t kNoAllocPartials = 1 + gmr::kL2LossMaxBlocks;
static_assert(gmr::l2_loss_partials_needed(INT64_MAX / 2) == kNoAllocPartials,
              "the scratch array holds the partials of every n");
static __device__ __align__(256) double g_l2_partials[kNoAllocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Device address of g_l2_partials on the current device (looked up once).
cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_l2_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gmr_status gmr_l2_loss_noalloc(const float* img, const float* target, int64_t n, float* dL_dimg,
                                          double* loss, gmr_stream stream) {
  if (n < 0 || !loss || (n > 0 && (!img || !target || !dL_dimg))) return GMR_ERR_INVALID_ARG;
  // a bound of this entry point (one call's work stays below ~1 GB of
  // traffic), not of the scratch array, which fits every n
  if (n > GMR_L2_NOALLOC_MAX_ELEMS) return GMR_ERR_CAPACITY;
  double* partials = nullptr;
  if (partials_address(&partials) != cudaSuccess) {
    cudaGetLastError();
    return GMR_ERR_CUDA;
  }
  int64_t launches = 0;
  cudaError_t e = gmr::launch_l2_loss(img, target, n, dL_dimg, loss, partials, kNoAllocPartials,
                                      (cudaStream_t)stream, &launches);
  return e == cudaSuccess ? GMR_OK : GMR_ERR_CUDA;
}
