// The optimisation loop around the renderer (Sec. 3.1): the parameter
// update and the geometric error metric.
//
// Update: Adam (Kingma and Ba, 2015) per element, or VectorAdam (the
// optimiser the paper uses, Sec. 3.1): the second moment of a vertex is kept
// per 3-vector from its squared gradient norm, so the step does not depend on
// the orientation of the coordinate axes. With g the gradient, t the step
// number (from 1):
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2 (or |g|^2 per vertex),
//   p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
//
// Metric: the chamfer distance (the paper's CD, Sec. 3.1) between two point
// sets A and B, taken here as mean_a min_b |a - b|^2 + mean_b min_a |b - a|^2
// over the vertex sets, by brute force (every pair).

#include "gmr_internal.cuh"

namespace gmr {

namespace {

constexpr int kAdamThreads = 256;

// group = 1: plain Adam; group = 3: VectorAdam over consecutive 3-vectors
// (v holds n / 3 entries).
template <int GROUP>
__global__ void __launch_bounds__(kAdamThreads) k_adam(float* __restrict__ p, const float* __restrict__ g,
                                                       float* __restrict__ m, float* __restrict__ v, int64_t n_groups,
                                                       float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * kAdamThreads + threadIdx.x;
  if (i >= n_groups) return;
  float gg[GROUP], mm[GROUP];
  float g2 = 0.0f;
#pragma unroll
  for (int k = 0; k < GROUP; ++k) {
    gg[k] = g[GROUP * i + k];
    g2 = fmaf(gg[k], gg[k], g2);
  }
  const float vn = b2 * v[i] + (1.0f - b2) * g2;
  v[i] = vn;
  const float den = sqrtf(vn / c2) + eps;
#pragma unroll
  for (int k = 0; k < GROUP; ++k) {
    mm[k] = b1 * m[GROUP * i + k] + (1.0f - b1) * gg[k];
    m[GROUP * i + k] = mm[k];
    p[GROUP * i + k] -= lr * (mm[k] / c1) / den;
  }
}

constexpr int kNNThreads = 256;
constexpr int kNNTile = 1024;  // points of B staged in shared memory at a time

// Squared distance from every point of A to its nearest point of B.
__global__ void __launch_bounds__(kNNThreads) k_nn_sqdist(const float* __restrict__ a, int64_t na,
                                                          const float* __restrict__ b, int64_t nb,
                                                          float* __restrict__ out) {
  __shared__ float sb[3][kNNTile];
  const int64_t i = (int64_t)blockIdx.x * kNNThreads + threadIdx.x;
  float ax = 0.f, ay = 0.f, az = 0.f;
  if (i < na) {
    ax = a[3 * i];
    ay = a[3 * i + 1];
    az = a[3 * i + 2];
  }
  float best = INFINITY;
  for (int64_t j0 = 0; j0 < nb; j0 += kNNTile) {
    const int cnt = nb - j0 < kNNTile ? (int)(nb - j0) : kNNTile;
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += kNNThreads) {
      sb[0][k] = b[3 * (j0 + k)];
      sb[1][k] = b[3 * (j0 + k) + 1];
      sb[2][k] = b[3 * (j0 + k) + 2];
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < cnt; ++k) {
      const float dx = ax - sb[0][k], dy = ay - sb[1][k], dz = az - sb[2][k];
      best = fminf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    }
  }
  if (i < na) out[i] = best;
}

}  // namespace

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int group, float lr, float b1,
                        float b2, float eps, int step, cudaStream_t s, int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  const int64_t ng = n / group;
  const unsigned blocks = (unsigned)((ng + kAdamThreads - 1) / kAdamThreads);
  if (group == 3)
    k_adam<3><<<blocks, kAdamThreads, 0, s>>>(p, g, m, v, ng, lr, b1, b2, eps, c1, c2);
  else
    k_adam<1><<<blocks, kAdamThreads, 0, s>>>(p, g, m, v, ng, lr, b1, b2, eps, c1, c2);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_chamfer(const float* a, int64_t na, const float* b, int64_t nb, float* scratch, double* out,
                           cudaStream_t s, int64_t* launches) {
  k_nn_sqdist<<<(unsigned)((na + kNNThreads - 1) / kNNThreads), kNNThreads, 0, s>>>(a, na, b, nb, scratch);
  k_nn_sqdist<<<(unsigned)((nb + kNNThreads - 1) / kNNThreads), kNNThreads, 0, s>>>(b, nb, a, na, scratch + na);
  *launches += 2;
  cudaError_t e = launch_sum_floats(scratch, na, 1.0 / (double)na, out, s, launches);
  if (e != cudaSuccess) return e;
  return launch_sum_floats(scratch + na, nb, 1.0 / (double)nb, out + 1, s, launches);
}

}  // namespace gmr
