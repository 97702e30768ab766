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


// ---------------------------------------------------------------- mesh regularisers
// The two mesh regularisers of the fitting loop (Sec. 3.1; the paper names
// them, this file takes the readings below), with their vertex gradients:
//  * edge length: the variance of the lengths of the 3F face edges (interior
//    edges counted once per face), L_edge = (1/3F) sum_i (l_i - mean l)^2,
//    dL/dv = (2/3F) sum_{i at v} (l_i - mean l) (v - other end) / l_i (the
//    mean's own derivative drops out, its deviations summing to zero);
//  * Laplacian smoothing, uniform weights over the face neighbourhood:
//    delta_v = v - (sum over faces at v of their two other vertices) /
//    (2 |faces at v|), L_lap = (1/V) sum_v |delta_v|^2, dL/dv = (2/V)
//    (delta_v - sum_w delta_w c_wv) with c_wv = (faces holding w and v) /
//    (2 |faces at w|).
// Gradients are added to dL/dverts with float atomics (weighted by w_edge,
// w_lap); the losses (unweighted) are summed in a fixed order.

namespace {

constexpr int kRegThreads = 256;

__device__ __forceinline__ bool reg_face(const int32_t* faces, int f, int32_t V, int& a, int& b, int& c) {
  a = faces[3 * f]; b = faces[3 * f + 1]; c = faces[3 * f + 2];
  return a >= 0 && a < V && b >= 0 && b < V && c >= 0 && c < V;
}

__device__ __forceinline__ float3 reg_v(const float* v, int i) { return make_float3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }

// per face: the three edge lengths; neighbour sums and counts of its corners
__global__ void __launch_bounds__(kRegThreads) k_reg_faces(const float* __restrict__ verts, int32_t V,
                                                          const int32_t* __restrict__ faces, int32_t F,
                                                          float* __restrict__ len, float* __restrict__ nsum,
                                                          float* __restrict__ ncnt) {
  const int f = blockIdx.x * kRegThreads + threadIdx.x;
  if (f >= F) return;
  int id[3];
  if (!reg_face(faces, f, V, id[0], id[1], id[2])) {
    len[3 * f] = len[3 * f + 1] = len[3 * f + 2] = 0.0f;
    return;
  }
  float3 p[3] = {reg_v(verts, id[0]), reg_v(verts, id[1]), reg_v(verts, id[2])};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float3 a = p[k], b = p[(k + 1) % 3];
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    len[3 * f + k] = sqrtf(dx * dx + dy * dy + dz * dz);
    const float3 u = p[(k + 1) % 3], w = p[(k + 2) % 3];
    atomicAdd(nsum + 3 * id[k], u.x + w.x);
    atomicAdd(nsum + 3 * id[k] + 1, u.y + w.y);
    atomicAdd(nsum + 3 * id[k] + 2, u.z + w.z);
    atomicAdd(ncnt + id[k], 2.0f);
  }
}

// per face: edge-length gradient; len[] becomes (l - mean l)^2 for the loss sum
__global__ void __launch_bounds__(kRegThreads) k_reg_edge_grad(const float* __restrict__ verts, int32_t V,
                                                              const int32_t* __restrict__ faces, int32_t F,
                                                              float* __restrict__ len, const double* __restrict__ len_mean,
                                                              float w_edge, float* __restrict__ dverts) {
  const int f = blockIdx.x * kRegThreads + threadIdx.x;
  if (f >= F) return;
  int id[3];
  if (!reg_face(faces, f, V, id[0], id[1], id[2])) return;
  const float lm = (float)*len_mean;
  const float scale = w_edge * 2.0f / (3.0f * (float)F);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float l = len[3 * f + k];
    const float dl = l - lm;
    len[3 * f + k] = dl * dl;
    if (!dverts || !(l > 0.0f)) continue;
    const int ia = id[k], ib = id[(k + 1) % 3];
    const float3 a = reg_v(verts, ia), b = reg_v(verts, ib);
    const float s = scale * dl / l;
    const float gx = s * (a.x - b.x), gy = s * (a.y - b.y), gz = s * (a.z - b.z);
    atomicAdd(dverts + 3 * ia, gx); atomicAdd(dverts + 3 * ia + 1, gy); atomicAdd(dverts + 3 * ia + 2, gz);
    atomicAdd(dverts + 3 * ib, -gx); atomicAdd(dverts + 3 * ib + 1, -gy); atomicAdd(dverts + 3 * ib + 2, -gz);
  }
}

// per vertex: delta_v, |delta_v|^2, the direct gradient term; keeps
// delta_v / (2 |faces at v|) in nsum for the scatter of the neighbour terms
__global__ void __launch_bounds__(kRegThreads) k_reg_lap_vert(const float* __restrict__ verts, int32_t V,
                                                             float* __restrict__ nsum, const float* __restrict__ ncnt,
                                                             float* __restrict__ sq, float w_lap,
                                                             float* __restrict__ dverts) {
  const int v = blockIdx.x * kRegThreads + threadIdx.x;
  if (v >= V) return;
  const float n = ncnt[v];
  float3 d = make_float3(0.f, 0.f, 0.f);
  if (n > 0.0f) {
    const float3 p = reg_v(verts, v);
    d = make_float3(p.x - nsum[3 * v] / n, p.y - nsum[3 * v + 1] / n, p.z - nsum[3 * v + 2] / n);
  }
  sq[v] = d.x * d.x + d.y * d.y + d.z * d.z;
  const float scale = w_lap * 2.0f / (float)V;
  if (dverts) {
    atomicAdd(dverts + 3 * v, scale * d.x);
    atomicAdd(dverts + 3 * v + 1, scale * d.y);
    atomicAdd(dverts + 3 * v + 2, scale * d.z);
  }
  const float inv = n > 0.0f ? 1.0f / n : 0.0f;
  nsum[3 * v] = d.x * inv; nsum[3 * v + 1] = d.y * inv; nsum[3 * v + 2] = d.z * inv;
}

// per face: -(2/V) delta_w / (2 |faces at w|) to each of the two other corners of w
__global__ void __launch_bounds__(kRegThreads) k_reg_lap_scatter(const int32_t* __restrict__ faces, int32_t F,
                                                                int32_t V, const float* __restrict__ dn,
                                                                float w_lap, float* __restrict__ dverts) {
  const int f = blockIdx.x * kRegThreads + threadIdx.x;
  if (f >= F) return;
  int id[3];
  if (!reg_face(faces, f, V, id[0], id[1], id[2])) return;
  const float scale = -w_lap * 2.0f / (float)V;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int w = id[k];
    const float gx = scale * dn[3 * w], gy = scale * dn[3 * w + 1], gz = scale * dn[3 * w + 2];
#pragma unroll
    for (int j = 1; j < 3; ++j) {
      const int u = id[(k + j) % 3];
      atomicAdd(dverts + 3 * u, gx); atomicAdd(dverts + 3 * u + 1, gy); atomicAdd(dverts + 3 * u + 2, gz);
    }
  }
}

}  // namespace

int64_t regularizer_scratch_floats(int32_t V, int32_t F) { return 3 * (int64_t)F + 3 * (int64_t)V + 2 * (int64_t)V; }

cudaError_t launch_regularizers(const float* verts, int32_t V, const int32_t* faces, int32_t F, float w_edge,
                                float w_lap, float* dverts, double* losses, float* scratch, double* mean_slot,
                                cudaStream_t s, int64_t* launches) {
  float* len = scratch;                 // 3F
  float* nsum = len + 3 * (int64_t)F;   // 3V
  float* ncnt = nsum + 3 * (int64_t)V;  // V
  float* sq = ncnt + V;                 // V
  cudaError_t e = cudaMemsetAsync(nsum, 0, sizeof(float) * 4 * (size_t)V, s);  // nsum and ncnt
  if (e != cudaSuccess) return e;
  const unsigned gf = (unsigned)((F + kRegThreads - 1) / kRegThreads), gv = (unsigned)((V + kRegThreads - 1) / kRegThreads);
  k_reg_faces<<<gf, kRegThreads, 0, s>>>(verts, V, faces, F, len, nsum, ncnt);
  *launches += 1;
  if ((e = launch_sum_floats(len, 3 * (int64_t)F, 1.0 / (3.0 * F), mean_slot, s, launches)) != cudaSuccess) return e;
  k_reg_edge_grad<<<gf, kRegThreads, 0, s>>>(verts, V, faces, F, len, mean_slot, w_edge, dverts);
  k_reg_lap_vert<<<gv, kRegThreads, 0, s>>>(verts, V, nsum, ncnt, sq, w_lap, dverts);
  *launches += 2;
  if (dverts) {
    k_reg_lap_scatter<<<gf, kRegThreads, 0, s>>>(faces, F, V, nsum, w_lap, dverts);
    *launches += 1;
  }
  if ((e = launch_sum_floats(len, 3 * (int64_t)F, 1.0 / (3.0 * F), losses, s, launches)) != cudaSuccess) return e;
  return launch_sum_floats(sq, V, 1.0 / (double)V, losses + 1, s, launches);
}

}  // namespace gmr
