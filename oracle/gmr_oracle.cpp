// Gaussian Mesh Renderer -- FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
// CUDA path is checked against. Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg load it. It shares no code, header, table or
// constant generator with the CUDA library, and the library never calls it.
//
// What it computes, in the paper's order:
//   * conversion of each facet to a Gaussian (Sec. 2.2): Gram-Schmidt facet
//     frame (Eq. 3), centroid (Eq. 4), barycentric parametrisation (Eq. 5),
//     uniform-density second moments by exact integration (Eq. 6-8), 2D
//     covariance (Eq. 9), eigendecomposition (Eq. 10), lifting (Eq. 11),
//     area matching (Eq. 12), 3D covariance (Eq. 13, or Eq. 15 literally),
//     face colour (Eq. 16) and opacity (Sec. 2.2, colour assignment);
//   * the standard 3DGS image formation the paper renders with (Sec. 2.1):
//     EWA projection of each Gaussian to the image plane with a 0.3 px^2
//     low-pass dilation, and front-to-back alpha compositing of every pixel by
//     brute force over ALL visible Gaussians sorted by (depth key, face index);
//   * a hand-derived reverse-mode backward pass of the above in FP64, and a
//     forward-mode (dual number) directional derivative used to pin it;
//   * the FP32 binning specification (depth key, screen-space rectangle of
//     tiles) that both sides evaluate with the same IEEE operations.
//
// Readings where the paper is silent (3DGS constants: alpha in
// [1/255, 0.99], stop before the transmittance would fall below 1e-4,
// dilation 0.3, no skip on a rounded-positive exponent; opacity clamped to
// [0, 1]; degenerate facets become zero-covariance points) are stated next to
// the code that takes them.
//
// Parity status: every function here is pinned by the CPU test suite
// (closed forms, quadrature, invariants, brute force, finite differences,
// dual numbers); none is "parity unpinned".
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (no -ffast-math).

#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// Host threads the oracle's loops use (OpenMP). Every parallel loop writes
// disjoint outputs, and every sum over pixels, views or faces is formed in the
// same fixed order as with one thread, so results do not depend on it.
int g_threads = 1;

// Binned compositing (off by default; gmr_oracle_set_binned): each pixel
// walks only the faces that a uniform grid of kCell x kCell-pixel cells lists
// for its cell, instead of every visible face. Same decisions, same order,
// same results as the brute force (tested on the CPU), much less work.
bool g_binned = false;
constexpr int kCell = 16;

// ---------------------------------------------------------------- constants
// 3DGS compositing constants (Sec. 2.1 follows the standard 3DGS rasterizer,
// which the paper does not restate).
const double kAlphaMin = 1.0 / 255.0;
const double kAlphaMax = 0.99;
const double kTMin = 1e-4;
const double kDilation = 0.3;
// Eq. 12
const double kEps = 1e-14;
const double kSz = 1e-6;
const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
// Forward-mode derivative carrier: value v and derivative d along one
// direction. Comparisons look at the value only, so every discrete decision
// (threshold, clamp, sort) is the one the plain FP64 evaluation takes.
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator==(Dual a, Dual b) { return a.v == b.v; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual atan2(Dual y, Dual x) {
  double r2 = x.v * x.v + y.v * y.v;
  return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

using std::sqrt;
using std::exp;
using std::sin;
using std::cos;
using std::atan2;

template <class T> inline T tmax(T a, T b) { return (a < b) ? b : a; }
template <class T> inline T tmin(T a, T b) { return (b < a) ? b : a; }

// ---------------------------------------------------------------- small vectors
template <class T> struct V3 { T x, y, z; };
template <class T> inline V3<T> mk(T x, T y, T z) { V3<T> r; r.x = x; r.y = y; r.z = z; return r; }
template <class T> inline V3<T> operator+(V3<T> a, V3<T> b) { return mk<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> inline V3<T> operator-(V3<T> a, V3<T> b) { return mk<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> inline V3<T> operator*(T s, V3<T> a) { return mk<T>(s * a.x, s * a.y, s * a.z); }
template <class T> inline T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(V3<T> a, V3<T> b) {
  return mk<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class T> inline T norm(V3<T> a) { return sqrt(dot(a, a)); }

// ---------------------------------------------------------------- inputs
// Camera as handed in: world-to-camera R (row-major), t, pinhole intrinsics,
// image size, near plane. All FP32 on input.
struct Cam {
  float R[9], t[3], fx, fy, cx, cy, znear;
  int W, H;
};

std::vector<Cam> read_cams(const float* cam_f, const int* cam_i, int C) {
  std::vector<Cam> cams(C);
  for (int c = 0; c < C; ++c) {
    const float* p = cam_f + 17 * c;
    for (int k = 0; k < 9; ++k) cams[c].R[k] = p[k];
    for (int k = 0; k < 3; ++k) cams[c].t[k] = p[9 + k];
    cams[c].fx = p[12]; cams[c].fy = p[13]; cams[c].cx = p[14]; cams[c].cy = p[15];
    cams[c].znear = p[16];
    cams[c].W = cam_i[2 * c]; cams[c].H = cam_i[2 * c + 1];
  }
  return cams;
}

// ---------------------------------------------------------------- conversion
// One facet's Gaussian, Sec. 2.2. cov is row-major 3x3.
template <class T> struct FaceGauss {
  T mean[3];
  T cov[9];
  bool degenerate;
  // intermediates kept for the pins and the reverse pass
  T xj, xk, yk;          // local 2D vertex coordinates (v_i at the origin)
  T sxx, sxy, syy;       // Sigma^(2D), Eq. 9
  T lam1, lam2;          // Eq. 10
  T kappa, area;         // Eq. 12
  V3<T> xa, ya, n;       // frame axes (columns of R_f)
};

// Second moment E[f g] of the uniform density on the triangle, with f and g
// affine in the barycentric coordinates of Eq. 5:
//   f(a,b) = f0 + a*fp + b*fq,  g(a,b) = g0 + a*gp + b*gq.
// dA = 2|A| da db over the unit simplex, so E[h] = 2 * int_simplex h. The
// monomial integrals over the unit simplex are 1/2 (1), 1/6 (a or b),
// 1/12 (a^2 or b^2) and 1/24 (ab), which make Eq. 6-8 exact (no sampling).
template <class T>
T simplex_moment(T f0, T fp, T fq, T g0, T gp, T gq) {
  T s = f0 * g0 * T(0.5)
      + (f0 * gp + fp * g0) * T(1.0 / 6.0)
      + (f0 * gq + fq * g0) * T(1.0 / 6.0)
      + fp * gp * T(1.0 / 12.0)
      + (fp * gq + fq * gp) * T(1.0 / 24.0)
      + fq * gq * T(1.0 / 12.0);
  return T(2.0) * s;
}

// cov_mode 0: Eq. 13 (area-matched eigen scales, s_z = 1e-6).
// cov_mode 1: Eq. 15 literally (raw Sigma^(2D) embedded, zero normal variance).
template <class T>
FaceGauss<T> convert_face(V3<T> vi, V3<T> vj, V3<T> vk, int cov_mode) {
  FaceGauss<T> g;
  for (int k = 0; k < 9; ++k) g.cov[k] = T(0.0);
  g.degenerate = false;
  // Eq. 3: orthonormal frame on the facet, origin v_i, x along v_j - v_i,
  // y by Gram-Schmidt of v_k - v_i, z the facet normal.
  V3<T> e1 = vj - vi;
  V3<T> e2 = vk - vi;
  T xj = norm(e1);
  if (!(val(xj) > 0.0)) { g.degenerate = true; }
  V3<T> xa = mk<T>(T(0.0), T(0.0), T(0.0)), ya = xa, n = xa;
  T xk = T(0.0), yk = T(0.0);
  if (!g.degenerate) {
    xa = (T(1.0) / xj) * e1;
    xk = dot(e2, xa);
    V3<T> w = e2 - xk * xa;
    yk = norm(w);
    if (!(val(yk) > 0.0)) g.degenerate = true;
    else {
      ya = (T(1.0) / yk) * w;
      n = cross(xa, ya);
    }
  }
  if (g.degenerate) {
    // Collinear or coincident vertices: |A| = 0, kappa = 0 and the frame is
    // undefined. Reading: a zero-covariance point at the vertex mean.
    V3<T> m = T(1.0 / 3.0) * (vi + vj + vk);
    g.mean[0] = m.x; g.mean[1] = m.y; g.mean[2] = m.z;
    g.xj = g.xk = g.yk = T(0.0);
    g.sxx = g.sxy = g.syy = T(0.0);
    g.lam1 = g.lam2 = g.kappa = g.area = T(0.0);
    g.xa = g.ya = g.n = mk<T>(T(0.0), T(0.0), T(0.0));
    return g;
  }
  // 2D vertices: v_i = (0,0), v_j = (xj, 0), v_k = (xk, yk).
  T xi = T(0.0), yi = T(0.0), yj = T(0.0);
  // Eq. 4: centroid.
  T mux = (xi + xj + xk) / T(3.0);
  T muy = (yi + yj + yk) / T(3.0);
  // Eq. 5-8: barycentric parametrisation and exact second moments.
  T Ex2 = simplex_moment(xi, xj - xi, xk - xi, xi, xj - xi, xk - xi);
  T Exy = simplex_moment(xi, xj - xi, xk - xi, yi, yj - yi, yk - yi);
  T Ey2 = simplex_moment(yi, yj - yi, yk - yi, yi, yj - yi, yk - yi);
  // Eq. 9
  T sxx = Ex2 - mux * mux;
  T sxy = Exy - mux * muy;
  T syy = Ey2 - muy * muy;
  // Eq. 10: Sigma2D = U diag(l1, l2) U^T, l1 >= l2; U is the rotation by
  // theta = atan2(2 sxy, sxx - syy) / 2.
  T th = T(0.5) * atan2(T(2.0) * sxy, sxx - syy);
  T c = cos(th), s = sin(th);
  T u1x = c, u1y = s, u2x = -s, u2y = c;
  T lam1 = sxx * c * c + T(2.0) * sxy * c * s + syy * s * s;
  T lam2 = sxx * s * s - T(2.0) * sxy * c * s + syy * c * c;
  // Eq. 11: lift the principal directions into 3D.
  V3<T> x3 = u1x * xa + u1y * ya;
  V3<T> y3 = u2x * xa + u2y * ya;
  // |A|: half base times height in the local frame.
  T area = T(0.5) * xj * yk;
  // Eq. 12
  T kappa = area / (T(kPi) * sqrt(tmax(lam1 * lam2, T(kEps))));
  if (cov_mode == 0) {
    T sx2 = kappa * lam1, sy2 = kappa * lam2, sz2 = T(kSz * kSz);
    // Eq. 13: R_local diag(sx^2, sy^2, sz^2) R_local^T, R_local = [x3 y3 n].
    T cols[3][3] = {{x3.x, x3.y, x3.z}, {y3.x, y3.y, y3.z}, {n.x, n.y, n.z}};
    T sc[3] = {sx2, sy2, sz2};
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        T acc = T(0.0);
        for (int k = 0; k < 3; ++k) acc += sc[k] * cols[k][r] * cols[k][q];
        g.cov[3 * r + q] = acc;
      }
  } else {
    // Eq. 15: R_f blkdiag(Sigma2D, 0) R_f^T with R_f = [xa ya n].
    T X[3][2] = {{xa.x, ya.x}, {xa.y, ya.y}, {xa.z, ya.z}};
    T S[2][2] = {{sxx, sxy}, {sxy, syy}};
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        T acc = T(0.0);
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) acc += X[r][a] * S[a][b] * X[q][b];
        g.cov[3 * r + q] = acc;
      }
  }
  // Mean: Eq. 3 evaluated at the Eq. 4 centroid.
  V3<T> m = vi + mux * xa + muy * ya;
  g.mean[0] = m.x; g.mean[1] = m.y; g.mean[2] = m.z;
  g.xj = xj; g.xk = xk; g.yk = yk;
  g.sxx = sxx; g.sxy = sxy; g.syy = syy;
  g.lam1 = lam1; g.lam2 = lam2;
  g.kappa = kappa; g.area = area;
  g.xa = xa; g.ya = ya; g.n = n;
  return g;
}

// Opacity reading: the paper fixes o = 1 (colour assignment, Sec. 2.2); a
// given opacity is taken as a probability and clamped to [0, 1].
template <class T> T clamp01(T o) { return tmin(tmax(o, T(0.0)), T(1.0)); }

// ---------------------------------------------------------------- view-dependent colour
// Spherical-harmonic colour, the extension of the facet colour that the
// colour assignment of Sec. 2.2 names: per facet and channel, K = (L + 1)^2
// coefficients a_k of the real spherical harmonics Y_k of degree <= L
// (L <= 3), evaluated at the unit direction d from the camera centre to the
// facet's centroid (Eq. 3-4); colour = max(0, sum_k a_k Y_k(d) + 1/2) (the
// offset and the clamp at zero are the 3DGS convention; the paper states
// none). Basis: real spherical harmonics without the Condon-Shortley phase,
// ordered (l, m) = (0, 0), (1, -1), (1, 0), (1, 1), (2, -2), ..., (3, 3), each
// a polynomial in the components (x, y, z) of the unit vector d; the
// normalisations follow from the closed forms below.
struct ShConst {
  double c0, c1, c2a, c2b, c2c, c3a, c3b, c3c, c3d, c3e;
  ShConst() {
    c0 = 0.5 * std::sqrt(1.0 / kPi);
    c1 = std::sqrt(3.0 / (4.0 * kPi));
    c2a = 0.5 * std::sqrt(15.0 / kPi);   // xy, yz, xz
    c2b = 0.25 * std::sqrt(5.0 / kPi);   // 3 z^2 - 1
    c2c = 0.25 * std::sqrt(15.0 / kPi);  // x^2 - y^2
    c3a = 0.25 * std::sqrt(35.0 / (2.0 * kPi));  // y (3 x^2 - y^2), x (x^2 - 3 y^2)
    c3b = 0.5 * std::sqrt(105.0 / kPi);          // x y z
    c3c = 0.25 * std::sqrt(21.0 / (2.0 * kPi));  // y (5 z^2 - 1), x (5 z^2 - 1)
    c3d = 0.25 * std::sqrt(7.0 / kPi);           // z (5 z^2 - 3)
    c3e = 0.25 * std::sqrt(105.0 / kPi);         // z (x^2 - y^2)
  }
};
const ShConst kSh;

inline int sh_count(int L) { return (L + 1) * (L + 1); }

template <class T>
void sh_basis(int L, T x, T y, T z, T* Y) {
  Y[0] = T(kSh.c0);
  if (L < 1) return;
  Y[1] = T(kSh.c1) * y;
  Y[2] = T(kSh.c1) * z;
  Y[3] = T(kSh.c1) * x;
  if (L < 2) return;
  Y[4] = T(kSh.c2a) * x * y;
  Y[5] = T(kSh.c2a) * y * z;
  Y[6] = T(kSh.c2b) * (T(3.0) * z * z - T(1.0));
  Y[7] = T(kSh.c2a) * x * z;
  Y[8] = T(kSh.c2c) * (x * x - y * y);
  if (L < 3) return;
  Y[9] = T(kSh.c3a) * y * (T(3.0) * x * x - y * y);
  Y[10] = T(kSh.c3b) * x * y * z;
  Y[11] = T(kSh.c3c) * y * (T(5.0) * z * z - T(1.0));
  Y[12] = T(kSh.c3d) * z * (T(5.0) * z * z - T(3.0));
  Y[13] = T(kSh.c3c) * x * (T(5.0) * z * z - T(1.0));
  Y[14] = T(kSh.c3e) * z * (x * x - y * y);
  Y[15] = T(kSh.c3a) * x * (x * x - T(3.0) * y * y);
}

// Gradient of each polynomial above with respect to (x, y, z) (as written,
// off the sphere too; callers project it onto the sphere's tangent plane).
void sh_basis_grad(int L, double x, double y, double z, double G[16][3]) {
  for (int k = 0; k < 16; ++k) G[k][0] = G[k][1] = G[k][2] = 0.0;
  if (L < 1) return;
  G[1][1] = kSh.c1;
  G[2][2] = kSh.c1;
  G[3][0] = kSh.c1;
  if (L < 2) return;
  G[4][0] = kSh.c2a * y; G[4][1] = kSh.c2a * x;
  G[5][1] = kSh.c2a * z; G[5][2] = kSh.c2a * y;
  G[6][2] = kSh.c2b * 6.0 * z;
  G[7][0] = kSh.c2a * z; G[7][2] = kSh.c2a * x;
  G[8][0] = kSh.c2c * 2.0 * x; G[8][1] = -kSh.c2c * 2.0 * y;
  if (L < 3) return;
  G[9][0] = kSh.c3a * 6.0 * x * y; G[9][1] = kSh.c3a * (3.0 * x * x - 3.0 * y * y);
  G[10][0] = kSh.c3b * y * z; G[10][1] = kSh.c3b * x * z; G[10][2] = kSh.c3b * x * y;
  G[11][1] = kSh.c3c * (5.0 * z * z - 1.0); G[11][2] = kSh.c3c * 10.0 * y * z;
  G[12][2] = kSh.c3d * (15.0 * z * z - 3.0);
  G[13][0] = kSh.c3c * (5.0 * z * z - 1.0); G[13][2] = kSh.c3c * 10.0 * x * z;
  G[14][0] = kSh.c3e * 2.0 * x * z; G[14][1] = -kSh.c3e * 2.0 * y * z; G[14][2] = kSh.c3e * (x * x - y * y);
  G[15][0] = kSh.c3a * (3.0 * x * x - 3.0 * y * y); G[15][1] = -kSh.c3a * 6.0 * x * y;
}

// ---------------------------------------------------------------- projection
// EWA splatting (Sec. 2.1, Zwicker et al.): the perspective map is replaced
// by its Jacobian J at the Gaussian's camera-space mean t.
template <class T> struct Proj {
  T t[3];     // camera-space mean
  T u[2];     // image-plane mean (pixels)
  T J[6];     // 2x3 Jacobian
  T M[6];     // J R
  T S[3];     // Sigma' = M Sigma M^T + 0.3 I : (A, B, C)
  T Q[3];     // conic = Sigma'^-1 : (a, b, c)
};

template <class T>
Proj<T> project(const FaceGauss<T>& g, const Cam& cam) {
  Proj<T> p;
  T R[9];
  for (int k = 0; k < 9; ++k) R[k] = T((double)cam.R[k]);
  for (int r = 0; r < 3; ++r)
    p.t[r] = R[3 * r] * g.mean[0] + R[3 * r + 1] * g.mean[1] + R[3 * r + 2] * g.mean[2] + T((double)cam.t[r]);
  T fx = T((double)cam.fx), fy = T((double)cam.fy);
  T x = p.t[0], y = p.t[1], z = p.t[2];
  p.u[0] = fx * x / z + T((double)cam.cx);
  p.u[1] = fy * y / z + T((double)cam.cy);
  p.J[0] = fx / z; p.J[1] = T(0.0); p.J[2] = -fx * x / (z * z);
  p.J[3] = T(0.0); p.J[4] = fy / z; p.J[5] = -fy * y / (z * z);
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 3; ++q)
      p.M[3 * r + q] = p.J[3 * r] * R[q] + p.J[3 * r + 1] * R[3 + q] + p.J[3 * r + 2] * R[6 + q];
  T MS[6];
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 3; ++q)
      MS[3 * r + q] = p.M[3 * r] * g.cov[q] + p.M[3 * r + 1] * g.cov[3 + q] + p.M[3 * r + 2] * g.cov[6 + q];
  T S00 = MS[0] * p.M[0] + MS[1] * p.M[1] + MS[2] * p.M[2];
  T S01 = MS[0] * p.M[3] + MS[1] * p.M[4] + MS[2] * p.M[5];
  T S11 = MS[3] * p.M[3] + MS[4] * p.M[4] + MS[5] * p.M[5];
  p.S[0] = S00 + T(kDilation);
  p.S[1] = S01;
  p.S[2] = S11 + T(kDilation);
  T det = p.S[0] * p.S[2] - p.S[1] * p.S[1];
  p.Q[0] = p.S[2] / det;
  p.Q[1] = -p.S[1] / det;
  p.Q[2] = p.S[0] / det;
  return p;
}

// ---------------------------------------------------------------- FP32 binning spec
// The binning decisions (which Gaussians are visible, their depth key and the
// rectangle of tiles they are listed in) are integer results of FP32
// arithmetic, so both sides take them with the same IEEE-754 single
// operations in the same order (round to nearest, no contraction). The
// rectangle is conservative: it is the bounding box, widened by 0.25 px, of
// the ellipse of pixel centres at which o * exp(power) could reach 1/255 for
// any o <= 1 (with the area scale kappa = 6 sqrt(3)/pi, the largest it
// takes), so the composited image does not depend on it.
struct Bin {
  bool visible;
  float depth;
  uint32_t depth_bits;
  float ux, uy, rx, ry;
  int x0, x1, y0, y1;  // inclusive tile rectangle; empty when x0 > x1
};

// 2 ln(255) and 6 sqrt(3) / (18 pi), rounded to FP32.
const float kTwoLn255F = 11.0825271606445312f;
const float kKappaOver18F = 0.18377630412578583f;

Bin bin_spec(const float* a, const float* b, const float* c, const Cam& cam, int tile) {
  Bin r;
  volatile float s;  // keeps each step a separate rounded FP32 operation
  float m[3];
  for (int k = 0; k < 3; ++k) {
    s = a[k] + b[k]; s = s + c[k]; s = s / 3.0f; m[k] = s;
  }
  const float* R = cam.R;
  float tc[3];
  for (int q = 0; q < 3; ++q) {
    float p0 = R[3 * q] * m[0];
    float p1 = R[3 * q + 1] * m[1];
    float p2 = R[3 * q + 2] * m[2];
    s = p0 + p1; s = s + p2; s = s + cam.t[q]; tc[q] = s;
  }
  r.depth = tc[2];
  std::memcpy(&r.depth_bits, &r.depth, 4);
  float fxx = cam.fx * tc[0];
  float fyy = cam.fy * tc[1];
  r.ux = fxx / tc[2]; r.ux = r.ux + cam.cx;
  r.uy = fyy / tc[2]; r.uy = r.uy + cam.cy;
  float e1[3], e2[3], q1[3], q2[3];
  for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; }
  for (int q = 0; q < 3; ++q) {
    float p0 = R[3 * q] * e1[0], p1 = R[3 * q + 1] * e1[1], p2 = R[3 * q + 2] * e1[2];
    s = p0 + p1; s = s + p2; q1[q] = s;
    p0 = R[3 * q] * e2[0]; p1 = R[3 * q + 1] * e2[1]; p2 = R[3 * q + 2] * e2[2];
    s = p0 + p1; s = s + p2; q2[q] = s;
  }
  float zz = tc[2] * tc[2];
  float j00 = cam.fx / tc[2];
  float j11 = cam.fy / tc[2];
  float j02 = -(fxx / zz);
  float j12 = -(fyy / zz);
  float p1x, p1y, p2x, p2y;
  { float u = j00 * q1[0], v = j02 * q1[2]; p1x = u + v; }
  { float u = j11 * q1[1], v = j12 * q1[2]; p1y = u + v; }
  { float u = j00 * q2[0], v = j02 * q2[2]; p2x = u + v; }
  { float u = j11 * q2[1], v = j12 * q2[2]; p2y = u + v; }
  float kxx, kyy;
  { float u = p1x * p1x, v = p2x * p2x, w = p1x * p2x; s = u + v; s = s - w; kxx = kKappaOver18F * s; }
  { float u = p1y * p1y, v = p2y * p2y, w = p1y * p2y; s = u + v; s = s - w; kyy = kKappaOver18F * s; }
  // half-widths of the bounding box of {d : d^T Sigma'^-1 d <= 2 ln 255}:
  // sqrt(2 ln 255 Sigma'_xx), sqrt(2 ln 255 Sigma'_yy), plus 0.25 px
  float sxx = kxx + 0.3f, syy = kyy + 0.3f;
  float rx = kTwoLn255F * sxx; rx = std::sqrt(rx); rx = rx + 0.25f;
  float ry = kTwoLn255F * syy; ry = std::sqrt(ry); ry = ry + 0.25f;
  r.rx = rx; r.ry = ry;
  r.visible = (r.depth > cam.znear) && std::isfinite(r.ux) && std::isfinite(r.uy) && std::isfinite(rx) &&
              std::isfinite(ry);
  r.x0 = 1; r.x1 = 0; r.y0 = 1; r.y1 = 0;
  if (!r.visible) return r;
  float inv = 1.0f / (float)tile;  // exact: tile is a power of two
  float bx0 = r.ux - rx; bx0 = bx0 - 0.5f; bx0 = bx0 * inv; bx0 = std::floor(bx0);
  float bx1 = r.ux + rx; bx1 = bx1 - 0.5f; bx1 = bx1 * inv; bx1 = std::floor(bx1);
  float by0 = r.uy - ry; by0 = by0 - 0.5f; by0 = by0 * inv; by0 = std::floor(by0);
  float by1 = r.uy + ry; by1 = by1 - 0.5f; by1 = by1 * inv; by1 = std::floor(by1);
  int tx = (cam.W + tile - 1) / tile, ty = (cam.H + tile - 1) / tile;
  bx0 = std::max(bx0, 0.0f); by0 = std::max(by0, 0.0f);
  bx1 = std::min(bx1, (float)(tx - 1)); by1 = std::min(by1, (float)(ty - 1));
  if (bx0 > bx1 || by0 > by1) return r;
  r.x0 = (int)bx0; r.x1 = (int)bx1; r.y0 = (int)by0; r.y1 = (int)by1;
  return r;
}

// Visible faces of one view in compositing order: ascending FP32 depth key,
// equal keys by ascending face index.
std::vector<int> sorted_visible(const std::vector<Bin>& bins, int F, int view) {
  std::vector<int> order;
  for (int f = 0; f < F; ++f)
    if (bins[(size_t)view * F + f].visible) order.push_back(f);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
    return bins[(size_t)view * F + i].depth_bits < bins[(size_t)view * F + j].depth_bits;
  });
  return order;
}

// ---------------------------------------------------------------- scene
struct Scene {
  int V, F, C;
  const float* verts;   // V x 3 FP32
  const int* faces;     // F x 3
  const float* rgb;     // F x 3 (per face) or V x 3 (per vertex)
  int color_mode;       // 0 per-face, 1 per-vertex averaged (Eq. 16), 2 spherical harmonics
  int sh_degree;        // colour mode 2: L, rgb is F x (L + 1)^2 x 3
  const float* opacity; // F, or null -> scalar
  float opacity_scalar;
  int cov_mode;
  std::vector<Cam> cams;
  double bg[3];
  int tile;
};

bool check_sh(const Scene& s) {
  return s.color_mode != 2 || (s.sh_degree >= 0 && s.sh_degree <= 3);
}

bool check_scene(const Scene& s) {
  if (s.V < 0 || s.F < 0 || s.C < 0) return false;
  for (int f = 0; f < s.F; ++f)
    for (int k = 0; k < 3; ++k)
      if (s.faces[3 * f + k] < 0 || s.faces[3 * f + k] >= s.V) return false;
  return true;
}

std::vector<Bin> all_bins(const Scene& s) {
  std::vector<Bin> bins((size_t)s.C * s.F);
  const long long n = (long long)s.C * s.F;
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (long long r = 0; r < n; ++r) {
    const int c = (int)(r / s.F), f = (int)(r % s.F);
    const int* fi = s.faces + 3 * f;
    bins[(size_t)r] = bin_spec(s.verts + 3 * fi[0], s.verts + 3 * fi[1], s.verts + 3 * fi[2], s.cams[c], s.tile);
  }
  return bins;
}

// Perturbation of the inputs along one direction (forward mode).
struct Direction {
  const double* dverts;  // V x 3 or null
  const double* drgb;    // same shape as rgb or null
  const double* dop;     // F or null
};

template <class T>
T input_vert(const Scene& s, const Direction* dir, int v, int k) {
  T x = T((double)s.verts[3 * v + k]);
  return x;
}
template <>
Dual input_vert<Dual>(const Scene& s, const Direction* dir, int v, int k) {
  return Dual((double)s.verts[3 * v + k], (dir && dir->dverts) ? dir->dverts[3 * v + k] : 0.0);
}

template <class T>
void face_colour(const Scene& s, const Direction* dir, int f, T out[3]) {
  for (int ch = 0; ch < 3; ++ch) {
    if (s.color_mode == 0) {
      T c = T((double)s.rgb[3 * f + ch]);
      out[ch] = c;
    } else {
      // Eq. 16: mean of the three vertex colours.
      T acc = T(0.0);
      for (int k = 0; k < 3; ++k) acc += T((double)s.rgb[3 * s.faces[3 * f + k] + ch]);
      out[ch] = acc / T(3.0);
    }
  }
}
template <>
void face_colour<Dual>(const Scene& s, const Direction* dir, int f, Dual out[3]) {
  for (int ch = 0; ch < 3; ++ch) {
    if (s.color_mode == 0) {
      out[ch] = Dual((double)s.rgb[3 * f + ch], (dir && dir->drgb) ? dir->drgb[3 * f + ch] : 0.0);
    } else {
      Dual acc(0.0);
      for (int k = 0; k < 3; ++k) {
        int v = s.faces[3 * f + k];
        acc += Dual((double)s.rgb[3 * v + ch], (dir && dir->drgb) ? dir->drgb[3 * v + ch] : 0.0);
      }
      out[ch] = acc / Dual(3.0);
    }
  }
}

template <class T>
T face_opacity(const Scene& s, const Direction* dir, int f) {
  double o = s.opacity ? (double)s.opacity[f] : (double)s.opacity_scalar;
  return clamp01(T(o));
}
template <>
Dual face_opacity<Dual>(const Scene& s, const Direction* dir, int f) {
  double o = s.opacity ? (double)s.opacity[f] : (double)s.opacity_scalar;
  double d = (s.opacity && dir && dir->dop) ? dir->dop[f] : 0.0;
  return clamp01(Dual(o, d));
}

// Coefficient k of channel ch of facet f (colour mode 2; rgb is F x K x 3).
template <class T>
T sh_coef(const Scene& s, const Direction* dir, int f, int k, int ch) {
  return T((double)s.rgb[((size_t)f * sh_count(s.sh_degree) + k) * 3 + ch]);
}
template <>
Dual sh_coef<Dual>(const Scene& s, const Direction* dir, int f, int k, int ch) {
  const size_t i = ((size_t)f * sh_count(s.sh_degree) + k) * 3 + ch;
  return Dual((double)s.rgb[i], (dir && dir->drgb) ? dir->drgb[i] : 0.0);
}

// Camera centre in world coordinates: x_cam = R x + t = 0 at x = -R^T t.
V3<double> cam_centre(const Cam& c) {
  double o[3];
  for (int q = 0; q < 3; ++q)
    o[q] = -((double)c.R[q] * c.t[0] + (double)c.R[3 + q] * c.t[1] + (double)c.R[6 + q] * c.t[2]);
  return mk(o[0], o[1], o[2]);
}

// Colour of facet f seen from camera cam (colour mode 2): out = max(0, raw),
// raw = sum_k a_k Y_k(d) + 1/2, d the unit vector from the camera centre to
// the facet's centroid g.mean.
template <class T>
void sh_colour(const Scene& s, const Direction* dir, const FaceGauss<T>& g, const Cam& cam, int f, T out[3],
               T raw[3]) {
  const V3<double> o = cam_centre(cam);
  const V3<T> w = mk<T>(g.mean[0] - T(o.x), g.mean[1] - T(o.y), g.mean[2] - T(o.z));
  const T r = norm(w);
  T Y[16];
  sh_basis<T>(s.sh_degree, w.x / r, w.y / r, w.z / r, Y);
  for (int ch = 0; ch < 3; ++ch) {
    T acc = T(0.5);
    for (int k = 0; k < sh_count(s.sh_degree); ++k) acc += sh_coef<T>(s, dir, f, k, ch) * Y[k];
    raw[ch] = acc;
    out[ch] = tmax(T(0.0), acc);
  }
}

// Ambiguity bands: a pixel is flagged when one of its discrete decisions is
// so close to its threshold that FP32 evaluation may take the other side.
struct Bands { double alpha_rel, t_rel; };

enum {
  FLAG_ALPHA_SKIP = 1,   // o*G within the band of 1/255 (image changes)
  FLAG_TERMINATE = 2,    // T*(1-alpha) within the band of 1e-4 (image changes)
  FLAG_ALPHA_CLAMP = 4,  // o*G within the band of 0.99 (gradient changes)
};

// One contributor of a pixel, recorded for the reverse pass.
struct Contrib {
  int face;
  double alpha, graw, G, Tb, dx, dy;
  bool clamped;
};

template <class T>
struct Prepared {
  std::vector<FaceGauss<T>> g;   // F
  std::vector<Proj<T>> p;        // C*F
  std::vector<T> col;            // F*3, or C*F*3 with view-dependent colour
  std::vector<T> op;             // F
  std::vector<Bin> bins;         // C*F
  std::vector<std::vector<int>> order;  // per view
  // binned mode: per view, per cell of the grid (row-major, cells_x[view]
  // per row), the faces of order[view] whose support meets the cell, in
  // that order
  std::vector<std::vector<std::vector<int>>> cells;
  std::vector<int> cells_x;
  bool per_view_colour = false;
  int F = 0;
  // index of the colour of facet f in view c
  size_t cidx(int view, int f) const { return per_view_colour ? (size_t)view * F + f : (size_t)f; }
};

// The grid of the binned mode. A face can change a pixel's result only
// where o G >= (1 - a) / 255 (a = 1e-3, above any ambiguity band the
// callers ask for, whose flag tests look at faces slightly below 1/255):
// d^T Sigma'^-1 d <= k = 2 ln(255 o / (1 - a)), an ellipse whose bounding box
// has half-widths sqrt(k Sigma'_xx) and sqrt(k Sigma'_yy). Every cell that
// the box (widened by 1e-6 relative and 1e-6 px) meets lists the face (a
// face with a non-finite box: every cell).
constexpr double kCellBand = 1e-3;

template <class T>
void build_cells(const Scene& s, Prepared<T>& P) {
  P.cells.assign(s.C, {});
  P.cells_x.assign(s.C, 0);
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
  for (int c = 0; c < s.C; ++c) {
    const int W = s.cams[c].W, H = s.cams[c].H;
    const int cx = (W + kCell - 1) / kCell, cy = (H + kCell - 1) / kCell;
    P.cells_x[c] = cx;
    std::vector<std::vector<int>>& cl = P.cells[c];
    cl.assign((size_t)cx * cy, {});
    for (int f : P.order[c]) {
      const Proj<T>& pr = P.p[(size_t)c * s.F + f];
      const double o = val(P.op[f]);
      if (!(o > 0.0)) continue;
      const double k = 2.0 * std::log(255.0 * o / (1.0 - kCellBand));
      if (!(k > 0.0)) continue;
      const double hx = std::sqrt(k * val(pr.S[0])) * (1.0 + 1e-6) + 1e-6;
      const double hy = std::sqrt(k * val(pr.S[2])) * (1.0 + 1e-6) + 1e-6;
      const double ux = val(pr.u[0]), uy = val(pr.u[1]);
      if (!std::isfinite(hx) || !std::isfinite(hy) || !std::isfinite(ux) || !std::isfinite(uy)) {
        for (std::vector<int>& list : cl) list.push_back(f);  // no bound: every cell, as the brute force
        continue;
      }
      // pixel p (centre p + 1/2) is inside when p lies in [u - h - 1/2, u + h - 1/2]
      const double x0 = std::max(0.0, std::ceil(ux - hx - 0.5)), x1 = std::min((double)W - 1, std::floor(ux + hx - 0.5));
      const double y0 = std::max(0.0, std::ceil(uy - hy - 0.5)), y1 = std::min((double)H - 1, std::floor(uy + hy - 0.5));
      if (x0 > x1 || y0 > y1) continue;
      for (int by = (int)y0 / kCell; by <= (int)y1 / kCell; ++by)
        for (int bx = (int)x0 / kCell; bx <= (int)x1 / kCell; ++bx) cl[(size_t)by * cx + bx].push_back(f);
    }
  }
}

template <class T>
Prepared<T> prepare(const Scene& s, const Direction* dir) {
  Prepared<T> P;
  P.per_view_colour = s.color_mode == 2;
  P.F = s.F;
  P.g.resize(s.F);
  P.col.resize((P.per_view_colour ? (size_t)s.C : 1) * (size_t)s.F * 3);
  P.op.resize(s.F);
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int f = 0; f < s.F; ++f) {
    const int* fi = s.faces + 3 * f;
    V3<T> v[3];
    for (int k = 0; k < 3; ++k)
      v[k] = mk<T>(input_vert<T>(s, dir, fi[k], 0), input_vert<T>(s, dir, fi[k], 1), input_vert<T>(s, dir, fi[k], 2));
    P.g[f] = convert_face<T>(v[0], v[1], v[2], s.cov_mode);
    if (!P.per_view_colour) face_colour<T>(s, dir, f, &P.col[3 * (size_t)f]);
    P.op[f] = face_opacity<T>(s, dir, f);
  }
  P.bins = all_bins(s);
  P.p.resize((size_t)s.C * s.F);
  P.order.resize(s.C);
  const long long n = (long long)s.C * s.F;
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (long long r = 0; r < n; ++r) {
    const int c = (int)(r / s.F), f = (int)(r % s.F);
    if (P.bins[(size_t)r].visible) P.p[(size_t)r] = project<T>(P.g[f], s.cams[c]);
    if (P.per_view_colour) {
      T raw[3];
      sh_colour<T>(s, dir, P.g[f], s.cams[c], f, &P.col[3 * (size_t)r], raw);
    }
  }
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
  for (int c = 0; c < s.C; ++c) P.order[c] = sorted_visible(P.bins, s.F, c);
  if (g_binned) build_cells(s, P);
  return P;
}

// Front-to-back compositing of one pixel (standard 3DGS rule): for each
// visible Gaussian in order, G = exp(-1/2 d^T Q d) with d the offset from the
// pixel centre, alpha = min(0.99, o G); skip when alpha < 1/255; stop, without
// adding it, when T (1 - alpha) < 1e-4; otherwise C += c alpha T and
// T *= (1 - alpha). I = C + T bg.
template <class T>
void composite_pixel(const Scene& s, const Prepared<T>& P, int view, int px, int py, T out[3],
                     T* Tfinal, int* last_face, int* ncontrib, int* flags, const Bands* bands,
                     std::vector<Contrib>* rec) {
  T Tr = T(1.0);
  T C[3] = {T(0.0), T(0.0), T(0.0)};
  int lastf = -1, nc = 0, fl = 0;
  double pcx = px + 0.5, pcy = py + 0.5;
  const std::vector<int>& list =
      P.cells.empty() ? P.order[view] : P.cells[view][(size_t)(py / kCell) * P.cells_x[view] + px / kCell];
  for (int f : list) {
    const Proj<T>& pr = P.p[(size_t)view * s.F + f];
    T dx = pr.u[0] - T(pcx), dy = pr.u[1] - T(pcy);
    T power = T(-0.5) * (pr.Q[0] * dx * dx + T(2.0) * pr.Q[1] * dx * dy + pr.Q[2] * dy * dy);
    T G = exp(power);
    T graw = P.op[f] * G;
    T alpha = tmin(T(kAlphaMax), graw);
    if (bands) {
      if (std::fabs(val(graw) - kAlphaMin) <= bands->alpha_rel * kAlphaMin) fl |= FLAG_ALPHA_SKIP;
      if (std::fabs(val(graw) - kAlphaMax) <= bands->alpha_rel * kAlphaMax) fl |= FLAG_ALPHA_CLAMP;
    }
    if (val(alpha) < kAlphaMin) continue;
    T test = Tr * (T(1.0) - alpha);
    if (bands && std::fabs(val(test) - kTMin) <= bands->t_rel * kTMin) fl |= FLAG_TERMINATE;
    if (val(test) < kTMin) break;
    if (rec) {
      Contrib cb;
      cb.face = f; cb.alpha = val(alpha); cb.graw = val(graw); cb.G = val(G); cb.Tb = val(Tr);
      cb.dx = val(dx); cb.dy = val(dy); cb.clamped = !(val(graw) < kAlphaMax);
      rec->push_back(cb);
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] += P.col[3 * P.cidx(view, f) + ch] * alpha * Tr;
    Tr = test;
    lastf = f;
    ++nc;
  }
  for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + Tr * T(s.bg[ch]);
  if (Tfinal) *Tfinal = Tr;
  if (last_face) *last_face = lastf;
  if (ncontrib) *ncontrib = nc;
  if (flags) *flags = fl;
}

void build_scene(Scene& s, int V, const float* verts, int F, const int* faces, const float* rgb, int color_mode,
                 const float* opacity, float opacity_scalar, int cov_mode, int C, const float* cam_f,
                 const int* cam_i, const double* bg, int tile, int sh_degree) {
  s.V = V; s.F = F; s.C = C; s.verts = verts; s.faces = faces; s.rgb = rgb; s.color_mode = color_mode;
  s.sh_degree = sh_degree;
  s.opacity = opacity; s.opacity_scalar = opacity_scalar; s.cov_mode = cov_mode;
  s.cams = read_cams(cam_f, cam_i, C);
  for (int k = 0; k < 3; ++k) s.bg[k] = bg ? bg[k] : 0.0;
  s.tile = tile;
}

// ---------------------------------------------------------------- reverse pass
// Hand-derived reverse mode of the chain above, for a scalar loss whose
// gradient with respect to the rendered pixels is given.

struct FaceGrad {
  double du[2], dQ[3];   // per (view, face): image mean and conic (a, b, c)
};

// d/d(inputs of project) given dL/du and dL/dQ (Q parameters a, b, c with
// Q = [[a, b], [b, c]]). Accumulates dL/dmean (world) and dL/dcov (3x3 full).
void project_backward(const FaceGauss<double>& g, const Proj<double>& p, const Cam& cam, const FaceGrad& fg,
                      double dmean[3], double dcov[9]) {
  double R[9];
  for (int k = 0; k < 9; ++k) R[k] = (double)cam.R[k];
  // Q = S^-1 (S symmetric): dL/dS = -Q dL/dQ Q, with the full symmetric
  // matrix gradient of Q whose off-diagonal entries carry half of dL/db.
  double Qm[2][2] = {{p.Q[0], p.Q[1]}, {p.Q[1], p.Q[2]}};
  double GQ[2][2] = {{fg.dQ[0], 0.5 * fg.dQ[1]}, {0.5 * fg.dQ[1], fg.dQ[2]}};
  double tmp[2][2], GS[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) tmp[i][j] = Qm[i][0] * GQ[0][j] + Qm[i][1] * GQ[1][j];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) GS[i][j] = -(tmp[i][0] * Qm[0][j] + tmp[i][1] * Qm[1][j]);
  // S = M Sigma M^T + 0.3 I: dSigma = M^T GS M, dM = 2 GS M Sigma.
  const double* M = p.M;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc += M[3 * a + i] * GS[a][b] * M[3 * b + j];
      dcov[3 * i + j] += acc;
    }
  double MS[6];
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 3; ++q)
      MS[3 * r + q] = M[3 * r] * g.cov[q] + M[3 * r + 1] * g.cov[3 + q] + M[3 * r + 2] * g.cov[6 + q];
  double dM[6];
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 3; ++q) dM[3 * r + q] = 2.0 * (GS[r][0] * MS[q] + GS[r][1] * MS[3 + q]);
  // M = J R: dJ = dM R^T.
  double dJ[6];
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 3; ++k) dJ[3 * r + k] = dM[3 * r] * R[3 * k] + dM[3 * r + 1] * R[3 * k + 1] + dM[3 * r + 2] * R[3 * k + 2];
  double x = p.t[0], y = p.t[1], z = p.t[2];
  double fx = cam.fx, fy = cam.fy;
  double dt[3] = {0.0, 0.0, 0.0};
  // J entries as functions of t.
  dt[2] += dJ[0] * (-fx / (z * z));
  dt[0] += dJ[2] * (-fx / (z * z));
  dt[2] += dJ[2] * (2.0 * fx * x / (z * z * z));
  dt[2] += dJ[4] * (-fy / (z * z));
  dt[1] += dJ[5] * (-fy / (z * z));
  dt[2] += dJ[5] * (2.0 * fy * y / (z * z * z));
  // u = (fx x / z + cx, fy y / z + cy)
  dt[0] += fg.du[0] * fx / z;
  dt[2] += fg.du[0] * (-fx * x / (z * z));
  dt[1] += fg.du[1] * fy / z;
  dt[2] += fg.du[1] * (-fy * y / (z * z));
  // t = R mean + t_cam
  for (int q = 0; q < 3; ++q) dmean[q] += R[q] * dt[0] + R[3 + q] * dt[1] + R[6 + q] * dt[2];
}

// Reverse pass of convert_face. The 3D covariance is differentiated in the
// embedding form R_f blkdiag(kappa Sigma2D, s_z^2) R_f^T, which equals Eq. 13
// by Eq. 14 (R_local = R_f blkdiag(U, 1)), so no eigenvector derivative is
// needed; lambda1 lambda2 in Eq. 12 is det Sigma2D.
void convert_backward(const FaceGauss<double>& g, V3<double> vi, V3<double> vj, V3<double> vk, int cov_mode,
                      const double dmean[3], const double dcov_in[9], double dv[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) dv[a][k] = 0.0;
  if (g.degenerate) {
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) dv[a][k] = dmean[k] / 3.0;
    return;
  }
  double G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[i][j] = 0.5 * (dcov_in[3 * i + j] + dcov_in[3 * j + i]);
  double X[3][2] = {{g.xa.x, g.ya.x}, {g.xa.y, g.ya.y}, {g.xa.z, g.ya.z}};
  double nn[3] = {g.n.x, g.n.y, g.n.z};
  double S2[2][2] = {{g.sxx, g.sxy}, {g.sxy, g.syy}};
  double scale = (cov_mode == 0) ? g.kappa : 1.0;
  // XtGX
  double GX[3][2];
  for (int i = 0; i < 3; ++i)
    for (int b = 0; b < 2; ++b) GX[i][b] = G[i][0] * X[0][b] + G[i][1] * X[1][b] + G[i][2] * X[2][b];
  double XtGX[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) XtGX[a][b] = X[0][a] * GX[0][b] + X[1][a] * GX[1][b] + X[2][a] * GX[2][b];
  // dX = 2 G X (scale S2)
  double dX[3][2];
  for (int i = 0; i < 3; ++i)
    for (int b = 0; b < 2; ++b) dX[i][b] = 2.0 * scale * (GX[i][0] * S2[0][b] + GX[i][1] * S2[1][b]);
  double dS[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) dS[a][b] = scale * XtGX[a][b];
  double dsxx = dS[0][0], dsyy = dS[1][1], dsxy = dS[0][1] + dS[1][0];
  double dn[3] = {0.0, 0.0, 0.0};
  double darea = 0.0;
  if (cov_mode == 0) {
    double sz2 = kSz * kSz;
    for (int i = 0; i < 3; ++i) dn[i] = 2.0 * sz2 * (G[i][0] * nn[0] + G[i][1] * nn[1] + G[i][2] * nn[2]);
    double dkappa = XtGX[0][0] * S2[0][0] + XtGX[0][1] * S2[0][1] + XtGX[1][0] * S2[1][0] + XtGX[1][1] * S2[1][1];
    double det = g.sxx * g.syy - g.sxy * g.sxy;
    if (det > kEps) {
      darea += dkappa / (kPi * std::sqrt(det));
      double ddet = dkappa * (-0.5 * g.kappa / det);
      dsxx += ddet * g.syy;
      dsyy += ddet * g.sxx;
      dsxy += ddet * (-2.0 * g.sxy);
    } else {
      darea += dkappa / (kPi * std::sqrt(kEps));
    }
  }
  double xj = g.xj, xk = g.xk, yk = g.yk;
  double mux = (xj + xk) / 3.0, muy = yk / 3.0;
  // Sigma2D (Eq. 9) with the moments of Eq. 6-8 at v_i=(0,0), v_j=(xj,0):
  // Ex2 = (xj^2 + xj xk + xk^2)/6, Exy = yk (xj + 2 xk)/12, Ey2 = yk^2/6.
  double dxj = 0.0, dxk = 0.0, dyk = 0.0, dmux = 0.0, dmuy = 0.0;
  dxj += dsxx * (2.0 * xj + xk) / 6.0;
  dxk += dsxx * (xj + 2.0 * xk) / 6.0;
  dmux += dsxx * (-2.0 * mux);
  dxj += dsxy * yk / 12.0;
  dxk += dsxy * yk / 6.0;
  dyk += dsxy * (xj + 2.0 * xk) / 12.0;
  dmux += dsxy * (-muy);
  dmuy += dsxy * (-mux);
  dyk += dsyy * yk / 3.0;
  dmuy += dsyy * (-2.0 * muy);
  // area = xj yk / 2
  dxj += darea * 0.5 * yk;
  dyk += darea * 0.5 * xj;
  // mean = vi + mux xa + muy ya
  V3<double> dm = mk(dmean[0], dmean[1], dmean[2]);
  dmux += dot(dm, g.xa);
  dmuy += dot(dm, g.ya);
  V3<double> dxa = mux * dm + mk(dX[0][0], dX[1][0], dX[2][0]);
  V3<double> dya = muy * dm + mk(dX[0][1], dX[1][1], dX[2][1]);
  V3<double> dvi = dm;
  // n = xa x ya
  V3<double> dnv = mk(dn[0], dn[1], dn[2]);
  dxa = dxa + cross(g.ya, dnv);
  dya = dya + cross(dnv, g.xa);
  dxj += dmux / 3.0;
  dxk += dmux / 3.0;
  dyk += dmuy / 3.0;
  // Gram-Schmidt reverse.
  V3<double> e2 = vk - vi;
  V3<double> dw = (1.0 / yk) * (dya - dot(g.ya, dya) * g.ya) + dyk * g.ya;
  V3<double> de2 = dw;
  dxk += -dot(dw, g.xa);
  dxa = dxa - xk * dw;
  de2 = de2 + dxk * g.xa;
  dxa = dxa + dxk * e2;
  V3<double> de1 = (1.0 / xj) * (dxa - dot(g.xa, dxa) * g.xa) + dxj * g.xa;
  V3<double> dvj = de1, dvk = de2;
  dvi = dvi - de1 - de2;
  dv[0][0] = dvi.x; dv[0][1] = dvi.y; dv[0][2] = dvi.z;
  dv[1][0] = dvj.x; dv[1][1] = dvj.y; dv[1][2] = dvj.z;
  dv[2][0] = dvk.x; dv[2][1] = dvk.y; dv[2][2] = dvk.z;
}

}  // namespace

// ============================================================== C interface
extern "C" {

// The real spherical harmonics of degree <= L (colour mode 2) at n unit
// directions dirs (n x 3): out is n x (L + 1)^2. Returns -1 for L outside
// [0, 3].
int gmr_oracle_sh_basis(int L, long long n, const double* dirs, double* out) {
  if (L < 0 || L > 3) return -1;
  const int K = sh_count(L);
  for (long long i = 0; i < n; ++i) {
    double Y[16];
    sh_basis<double>(L, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    for (int k = 0; k < K; ++k) out[i * K + k] = Y[k];
  }
  return 0;
}

// Host threads of the oracle's parallel loops (1 by default; n < 1 means all
// cores OpenMP reports). Results are identical for every thread count.
// Returns the count now in use.
int gmr_oracle_set_threads(int n) {
  g_threads = n >= 1 ? n : omp_get_num_procs();
  return g_threads;
}

// Binned compositing on (1) or off (0, the default) for the calls that
// follow; returns the previous setting. Results are the same either way.
int gmr_oracle_set_binned(int on) {
  const int prev = g_binned ? 1 : 0;
  g_binned = on != 0;
  return prev;
}

// Conversion of every facet (Sec. 2.2). means F x 3, cov F x 9 (row-major),
// aux F x 8 = (sxx, sxy, syy, lam1, lam2, kappa, area, degenerate),
// frame F x 9 = (xa, ya, n). Any output may be null. Returns 0, or -1 on a
// face index out of range.
int gmr_oracle_convert(int V, const double* verts, int F, const int* faces, int cov_mode, double* means,
                       double* cov, double* aux, double* frame) {
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < 3; ++k)
      if (faces[3 * f + k] < 0 || faces[3 * f + k] >= V) return -1;
  for (int f = 0; f < F; ++f) {
    const int* fi = faces + 3 * f;
    V3<double> v[3];
    for (int k = 0; k < 3; ++k) v[k] = mk(verts[3 * fi[k]], verts[3 * fi[k] + 1], verts[3 * fi[k] + 2]);
    FaceGauss<double> g = convert_face<double>(v[0], v[1], v[2], cov_mode);
    if (means) for (int k = 0; k < 3; ++k) means[3 * f + k] = g.mean[k];
    if (cov) for (int k = 0; k < 9; ++k) cov[9 * f + k] = g.cov[k];
    if (aux) {
      double a[8] = {g.sxx, g.sxy, g.syy, g.lam1, g.lam2, g.kappa, g.area, g.degenerate ? 1.0 : 0.0};
      for (int k = 0; k < 8; ++k) aux[8 * f + k] = a[k];
    }
    if (frame) {
      double fr[9] = {g.xa.x, g.xa.y, g.xa.z, g.ya.x, g.ya.y, g.ya.z, g.n.x, g.n.y, g.n.z};
      for (int k = 0; k < 9; ++k) frame[9 * f + k] = fr[k];
    }
  }
  return 0;
}

// EWA projection of given Gaussians (means F x 3, cov F x 9) into C views.
// Output per (view, face), view-major: u (2), Sigma' (3: A, B, C), conic (3),
// camera-space mean (3); each array may be null.
int gmr_oracle_project(int F, const double* means, const double* cov, int C, const float* cam_f, const int* cam_i,
                       double* u, double* sig, double* conic, double* tcam) {
  std::vector<Cam> cams = read_cams(cam_f, cam_i, C);
  for (int c = 0; c < C; ++c)
    for (int f = 0; f < F; ++f) {
      FaceGauss<double> g;
      for (int k = 0; k < 3; ++k) g.mean[k] = means[3 * f + k];
      for (int k = 0; k < 9; ++k) g.cov[k] = cov[9 * f + k];
      Proj<double> p = project<double>(g, cams[c]);
      size_t r = (size_t)c * F + f;
      if (u) { u[2 * r] = p.u[0]; u[2 * r + 1] = p.u[1]; }
      if (sig) for (int k = 0; k < 3; ++k) sig[3 * r + k] = p.S[k];
      if (conic) for (int k = 0; k < 3; ++k) conic[3 * r + k] = p.Q[k];
      if (tcam) for (int k = 0; k < 3; ++k) tcam[3 * r + k] = p.t[k];
    }
  return 0;
}

// FP32 binning specification per (view, face), view-major: visible flag,
// depth key bits, tile rectangle (x0, x1, y0, y1 inclusive; x0 > x1 when
// empty), and the FP32 screen mean and box half-widths it was derived from.
int gmr_oracle_bins(int V, const float* verts, int F, const int* faces, int C, const float* cam_f, const int* cam_i,
                    int tile, uint8_t* visible, uint32_t* depth_bits, int32_t* rect, float* uxyr) {
  if (tile <= 0 || (tile & (tile - 1))) return -2;
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < 3; ++k)
      if (faces[3 * f + k] < 0 || faces[3 * f + k] >= V) return -1;
  std::vector<Cam> cams = read_cams(cam_f, cam_i, C);
  for (int c = 0; c < C; ++c)
    for (int f = 0; f < F; ++f) {
      const int* fi = faces + 3 * f;
      Bin b = bin_spec(verts + 3 * fi[0], verts + 3 * fi[1], verts + 3 * fi[2], cams[c], tile);
      size_t r = (size_t)c * F + f;
      if (visible) visible[r] = b.visible ? 1 : 0;
      if (depth_bits) depth_bits[r] = b.depth_bits;
      if (rect) { rect[4 * r] = b.x0; rect[4 * r + 1] = b.x1; rect[4 * r + 2] = b.y0; rect[4 * r + 3] = b.y1; }
      if (uxyr) { uxyr[4 * r] = b.ux; uxyr[4 * r + 1] = b.uy; uxyr[4 * r + 2] = b.rx; uxyr[4 * r + 3] = b.ry; }
    }
  return 0;
}

// Number of (tile, Gaussian) pairs the binning spec produces.
long long gmr_oracle_count_pairs(int V, const float* verts, int F, const int* faces, int C, const float* cam_f,
                                 const int* cam_i, int tile) {
  std::vector<Cam> cams = read_cams(cam_f, cam_i, C);
  long long n = 0;
  for (int c = 0; c < C; ++c)
    for (int f = 0; f < F; ++f) {
      const int* fi = faces + 3 * f;
      Bin b = bin_spec(verts + 3 * fi[0], verts + 3 * fi[1], verts + 3 * fi[2], cams[c], tile);
      if (b.visible && b.x0 <= b.x1 && b.y0 <= b.y1) n += (long long)(b.x1 - b.x0 + 1) * (b.y1 - b.y0 + 1);
    }
  return n;
}

// Sorted (tile, face) pairs and per-tile ranges. Global tile ids number the
// tiles of view 0 row-major, then view 1, and so on. Pairs are ordered by
// (global tile, depth key, face index). ranges holds [start, end) per global
// tile, (0, 0) for a tile with no pairs. Returns the pair count, or -1 when
// cap is too small.
long long gmr_oracle_sorted_pairs(int V, const float* verts, int F, const int* faces, int C, const float* cam_f,
                                  const int* cam_i, int tile, long long cap, uint32_t* tile_ids, uint32_t* face_ids,
                                  uint32_t* ranges) {
  std::vector<Cam> cams = read_cams(cam_f, cam_i, C);
  struct P { uint32_t tile, depth, face; };
  std::vector<P> pairs;
  long long base = 0;
  std::vector<long long> bases(C);
  for (int c = 0; c < C; ++c) {
    bases[c] = base;
    base += (long long)((cams[c].W + tile - 1) / tile) * ((cams[c].H + tile - 1) / tile);
  }
  long long total_tiles = base;
  for (int c = 0; c < C; ++c) {
    int tx = (cams[c].W + tile - 1) / tile;
    for (int f = 0; f < F; ++f) {
      const int* fi = faces + 3 * f;
      Bin b = bin_spec(verts + 3 * fi[0], verts + 3 * fi[1], verts + 3 * fi[2], cams[c], tile);
      if (!b.visible) continue;
      for (int y = b.y0; y <= b.y1; ++y)
        for (int x = b.x0; x <= b.x1; ++x) {
          P p;
          p.tile = (uint32_t)(bases[c] + (long long)y * tx + x);
          p.depth = b.depth_bits;
          p.face = (uint32_t)f;
          pairs.push_back(p);
        }
    }
  }
  if ((long long)pairs.size() > cap) return -1;
  std::stable_sort(pairs.begin(), pairs.end(), [](const P& a, const P& b) {
    if (a.tile != b.tile) return a.tile < b.tile;
    if (a.depth != b.depth) return a.depth < b.depth;
    return a.face < b.face;
  });
  if (ranges)
    for (long long t = 0; t < 2 * total_tiles; ++t) ranges[t] = 0;
  for (size_t i = 0; i < pairs.size(); ++i) {
    if (tile_ids) tile_ids[i] = pairs[i].tile;
    if (face_ids) face_ids[i] = pairs[i].face;
    if (ranges) {
      uint32_t t = pairs[i].tile;
      if (i == 0 || pairs[i - 1].tile != t) ranges[2 * (size_t)t] = (uint32_t)i;
      if (i + 1 == pairs.size() || pairs[i + 1].tile != t) ranges[2 * (size_t)t + 1] = (uint32_t)(i + 1);
    }
  }
  return (long long)pairs.size();
}

// Brute-force render of a list of pixels (view, x, y). Outputs per pixel:
// rgb (3), final transmittance, last contributing face (-1 if none), number
// of contributors, ambiguity flags (see FLAG_*). bands = (alpha_rel, t_rel).
int gmr_oracle_render(int V, const float* verts, int F, const int* faces, const float* rgb, int color_mode,
                      const float* opacity, float opacity_scalar, int cov_mode, int C, const float* cam_f,
                      const int* cam_i, const double* bg, int tile, long long npix, const int* pix, double* out_rgb,
                      double* out_T, int* out_last, int* out_nc, int* out_flags, const double* bands,
                      int sh_degree) {
  Scene s;
  build_scene(s, V, verts, F, faces, rgb, color_mode, opacity, opacity_scalar, cov_mode, C, cam_f, cam_i, bg, tile,
              sh_degree);
  if (!check_sh(s)) return -4;
  if (!check_scene(s)) return -1;
  Prepared<double> P = prepare<double>(s, nullptr);
  Bands b;
  if (bands) { b.alpha_rel = bands[0]; b.t_rel = bands[1]; }
  for (long long i = 0; i < npix; ++i)
    if (pix[3 * i] < 0 || pix[3 * i] >= C) return -3;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
  for (long long i = 0; i < npix; ++i) {
    int view = pix[3 * i], x = pix[3 * i + 1], y = pix[3 * i + 2];
    double o[3], Tf;
    int lf, nc, fl;
    composite_pixel<double>(s, P, view, x, y, o, &Tf, &lf, &nc, &fl, bands ? &b : nullptr, nullptr);
    if (out_rgb) for (int k = 0; k < 3; ++k) out_rgb[3 * i + k] = o[k];
    if (out_T) out_T[i] = Tf;
    if (out_last) out_last[i] = lf;
    if (out_nc) out_nc[i] = nc;
    if (out_flags) out_flags[i] = fl;
  }
  return 0;
}

// Reverse pass: given dL/dI at the listed pixels (npix x 3; all other pixels
// contribute nothing) and optionally dL/dT_final there (npix; NULL: zero),
// writes dL/dverts (V x 3), dL/drgb (shape of rgb) and
// dL/dopacity (F, when opacity is per face). rec_grads, if not null, receives
// per (view, face) the 9 values (du_x, du_y, dQ_a, dQ_b, dQ_c, do, dr, dg, db).
int gmr_oracle_backward(int V, const float* verts, int F, const int* faces, const float* rgb, int color_mode,
                        const float* opacity, float opacity_scalar, int cov_mode, int C, const float* cam_f,
                        const int* cam_i, const double* bg, int tile, long long npix, const int* pix,
                        const double* dLdI, double* dverts, double* drgb, double* dopac, double* rec_grads,
                        const double* dLdT, int sh_degree) {
  Scene s;
  build_scene(s, V, verts, F, faces, rgb, color_mode, opacity, opacity_scalar, cov_mode, C, cam_f, cam_i, bg, tile,
              sh_degree);
  if (!check_sh(s)) return -4;
  if (!check_scene(s)) return -1;
  Prepared<double> P = prepare<double>(s, nullptr);
  std::vector<FaceGrad> fg((size_t)C * F);
  for (auto& x : fg) { x.du[0] = x.du[1] = 0.0; x.dQ[0] = x.dQ[1] = x.dQ[2] = 0.0; }
  std::vector<double> dcol(P.col.size(), 0.0), dop(F, 0.0);
  for (long long i = 0; i < npix; ++i)
    if (pix[3 * i] < 0 || pix[3 * i] >= C) return -3;
  // One pixel's terms, in the order they are added: the pixels are walked in
  // parallel over fixed chunks (each chunk lists its terms), and the terms
  // are then added in pixel order, so every sum has the same order as with
  // one thread.
  struct Term {
    int f, view;
    bool clamped;
    double dcol[3], dop, dQ[3], du[2];
  };
  const long long kChunk = 32;
  const long long nchunks = (npix + kChunk - 1) / kChunk;
  const long long wave = (long long)std::max(g_threads, 1) * 16;
  std::vector<std::vector<Term>> terms;
  for (long long w0 = 0; w0 < nchunks; w0 += wave) {
    const long long w1 = std::min(nchunks, w0 + wave);
    terms.assign((size_t)(w1 - w0), std::vector<Term>());
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (long long chk = w0; chk < w1; ++chk) {
      std::vector<Contrib> rec;
      std::vector<Term>& out = terms[(size_t)(chk - w0)];
      for (long long i = chk * kChunk; i < std::min(npix, (chk + 1) * kChunk); ++i) {
        int view = pix[3 * i], x = pix[3 * i + 1], y = pix[3 * i + 2];
        const double* g = dLdI + 3 * i;
        const double gT = dLdT ? dLdT[i] : 0.0;
        if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0 && gT == 0.0) continue;
        rec.clear();
        double o[3], Tf;
        composite_pixel<double>(s, P, view, x, y, o, &Tf, nullptr, nullptr, nullptr, nullptr, &rec);
        // I = sum_i c_i alpha_i T_i + T_N bg. Walking back, S is the part of I
        // contributed after Gaussian i: dI/dalpha_i = c_i T_i - S / (1 - alpha_i).
        double S[3] = {Tf * s.bg[0], Tf * s.bg[1], Tf * s.bg[2]};
        for (int k = (int)rec.size() - 1; k >= 0; --k) {
          const Contrib& cb = rec[k];
          int f = cb.face;
          const double* col = &P.col[3 * P.cidx(view, f)];
          Term t;
          t.f = f;
          t.view = view;
          double dalpha = 0.0;
          for (int ch = 0; ch < 3; ++ch) {
            t.dcol[ch] = cb.alpha * cb.Tb * g[ch];
            dalpha += g[ch] * (col[ch] * cb.Tb - S[ch] / (1.0 - cb.alpha));
          }
          // final transmittance T_N = prod_j (1 - alpha_j): dT_N/dalpha_i = -T_N / (1 - alpha_i)
          dalpha += gT * (-Tf / (1.0 - cb.alpha));
          for (int ch = 0; ch < 3; ++ch) S[ch] += col[ch] * cb.alpha * cb.Tb;
          // alpha = 0.99 does not depend on o or the geometry
          t.clamped = cb.clamped;
          if (!cb.clamped) {
            // alpha = o exp(power)
            t.dop = dalpha * cb.G;
            double dpower = dalpha * cb.alpha;
            const Proj<double>& pr = P.p[(size_t)view * F + f];
            // power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), d = u - pixel centre
            t.dQ[0] = dpower * (-0.5 * cb.dx * cb.dx);
            t.dQ[1] = dpower * (-cb.dx * cb.dy);
            t.dQ[2] = dpower * (-0.5 * cb.dy * cb.dy);
            t.du[0] = dpower * (-(pr.Q[0] * cb.dx + pr.Q[1] * cb.dy));
            t.du[1] = dpower * (-(pr.Q[1] * cb.dx + pr.Q[2] * cb.dy));
          }
          out.push_back(t);
        }
      }
    }
    for (const std::vector<Term>& tv : terms)
      for (const Term& t : tv) {
        for (int ch = 0; ch < 3; ++ch) dcol[3 * P.cidx(t.view, t.f) + ch] += t.dcol[ch];
        if (t.clamped) continue;
        dop[t.f] += t.dop;
        FaceGrad& G = fg[(size_t)t.view * F + t.f];
        for (int q = 0; q < 3; ++q) G.dQ[q] += t.dQ[q];
        G.du[0] += t.du[0];
        G.du[1] += t.du[1];
      }
  }
  if (rec_grads) {
    for (int c = 0; c < C; ++c)
      for (int f = 0; f < F; ++f) {
        size_t r = (size_t)c * F + f;
        double* o = rec_grads + 9 * r;
        o[0] = fg[r].du[0]; o[1] = fg[r].du[1];
        o[2] = fg[r].dQ[0]; o[3] = fg[r].dQ[1]; o[4] = fg[r].dQ[2];
        o[5] = 0.0; o[6] = o[7] = o[8] = 0.0;
      }
  }
  // Chain through projection (per view) and conversion (per face).
  // (per face, the views are added in ascending order whatever the threads)
  std::vector<double> dmean((size_t)F * 3, 0.0), dcov((size_t)F * 9, 0.0);
  // colour mode 2: dL/d(coefficients), per face summed over the views
  const int K = color_mode == 2 ? sh_count(sh_degree) : 0;
  std::vector<double> dsh((size_t)F * K * 3, 0.0);
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int f = 0; f < F; ++f)
    for (int c = 0; c < C; ++c) {
      size_t r = (size_t)c * F + f;
      const FaceGrad& G = fg[r];
      if (!(G.du[0] == 0.0 && G.du[1] == 0.0 && G.dQ[0] == 0.0 && G.dQ[1] == 0.0 && G.dQ[2] == 0.0))
        project_backward(P.g[f], P.p[r], s.cams[c], G, &dmean[3 * (size_t)f], &dcov[9 * (size_t)f]);
      if (color_mode != 2) continue;
      // colour = max(0, sum_k a_k Y_k(d) + 1/2), d = w / |w|, w = mean - o
      const double* gc = &dcol[3 * r];
      if (gc[0] == 0.0 && gc[1] == 0.0 && gc[2] == 0.0) continue;
      double col[3], raw[3];
      sh_colour<double>(s, nullptr, P.g[f], s.cams[c], f, col, raw);
      const V3<double> o = cam_centre(s.cams[c]);
      const V3<double> w = mk(P.g[f].mean[0] - o.x, P.g[f].mean[1] - o.y, P.g[f].mean[2] - o.z);
      const double rn = norm(w);
      const V3<double> d = (1.0 / rn) * w;
      double Y[16], GY[16][3];
      sh_basis<double>(sh_degree, d.x, d.y, d.z, Y);
      sh_basis_grad(sh_degree, d.x, d.y, d.z, GY);
      V3<double> dd = mk(0.0, 0.0, 0.0);
      for (int ch = 0; ch < 3; ++ch) {
        if (!(raw[ch] > 0.0)) continue;  // clamped at zero: no gradient
        for (int k = 0; k < K; ++k) {
          dsh[((size_t)f * K + k) * 3 + ch] += gc[ch] * Y[k];
          const double a = (double)rgb[((size_t)f * K + k) * 3 + ch];
          dd = dd + (gc[ch] * a) * mk(GY[k][0], GY[k][1], GY[k][2]);
        }
      }
      // d = w / |w|: dL/dw = (dL/dd - d (d . dL/dd)) / |w|, and w = mean - o
      const V3<double> dw = (1.0 / rn) * (dd - dot(d, dd) * d);
      dmean[3 * (size_t)f] += dw.x;
      dmean[3 * (size_t)f + 1] += dw.y;
      dmean[3 * (size_t)f + 2] += dw.z;
    }
  if (dverts)
    for (long long k = 0; k < 3LL * V; ++k) dverts[k] = 0.0;
  std::vector<double> dvf((size_t)F * 9);
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int f = 0; f < F; ++f) {
    const int* fi = faces + 3 * f;
    V3<double> v[3];
    for (int k = 0; k < 3; ++k)
      v[k] = mk((double)verts[3 * fi[k]], (double)verts[3 * fi[k] + 1], (double)verts[3 * fi[k] + 2]);
    double dv[3][3];
    // A face that reached no pixel (culled in every view, e.g. with a
    // non-finite vertex) has exactly zero gradient; the chain is skipped so
    // that 0 times its non-finite geometry does not give NaN.
    bool reached = false;
    for (int k = 0; k < 3; ++k) reached |= dmean[3 * (size_t)f + k] != 0.0;
    for (int k = 0; k < 9; ++k) reached |= dcov[9 * (size_t)f + k] != 0.0;
    if (reached) {
      convert_backward(P.g[f], v[0], v[1], v[2], cov_mode, &dmean[3 * (size_t)f], &dcov[9 * (size_t)f], dv);
    } else {
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) dv[a][k] = 0.0;
    }
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) dvf[9 * (size_t)f + 3 * a + k] = dv[a][k];
  }
  if (dverts)  // the vertex sums in face order
    for (int f = 0; f < F; ++f) {
      const int* fi = faces + 3 * f;
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) dverts[3 * (size_t)fi[a] + k] += dvf[9 * (size_t)f + 3 * a + k];
    }
  if (drgb) {
    if (color_mode == 0) {
      for (long long k = 0; k < 3LL * F; ++k) drgb[k] = dcol[k];
    } else if (color_mode == 2) {
      for (size_t k = 0; k < dsh.size(); ++k) drgb[k] = dsh[k];
    } else {
      for (long long k = 0; k < 3LL * V; ++k) drgb[k] = 0.0;
      for (int f = 0; f < F; ++f)
        for (int a = 0; a < 3; ++a)
          for (int ch = 0; ch < 3; ++ch) drgb[3 * (size_t)faces[3 * f + a] + ch] += dcol[3 * (size_t)f + ch] / 3.0;
    }
  }
  if (dopac && opacity) {
    for (int f = 0; f < F; ++f) {
      double o = opacity[f];
      dopac[f] = (o >= 0.0 && o <= 1.0) ? dop[f] : 0.0;  // clamp to [0, 1]
    }
  }
  if (rec_grads) {
    // per-face opacity gradients (and colour gradients, unless the colour is
    // view-dependent: then per record) are reported in view 0's slot
    for (int f = 0; f < F && C > 0; ++f) {
      double* o = rec_grads + 9 * (size_t)f;
      o[5] = dop[f];
    }
    for (size_t i = 0; i < dcol.size() / 3; ++i) {
      double* o = rec_grads + 9 * i;
      o[6] = dcol[3 * i]; o[7] = dcol[3 * i + 1]; o[8] = dcol[3 * i + 2];
    }
  }
  return 0;
}

// Forward-mode directional derivative d/de sum_pixels (<w, I(x + e dir)> +
// wT T_final(x + e dir)) at e = 0 (wT may be NULL), evaluated with dual
// numbers through the same forward code (eigen route of Eq. 10-13 included).
// Returns it in *out.
int gmr_oracle_jvp(int V, const float* verts, int F, const int* faces, const float* rgb, int color_mode,
                   const float* opacity, float opacity_scalar, int cov_mode, int C, const float* cam_f,
                   const int* cam_i, const double* bg, int tile, long long npix, const int* pix, const double* w,
                   const double* dverts, const double* drgb, const double* dop, double* out, const double* wT,
                   int sh_degree) {
  Scene s;
  build_scene(s, V, verts, F, faces, rgb, color_mode, opacity, opacity_scalar, cov_mode, C, cam_f, cam_i, bg, tile,
              sh_degree);
  if (!check_sh(s)) return -4;
  if (!check_scene(s)) return -1;
  Direction dir;
  dir.dverts = dverts; dir.drgb = drgb; dir.dop = dop;
  Prepared<Dual> P = prepare<Dual>(s, &dir);
  double acc = 0.0;
  for (long long i = 0; i < npix; ++i) {
    int view = pix[3 * i], x = pix[3 * i + 1], y = pix[3 * i + 2];
    if (view < 0 || view >= C) return -3;
    Dual o[3], Tf;
    composite_pixel<Dual>(s, P, view, x, y, o, &Tf, nullptr, nullptr, nullptr, nullptr, nullptr);
    for (int k = 0; k < 3; ++k) acc += w[3 * i + k] * o[k].d;
    if (wT) acc += wT[i] * Tf.d;
  }
  *out = acc;
  return 0;
}

}  // extern "C"
