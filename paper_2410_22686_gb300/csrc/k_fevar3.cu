// Trilinear elements with a nodal coefficient (Section 1: M and K of a finite-element
// discretisation), 3D.  K(a) = sum_e a_e K_e with a_e the mean of element e's eight
// corner values and K_e the element stiffness of a = 1; M the consistent mass matrix.
// For two corners of one element that differ in t coordinates,
//   K_e = h/12 (4, 0, -1, -1)   and   M_e = h^3/216 (8, 4, 2, 1)   for t = 0, 1, 2, 3,
// so on the uniform grid both are 27-point stencils: at interior node P and offset o,
//   M_Po = h^3/216 4^(3-t(o)),
//   K_Po = h/12 k(t(o)) sum of a_e over the elements holding both P and P+o,
// k = (4, 0, -1, -1): the six face neighbours (t = 1) are not coupled by K, the twelve
// edge-diagonal neighbours share two elements, the eight corner-diagonal ones one.
// Elements are numbered by their lower corner on the grid with boundary ((m+1)^3 per
// level, x1 fastest); interior node i sits at grid node i + 1, so the element with
// lower corner (i + 1 - c), c in {0, 1}^3, holds it at its corner c.
// This file: the element coefficients of a level, the products (single fields and the
// all-at-once product), the multicolour V(1,0) multigrid kernels for
// (sigma M + tau K(a)) (eight colours: the 27-point stencils never couple two points of
// one colour), the stiffness derivative of the gradient and the element objective.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace pcopt {

namespace {

// the eight element values around interior node (i1, i2, i3): A[c] for the element
// holding the node at its corner c = c1 + 2 c2 + 4 c3
template <typename T>
struct Around {
  T a[8];
};

template <typename T>
__device__ __forceinline__ Around<T> around(const T* __restrict__ E, int m, int i1, int i2, int i3) {
  const int me = m + 1;
  Around<T> A;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int k1 = i1 + 1 - (c & 1), k2 = i2 + 1 - ((c >> 1) & 1), k3 = i3 + 1 - (c >> 2);
    A.a[c] = E[((int64_t)k3 * me + k2) * me + k1];
  }
  return A;
}

// k(t) times the sum of a_e over the elements holding the node and its neighbour at
// offset (o1, o2, o3) (constant offsets once the callers' loops are unrolled): the
// corner c of such an element has c_k = 0 where o_k = +1, 1 where o_k = -1, either where 0
template <typename T>
__device__ __forceinline__ T k_entry(const Around<T>& A, int o1, int o2, int o3) {
  const int t = (o1 != 0) + (o2 != 0) + (o3 != 0);
  if (t == 1) return T(0);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int c1 = c & 1, c2 = (c >> 1) & 1, c3 = c >> 2;
    const bool in1 = o1 == 0 || c1 == (o1 < 0 ? 1 : 0);
    const bool in2 = o2 == 0 || c2 == (o2 < 0 ? 1 : 0);
    const bool in3 = o3 == 0 || c3 == (o3 < 0 ? 1 : 0);
    if (in1 && in2 && in3) s += A.a[c];
  }
  return t == 0 ? T(4) * s : -s;
}

// integer mass weight 4^(3 - t) of offset o
__device__ __forceinline__ constexpr int m_weight(int o1, int o2, int o3) {
  return (o1 == 0 ? 4 : 1) * (o2 == 0 ? 4 : 1) * (o3 == 0 ? 4 : 1);
}

// (M u)_P * 216 / h^3 and (K u)_P * 12 / h for a real field with zero boundary values
template <typename T, typename Tin>
__device__ __forceinline__ void mk_apply3(const Tin* __restrict__ u, const Around<T>& A, int m, int i1, int i2,
                                          int i3, T& mu, T& ku) {
  const int64_t s = ((int64_t)i3 * m + i2) * m + i1;
  mu = T(0);
  ku = T(0);
#pragma unroll
  for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
    for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
      for (int o1 = -1; o1 <= 1; ++o1) {
        const int q1 = i1 + o1, q2 = i2 + o2, q3 = i3 + o3;
        if (q1 < 0 || q1 >= m || q2 < 0 || q2 >= m || q3 < 0 || q3 >= m) continue;
        // FP32 inputs widen on the integer pipes (cvt): GB300 runs F2F on its FP64 unit
        const T v = cvt<T>(u[s + ((int64_t)o3 * m + o2) * m + o1]);
        mu = fma(T(m_weight(o1, o2, o3)), v, mu);
        if ((o1 != 0) + (o2 != 0) + (o3 != 0) != 1) ku = fma(k_entry(A, o1, o2, o3), v, ku);
      }
}

__device__ __forceinline__ void coords3(int64_t s, int m, int& i1, int& i2, int& i3) {
  const int64_t r = s / m;
  i1 = (int)(s - r * m);
  i3 = (int)(r / m);
  i2 = (int)(r - (int64_t)i3 * m);
}

// out_p = cM M in_p + cK K in_p + beta out_p, FP64, `planes` fields of m^3 values
__global__ void __launch_bounds__(256) fevar3_apply_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                           const double* __restrict__ E, int m, double mh, double kh,
                                                           int planes, double cM, double cK, double beta) {
  const int64_t np = (int64_t)m * m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (s >= np || p >= planes) return;
  int i1, i2, i3;
  coords3(s, m, i1, i2, i3);
  const Around<double> A = around(E, m, i1, i2, i3);
  double mu, ku;
  mk_apply3(in + p * np, A, m, i1, i2, i3, mu, ku);
  double v = cM * mh * mu + cK * kh * ku;
  if (beta != 0.0) v = fma(beta, out[p * np + s], v);
  out[p * np + s] = v;
}

// All-at-once product A x (or A^T x), A = [[alpha I(x)M, T^T], [-T, alpha I(x)M]],
// (T v)_j = M v_j - M v_{j-1} + tau K v_j, in FP64 arithmetic for FP64 inputs (FP32
// inputs take the double-float kernel below).  One thread per spatial point and chunk
// of time blocks [j0, j1):
//   y1_j = alpha M x1_j + sg (M x2_j - M x2_{j+1} + tau K x2_j)
//   y2_j = alpha M x2_j - sg (M x1_j - M x1_{j-1} + tau K x1_j),   sg = -1 for A^T.
template <typename Tin, bool TRANSPOSE>
__global__ void __launch_bounds__(256) fevar3_matvec_kernel(const Tin* __restrict__ x, double* __restrict__ y,
                                                            const double* __restrict__ E, int m, int n, int tj,
                                                            double mh, double kh, double alpha, double tau,
                                                            size_t xstride, size_t ystride,
                                                            const int* __restrict__ jdev) {
  const int64_t np = (int64_t)m * m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  if (jdev) {  // device-resident Arnoldi index: x = Z_j, y = V_{j+1}
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int j0 = blockIdx.y * tj, j1 = min(n, j0 + tj);
  if (j0 >= n) return;
  int i1, i2, i3;
  coords3(s, m, i1, i2, i3);
  const Around<double> A = around(E, m, i1, i2, i3);
  const double sg = TRANSPOSE ? -1.0 : 1.0, tk = tau * kh;
  const Tin* x1 = x;
  const Tin* x2 = x + (int64_t)n * np;
  double* y1 = y;
  double* y2 = y + (int64_t)n * np;
  double Mx1p = 0.0;  // M x1_{j-1}
  if (j0 > 0) {
    double mu, ku;
    mk_apply3(x1 + (int64_t)(j0 - 1) * np, A, m, i1, i2, i3, mu, ku);
    Mx1p = mh * mu;
  }
  double pMx1 = 0.0, pMx2 = 0.0, pKx2 = 0.0;  // block j - 1 of this chunk
  for (int j = j0; j < j1; ++j) {
    double mu1, ku1, mu2, ku2;
    mk_apply3(x1 + (int64_t)j * np, A, m, i1, i2, i3, mu1, ku1);
    mk_apply3(x2 + (int64_t)j * np, A, m, i1, i2, i3, mu2, ku2);
    const double Mx1 = mh * mu1, Mx2 = mh * mu2;
    y2[(int64_t)j * np + s] = alpha * Mx2 - sg * (Mx1 - Mx1p + tk * ku1);
    if (j > j0) y1[(int64_t)(j - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2 + tk * pKx2);
    Mx1p = Mx1;
    pMx1 = Mx1;
    pMx2 = Mx2;
    pKx2 = ku2;
  }
  double Mx2n = 0.0;  // M x2_{j1}
  if (j1 < n) {
    double mu, ku;
    mk_apply3(x2 + (int64_t)j1 * np, A, m, i1, i2, i3, mu, ku);
    Mx2n = mh * mu;
  }
  y1[(int64_t)(j1 - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2n + tk * pKx2);
}

// ---------------------------------------------------------------------------
// Element product of an FP32 vector (the inner product of flexible GMRES) in
// double-float arithmetic, as the 2D kernel: the 21 K entries of a point that can be
// nonzero are split once into FP32 (hi, lo) pairs and kept for all its time blocks;
// per time block and half, M u (power-of-two weights on FP32 values, every term
// exact) and K u (exact products hi * u by FMA, lo * u rounded) are summed with
// Knuth's TwoSum into (sum, error) pairs, widened on the integer pipes and combined
// in FP64.  Relative error of a sum: about 2^-44 of the sum of the magnitudes of its
// terms, against ~100 FP64 operations per point and time block otherwise.
// ---------------------------------------------------------------------------
struct DF3 {
  float hi, lo;
};

// (hi, lo) += x exactly (TwoSum; no contraction into FMA)
__device__ __forceinline__ void df3_add(DF3& a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

// (hi, lo) += (kh + kl) u
__device__ __forceinline__ void df3_add_prod(DF3& a, float kh, float kl, float u) {
  const float p = __fmul_rn(kh, u);
  const float e = fmaf(kh, u, -p);
  df3_add(a, p);
  a.lo = __fadd_rn(a.lo, fmaf(kl, u, e));
}

__device__ __forceinline__ double df3_val(const DF3& a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }

// the K entries of the 21 offsets not in a single coordinate, in loop order
struct KSplit3 {
  float h[21], l[21];
};

__device__ __forceinline__ void mk_apply3_df(const float* __restrict__ u, const KSplit3& k, int m, int i1, int i2,
                                             int i3, double& mu, double& ku) {
  const int64_t s = ((int64_t)i3 * m + i2) * m + i1;
  DF3 am{0.0f, 0.0f}, ak{0.0f, 0.0f};
  int q = 0;
#pragma unroll
  for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
    for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
      for (int o1 = -1; o1 <= 1; ++o1) {
        const int q1 = i1 + o1, q2 = i2 + o2, q3 = i3 + o3;
        const bool in = q1 >= 0 && q1 < m && q2 >= 0 && q2 < m && q3 >= 0 && q3 < m;
        const float v = in ? u[s + ((int64_t)o3 * m + o2) * m + o1] : 0.0f;
        df3_add(am, __fmul_rn((float)m_weight(o1, o2, o3), v));  // a power of two: exact
        if ((o1 != 0) + (o2 != 0) + (o3 != 0) != 1) {
          df3_add_prod(ak, k.h[q], k.l[q], v);
          ++q;
        }
      }
  mu = df3_val(am);
  ku = df3_val(ak);
}

template <bool TRANSPOSE>
__global__ void __launch_bounds__(256, 2) fevar3_matvec_df_kernel(const float* __restrict__ x, double* __restrict__ y,
                                                               const double* __restrict__ E, int m, int n, int tj,
                                                               double mh, double kh, double alpha, double tau,
                                                               size_t xstride, size_t ystride,
                                                               const int* __restrict__ jdev) {
  const int64_t np = (int64_t)m * m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  if (jdev) {  // device-resident Arnoldi index: x = Z_j, y = V_{j+1}
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int j0 = blockIdx.y * tj, j1 = min(n, j0 + tj);
  if (j0 >= n) return;
  int i1, i2, i3;
  coords3(s, m, i1, i2, i3);
  KSplit3 k;
  {
    const Around<double> A = around(E, m, i1, i2, i3);
    int q = 0;
#pragma unroll
    for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
      for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
        for (int o1 = -1; o1 <= 1; ++o1) {
          if ((o1 != 0) + (o2 != 0) + (o3 != 0) == 1) continue;
          const double kv = k_entry(A, o1, o2, o3);
          k.h[q] = f64_to_f32(kv);
          k.l[q] = f64_to_f32(kv - f32_to_f64(k.h[q]));
          ++q;
        }
  }
  const double sg = TRANSPOSE ? -1.0 : 1.0, tk = tau * kh;
  const float* x1 = x;
  const float* x2 = x + (int64_t)n * np;
  double* y1 = y;
  double* y2 = y + (int64_t)n * np;
  double Mx1p = 0.0;
  if (j0 > 0) {
    double mu, ku;
    mk_apply3_df(x1 + (int64_t)(j0 - 1) * np, k, m, i1, i2, i3, mu, ku);
    Mx1p = mh * mu;
  }
  double pMx1 = 0.0, pMx2 = 0.0, pKx2 = 0.0;
  for (int j = j0; j < j1; ++j) {
    double mu1, ku1, mu2, ku2;
    mk_apply3_df(x1 + (int64_t)j * np, k, m, i1, i2, i3, mu1, ku1);
    mk_apply3_df(x2 + (int64_t)j * np, k, m, i1, i2, i3, mu2, ku2);
    const double Mx1 = mh * mu1, Mx2 = mh * mu2;
    y2[(int64_t)j * np + s] = alpha * Mx2 - sg * (Mx1 - Mx1p + tk * ku1);
    if (j > j0) y1[(int64_t)(j - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2 + tk * pKx2);
    Mx1p = Mx1;
    pMx1 = Mx1;
    pMx2 = Mx2;
    pKx2 = ku2;
  }
  double Mx2n = 0.0;
  if (j1 < n) {
    double mu, ku;
    mk_apply3_df(x2 + (int64_t)j1 * np, k, m, i1, i2, i3, mu, ku);
    Mx2n = mh * mu;
  }
  y1[(int64_t)(j1 - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2n + tk * pKx2);
}

// ---------------------------------------------------------------------------
// Multigrid for (sigma M + tau K(a)): one Gauss-Seidel sweep from zero in colour
// order (colour c = (i1 & 1) + 2 (i2 & 1) + 4 (i3 & 1)), residual, restriction by
// P^T, recursion, trilinear correction (launch_mg_prolong); the one-point level is
// solved by the sweep itself.
// ---------------------------------------------------------------------------

// sums over the neighbours q of P selected by `take` of M_Pq u_q * 216 / h^3 and
// K_Pq u_q * 12 / h, complex
template <typename Tc, typename Take>
__device__ __forceinline__ void mk_offdiag3(const typename Cx<Tc>::t* __restrict__ u, const Around<Tc>& A, int m,
                                            int i1, int i2, int i3, Take take, typename Cx<Tc>::t& mu,
                                            typename Cx<Tc>::t& ku) {
  typedef typename Cx<Tc>::t C;
  mu = czero<Tc>();
  ku = czero<Tc>();
  const int64_t s = ((int64_t)i3 * m + i2) * m + i1;
#pragma unroll
  for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
    for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
      for (int o1 = -1; o1 <= 1; ++o1) {
        if (o1 == 0 && o2 == 0 && o3 == 0) continue;
        const int q1 = i1 + o1, q2 = i2 + o2, q3 = i3 + o3;
        if (q1 < 0 || q1 >= m || q2 < 0 || q2 >= m || q3 < 0 || q3 >= m || !take(o1, o2, o3)) continue;
        const C v = u[s + ((int64_t)o3 * m + o2) * m + o1];
        const Tc wm = Tc(m_weight(o1, o2, o3));
        mu.x = fma(wm, v.x, mu.x);
        mu.y = fma(wm, v.y, mu.y);
        if ((o1 != 0) + (o2 != 0) + (o3 != 0) != 1) {
          const Tc wk = k_entry(A, o1, o2, o3);
          ku.x = fma(wk, v.x, ku.x);
          ku.y = fma(wk, v.y, ku.y);
        }
      }
}

// sigma mh mu + tk ku (mh = h^3/216, tk = tau h / 12)
template <typename Tc>
__device__ __forceinline__ typename Cx<Tc>::t shifted3(typename Cx<Tc>::t sig, typename Cx<Tc>::t mu, Tc mh,
                                                       typename Cx<Tc>::t ku, Tc tk) {
  typename Cx<Tc>::t r;
  r.x = mh * (sig.x * mu.x - sig.y * mu.y) + tk * ku.x;
  r.y = mh * (sig.x * mu.y + sig.y * mu.x) + tk * ku.y;
  return r;
}

// points of colour c: i_k = bit k of c + 2 t_k
template <typename Tc>
__global__ void __launch_bounds__(256) fevar3_smooth_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                            typename Cx<Tc>::t* __restrict__ u,
                                                            const Tc* __restrict__ E,
                                                            const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                            Tc mh, Tc tk, int colour, int planes) {
  typedef typename Cx<Tc>::t C;
  const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
  const int nx = (m - px + 1) / 2, ny = (m - py + 1) / 2, nz = (m - pz + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (t >= (int64_t)nx * ny * nz || p >= planes) return;
  const int tx = (int)(t % nx);
  const int64_t tr = t / nx;
  const int ty = (int)(tr % ny), tz = (int)(tr / ny);
  const int i1 = px + 2 * tx, i2 = py + 2 * ty, i3 = pz + 2 * tz;
  const int64_t np = (int64_t)m * m * m;
  const C* rp = r + p * np;
  C* up = u + p * np;
  const Around<Tc> A = around(E, m, i1, i2, i3);
  // a neighbour counts once its colour has been swept (the others are still zero)
  auto take = [&](int o1, int o2, int o3) {
    return ((px ^ (o1 & 1)) + 2 * (py ^ (o2 & 1)) + 4 * (pz ^ (o3 & 1))) < colour;
  };
  C mu, ku;
  mk_offdiag3<Tc>(up, A, m, i1, i2, i3, take, mu, ku);
  const C sig = sigma[p];
  const C off = shifted3<Tc>(sig, mu, mh, ku, tk);
  const int64_t s = ((int64_t)i3 * m + i2) * m + i1;
  C acc = rp[s];
  acc.x -= off.x;
  acc.y -= off.y;
  C dg;
  dg.x = sig.x * (Tc(64) * mh) + tk * k_entry(A, 0, 0, 0);
  dg.y = sig.y * (Tc(64) * mh);
  up[s] = cmul(acc, cinv(dg));
}

// res = r - (sigma M + tau K) u at every point
template <typename Tc>
__global__ void __launch_bounds__(256) fevar3_residual_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                              const typename Cx<Tc>::t* __restrict__ u,
                                                              typename Cx<Tc>::t* __restrict__ res,
                                                              const Tc* __restrict__ E,
                                                              const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                              Tc mh, Tc tk, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t np = (int64_t)m * m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (s >= np || p >= planes) return;
  int i1, i2, i3;
  coords3(s, m, i1, i2, i3);
  const C* up = u + p * np;
  const Around<Tc> A = around(E, m, i1, i2, i3);
  C mu, ku;
  mk_offdiag3<Tc>(up, A, m, i1, i2, i3, [](int, int, int) { return true; }, mu, ku);
  const C uc = up[s];
  const Tc kc = k_entry(A, 0, 0, 0);
  mu.x = fma(Tc(64), uc.x, mu.x);
  mu.y = fma(Tc(64), uc.y, mu.y);
  ku.x = fma(kc, uc.x, ku.x);
  ku.y = fma(kc, uc.y, ku.y);
  const C au = shifted3<Tc>(sigma[p], mu, mh, ku, tk);
  res[p * np + s] = r[p * np + s] - au;
}

// rc(I, J, K) = sum_{o in -1..1} w(o1) w(o2) w(o3) res(2I+1+o1, 2J+1+o2, 2K+1+o3),
// w(0) = 1, w(+-1) = 1/2: the transpose of trilinear interpolation
template <typename Tc>
__global__ void __launch_bounds__(256) fevar3_restrict_kernel(const typename Cx<Tc>::t* __restrict__ res,
                                                              typename Cx<Tc>::t* __restrict__ rc, int m,
                                                              int planes) {
  typedef typename Cx<Tc>::t C;
  const int mc = (m - 1) / 2;
  const int64_t npc = (int64_t)mc * mc * mc;
  const int64_t sc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (sc >= npc || p >= planes) return;
  int I, J, K;
  coords3(sc, mc, I, J, K);
  const C* rp = res + (int64_t)p * m * m * m;
  C acc = czero<Tc>();
#pragma unroll
  for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
    for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
      for (int o1 = -1; o1 <= 1; ++o1) {
        const Tc wt = (o1 == 0 ? Tc(1) : Tc(0.5)) * (o2 == 0 ? Tc(1) : Tc(0.5)) * (o3 == 0 ? Tc(1) : Tc(0.5));
        const C v = rp[((int64_t)(2 * K + 1 + o3) * m + 2 * J + 1 + o2) * m + 2 * I + 1 + o1];
        acc.x = fma(wt, v.x, acc.x);
        acc.y = fma(wt, v.y, acc.y);
      }
  rc[(int64_t)p * npc + sc] = acc;
}

// ---------------------------------------------------------------------------
// Gradient and objective with element matrices
// ---------------------------------------------------------------------------

// value of field u (m^3 per time block) at grid node (g1, g2, g3) of the grid with boundary
__device__ __forceinline__ double node_val3(const double* __restrict__ u, int m, int g1, int g2, int g3) {
  return (g1 >= 1 && g1 <= m && g2 >= 1 && g2 <= m && g3 >= 1 && g3 <= m)
             ? u[((int64_t)(g3 - 1) * m + (g2 - 1)) * m + (g1 - 1)]
             : 0.0;
}

// u_e^T K_e v_e * 12 / h for the element with lower grid node (k1, k2, k3):
// 4 u_p v_p, -1 for corners differing in two or three coordinates, 0 in one
__device__ __forceinline__ double elem_form3(const double* __restrict__ u, const double* __restrict__ v, int m,
                                             int k1, int k2, int k3) {
  double uc[8], vc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uc[c] = node_val3(u, m, k1 + (c & 1), k2 + ((c >> 1) & 1), k3 + (c >> 2));
    vc[c] = node_val3(v, m, k1 + (c & 1), k2 + ((c >> 1) & 1), k3 + (c >> 2));
  }
  double acc = 0.0;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    // the corners differing from p in two coordinates and the opposite one
    const double far = vc[p ^ 3] + vc[p ^ 5] + vc[p ^ 6] + vc[p ^ 7];
    acc = fma(uc[p], fma(4.0, vc[p], -far), acc);
  }
  return acc;
}

// part[c][e] = sum_{j in chunk c} (lam1_j^T K_e x2_j - lam2_j^T K_e x1_j) * 12 / h
__global__ void __launch_bounds__(256) fevar3_grad_elem_kernel(const double* __restrict__ x,
                                                               const double* __restrict__ lam, int m, int n, int tj,
                                                               double* __restrict__ part) {
  const int me = m + 1;
  const int64_t nel = (int64_t)me * me * me;
  const int64_t el = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= nel) return;
  int k1, k2, k3;
  coords3(el, me, k1, k2, k3);
  const int64_t np = (int64_t)m * m * m;
  const int j0 = blockIdx.y * tj, j1 = min(n, j0 + tj);
  double acc = 0.0;
  for (int j = j0; j < j1; ++j) {
    const double* x1 = x + (int64_t)j * np;
    const double* x2 = x + ((int64_t)n + j) * np;
    const double* l1 = lam + (int64_t)j * np;
    const double* l2 = lam + ((int64_t)n + j) * np;
    acc += elem_form3(l1, x2, m, k1, k2, k3) - elem_form3(l2, x1, m, k1, k2, k3);
  }
  part[(int64_t)blockIdx.y * nel + el] = acc;
}

// grad_P = -tau (h/12) a_P / 8 sum over the eight elements around P and the chunks
__global__ void __launch_bounds__(256) fevar3_grad_node_kernel(const double* __restrict__ part, int nchunks, int m,
                                                               double tau_h12, const double* __restrict__ a_int,
                                                               double* __restrict__ grad) {
  const int64_t np = (int64_t)m * m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  int i1, i2, i3;
  coords3(s, m, i1, i2, i3);
  const int me = m + 1;
  const int64_t nel = (int64_t)me * me * me;
  double acc = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const double* pc = part + (int64_t)c * nel;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      acc += pc[((int64_t)(i3 + (q >> 2)) * me + i2 + ((q >> 1) & 1)) * me + i1 + (q & 1)];
  }
  grad[s] = -0.125 * tau_h12 * a_int[s] * acc;
}

// (M u)_s * 216 / h^3 for u = x1/sqrt(gamma) - g (g != null) or x1, on one time block
__device__ __forceinline__ double m_err3(const double* __restrict__ x1, const double* __restrict__ g, double isg,
                                         int m, int i1, int i2, int i3) {
  double acc = 0.0;
#pragma unroll
  for (int o3 = -1; o3 <= 1; ++o3)
#pragma unroll
    for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
      for (int o1 = -1; o1 <= 1; ++o1) {
        const int q1 = i1 + o1, q2 = i2 + o2, q3 = i3 + o3;
        if (q1 < 0 || q1 >= m || q2 < 0 || q2 >= m || q3 < 0 || q3 >= m) continue;
        const int64_t q = ((int64_t)q3 * m + q2) * m + q1;
        acc = fma((double)m_weight(o1, o2, o3), g ? fma(x1[q], isg, -g[q]) : x1[q], acc);
      }
  return acc;
}

// partial[b] = sum over the block's points of e (M e) + p (M p) / gamma (times 216 / h^3)
__global__ void __launch_bounds__(256) fevar3_objective_kernel(const double* __restrict__ x,
                                                               const double* __restrict__ g, int m, int n, double isg,
                                                               double igam, double* __restrict__ partial) {
  __shared__ double red[8];
  const int64_t np = (int64_t)m * m * m, tot = np * n;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / np);
    const int64_t s = t - (int64_t)j * np;
    int i1, i2, i3;
    coords3(s, m, i1, i2, i3);
    const double* x1 = x + (int64_t)j * np;
    const double* x2 = x + ((int64_t)n + j) * np;
    const double* gj = g + (int64_t)j * np;
    const double e = fma(x1[s], isg, -gj[s]);
    acc = fma(e, m_err3(x1, gj, isg, m, i1, i2, i3), acc);
    acc = fma(igam * x2[s], m_err3(x2, nullptr, 0.0, m, i1, i2, i3), acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void fevar3_objective_finish_kernel(const double* __restrict__ partial, int nb, double c,
                                               double* __restrict__ J) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) acc += partial[b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) *J = 0.5 * c * acc;
}

// gJ times: dJ/dx1 = c M e / sqrt(gamma), dJ/dx2 = c M p / gamma, dJ/dg = -c M e
// (c = tau h^3 / 216 with the integer mass stencil)
__global__ void __launch_bounds__(256) fevar3_objective_grad_kernel(const double* __restrict__ x,
                                                                    const double* __restrict__ g, int m, int n,
                                                                    double isg, double igam, double c,
                                                                    const double* __restrict__ gJ,
                                                                    double* __restrict__ gx, double* __restrict__ gg) {
  const int64_t np = (int64_t)m * m * m, tot = np * n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int j = (int)(t / np);
  const int64_t s = t - (int64_t)j * np;
  int i1, i2, i3;
  coords3(s, m, i1, i2, i3);
  const double sc = c * (gJ ? *gJ : 1.0);
  const double* x1 = x + (int64_t)j * np;
  const double* x2 = x + ((int64_t)n + j) * np;
  const double Me = m_err3(x1, g + (int64_t)j * np, isg, m, i1, i2, i3);
  if (gx) {
    gx[t] = sc * Me * isg;
    gx[tot + t] = sc * igam * m_err3(x2, nullptr, 0.0, m, i1, i2, i3);
  }
  if (gg) gg[t] = -sc * Me;
}

// element coefficients of the level whose node I is node stride * I of the finest
// grid with boundary (M0 nodes per axis): the mean of each element's corner values
__global__ void __launch_bounds__(256) fevar3_level_elements_kernel(const double* __restrict__ a_nodes, int M0,
                                                                    int stride, int m, double* __restrict__ e64,
                                                                    float* __restrict__ e32) {
  const int me = m + 1;
  const int64_t el = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= (int64_t)me * me * me) return;
  int k1, k2, k3;
  coords3(el, me, k1, k2, k3);
  double v = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const size_t n1 = (size_t)(k1 + (c & 1)) * stride, n2 = (size_t)(k2 + ((c >> 1) & 1)) * stride,
                 n3 = (size_t)(k3 + (c >> 2)) * stride;
    v += a_nodes[(n3 * M0 + n2) * M0 + n1];
  }
  v *= 0.125;
  e64[el] = v;
  e32[el] = (float)v;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers (h: the level's mesh width)
// ---------------------------------------------------------------------------
static dim3 grid3(int64_t count, int y) { return dim3((unsigned)((count + 255) / 256), (unsigned)y); }

cudaError_t launch_fevar3_apply(Launch& L, int m, int planes, double h, const double* E, double cM, double cK,
                                const double* in, double beta, double* out) {
  const int64_t np = (int64_t)m * m * m;
  L.begin(KC_FE_APPLY);
  fevar3_apply_kernel<<<grid3(np, planes), 256, 0, L.stream>>>(in, out, E, m, h * h * h / 216.0, h / 12.0, planes,
                                                               cM, cK, beta);
  return L.end(KC_FE_APPLY, (double)np * planes * (beta != 0.0 ? 24.0 : 16.0), (double)np * planes * 100.0);
}

template <typename Tin>
cudaError_t launch_matvec_fevar3(Launch& L, int m, int n, double h, double alpha, double tau, const double* E,
                                 const Tin* x, double* y, bool transpose, size_t xstride, size_t ystride,
                                 const int* jdev) {
  const int64_t np = (int64_t)m * m * m;
  const int tj = n < 16 ? n : 16;
  const dim3 grid = grid3(np, (n + tj - 1) / tj);
  const double tot = 2.0 * n * (double)np, mh = h * h * h / 216.0, kh = h / 12.0;
  L.begin(KC_MATVEC);
  if constexpr (std::is_same<Tin, float>::value) {
    if (transpose)
      fevar3_matvec_df_kernel<true><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, mh, kh, alpha, tau, xstride,
                                                                ystride, jdev);
    else
      fevar3_matvec_df_kernel<false><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, mh, kh, alpha, tau, xstride,
                                                                 ystride, jdev);
    return L.end(KC_MATVEC, tot * (sizeof(Tin) + 8.0), tot * 400.0);
  } else {
    if (transpose)
      fevar3_matvec_kernel<Tin, true><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, mh, kh, alpha, tau, xstride,
                                                                  ystride, jdev);
    else
      fevar3_matvec_kernel<Tin, false><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, mh, kh, alpha, tau, xstride,
                                                                   ystride, jdev);
    return L.end(KC_MATVEC, tot * (sizeof(Tin) + 8.0), tot * 100.0);
  }
}

template <typename Tc>
cudaError_t launch_fevar3_smooth(Launch& L, int m, int planes, Tc h, Tc tau, const Tc* E,
                                 const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r,
                                 typename Cx<Tc>::t* u) {
  const double cs = sizeof(typename Cx<Tc>::t);
  const double np = (double)m * m * m;
  L.begin(KC_MG_SMOOTH);
  for (int c = 0; c < 8; ++c) {
    const int64_t nx = (m - (c & 1) + 1) / 2, ny = (m - ((c >> 1) & 1) + 1) / 2, nz = (m - (c >> 2) + 1) / 2;
    if (nx * ny * nz == 0) continue;
    fevar3_smooth_kernel<Tc><<<grid3(nx * ny * nz, planes), 256, 0, L.stream>>>(
        r, u, E, sigma, m, h * h * h / Tc(216), tau * h / Tc(12), c, planes);
  }
  return L.end(KC_MG_SMOOTH, np * planes * 3.0 * cs, np * planes * 150.0);
}

template <typename Tc>
cudaError_t launch_fevar3_resid_restrict(Launch& L, int m, int planes, Tc h, Tc tau, const Tc* E,
                                         const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r,
                                         const typename Cx<Tc>::t* u, typename Cx<Tc>::t* res,
                                         typename Cx<Tc>::t* rc) {
  const double cs = sizeof(typename Cx<Tc>::t);
  const int64_t mc = (m - 1) / 2;
  const int64_t np = (int64_t)m * m * m;
  L.begin(KC_MG_RESID_RESTRICT);
  fevar3_residual_kernel<Tc><<<grid3(np, planes), 256, 0, L.stream>>>(r, u, res, E, sigma, m, h * h * h / Tc(216),
                                                                      tau * h / Tc(12), planes);
  fevar3_restrict_kernel<Tc><<<grid3(mc * mc * mc, planes), 256, 0, L.stream>>>(res, rc, m, planes);
  return L.end(KC_MG_RESID_RESTRICT, (double)np * planes * 4.0 * cs, (double)np * planes * 150.0);
}

cudaError_t launch_fevar3_level_elements(Launch& L, const double* a_nodes, int M0, int stride, int m, double* e64,
                                         float* e32) {
  const int64_t me = m + 1;
  fevar3_level_elements_kernel<<<(unsigned)((me * me * me + 255) / 256), 256, 0, L.stream>>>(a_nodes, M0, stride, m,
                                                                                            e64, e32);
  return cudaGetLastError();
}

cudaError_t launch_fevar3_grad(Launch& L, int m, int n, double h, double tau, const double* a_int, const double* x,
                               const double* lam, double* part, int max_chunks, double* grad) {
  int tj = 1;
  while ((n + tj - 1) / tj > max_chunks) tj *= 2;
  const int nchunks = (n + tj - 1) / tj;
  const int64_t me = m + 1, np = (int64_t)m * m * m;
  L.begin(KC_GRAD);
  fevar3_grad_elem_kernel<<<grid3(me * me * me, nchunks), 256, 0, L.stream>>>(x, lam, m, n, tj, part);
  fevar3_grad_node_kernel<<<(unsigned)((np + 255) / 256), 256, 0, L.stream>>>(part, nchunks, m, tau * h / 12.0,
                                                                             a_int, grad);
  return L.end(KC_GRAD, 32.0 * n * (double)np, 200.0 * n * (double)np);
}

cudaError_t launch_fevar3_objective(Launch& L, int m, int n, double h, double tau, double gamma, const double* x,
                                    const double* g, double* partial, int max_partial, double* J) {
  const int64_t tot = (int64_t)m * m * m * n;
  int nb = (int)std::min<int64_t>((tot + 255) / 256, 1216);
  if (nb > max_partial) nb = max_partial;
  if (nb < 1) return cudaErrorInvalidValue;
  L.begin(KC_REDUCE);
  fevar3_objective_kernel<<<nb, 256, 0, L.stream>>>(x, g, m, n, 1.0 / sqrt(gamma), 1.0 / gamma, partial);
  fevar3_objective_finish_kernel<<<1, 32, 0, L.stream>>>(partial, nb, tau * h * h * h / 216.0, J);
  return L.end(KC_REDUCE, 24.0 * tot, 80.0 * tot);
}

cudaError_t launch_fevar3_objective_grad(Launch& L, int m, int n, double h, double tau, double gamma,
                                         const double* x, const double* g, const double* gJ, double* gx,
                                         double* gg) {
  const int64_t tot = (int64_t)m * m * m * n;
  L.begin(KC_GRAD);
  fevar3_objective_grad_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(
      x, g, m, n, 1.0 / sqrt(gamma), 1.0 / gamma, tau * h * h * h / 216.0, gJ, gx, gg);
  return L.end(KC_GRAD, 32.0 * tot, 100.0 * tot);
}

template cudaError_t launch_matvec_fevar3<double>(Launch&, int, int, double, double, double, const double*,
                                                  const double*, double*, bool, size_t, size_t, const int*);
template cudaError_t launch_matvec_fevar3<float>(Launch&, int, int, double, double, double, const double*,
                                                 const float*, double*, bool, size_t, size_t, const int*);
#define PCOPT_FV3(Tc)                                                                                              \
  template cudaError_t launch_fevar3_smooth<Tc>(Launch&, int, int, Tc, Tc, const Tc*, const Cx<Tc>::t*,           \
                                                const Cx<Tc>::t*, Cx<Tc>::t*);                                    \
  template cudaError_t launch_fevar3_resid_restrict<Tc>(Launch&, int, int, Tc, Tc, const Tc*, const Cx<Tc>::t*,   \
                                                        const Cx<Tc>::t*, const Cx<Tc>::t*, Cx<Tc>::t*,           \
                                                        Cx<Tc>::t*);
PCOPT_FV3(double)
PCOPT_FV3(float)
#undef PCOPT_FV3

}  // namespace pcopt
