// Bilinear elements with a nodal coefficient (Section 1: M and K of a finite-element
// discretisation), 2D.  K(a) = sum_e a_e K_e with a_e the mean of element e's four
// corner values and K_e the element stiffness of a = 1; M the consistent mass matrix.
// On the uniform grid both are 9-point stencils; at interior node (i1, i2), with the
// coefficients of its four elements SW = E(i1, i2), SE = E(i1+1, i2), NW = E(i1, i2+1),
// NE = E(i1+1, i2+1) (element (k1, k2) has its lower-left corner at node (k1, k2) of the
// grid with boundary, so interior node (i1, i2) is grid node (i1+1, i2+1)):
//   K: centre 2/3 (SW+SE+NW+NE); east -(SE+NE)/6, west -(SW+NW)/6, north -(NW+NE)/6,
//      south -(SW+SE)/6; corners -NE/3, -NW/3, -SE/3, -SW/3 (independent of h in 2D);
//   M: h^2 (16, 4, 1)/36 for the centre, the edges and the corners.
// This file: the all-at-once product, the product of single fields, the multicolour
// V(1,0) multigrid kernels for (sigma M + tau K(a)), the stiffness derivative of the
// gradient and the element objective.
#include <algorithm>

#include "common.cuh"

namespace pcopt {

namespace {

// the nine K entries of interior node (i1, i2) from the element coefficients
template <typename T>
struct KStencil {
  T c, e, w, n, s, ne, nw, se, sw;
};

template <typename T>
__device__ __forceinline__ KStencil<T> k_stencil(const T* __restrict__ E, int m, int i1, int i2) {
  const int me = m + 1;
  const T SW = E[i2 * me + i1], SE = E[i2 * me + i1 + 1];
  const T NW = E[(i2 + 1) * me + i1], NE = E[(i2 + 1) * me + i1 + 1];
  const T s6 = T(1) / T(6), s3 = T(1) / T(3);
  KStencil<T> k;
  k.c = T(2) / T(3) * (SW + SE + NW + NE);
  k.e = -s6 * (SE + NE);
  k.w = -s6 * (SW + NW);
  k.n = -s6 * (NW + NE);
  k.s = -s6 * (SW + SE);
  k.ne = -s3 * NE;
  k.nw = -s3 * NW;
  k.se = -s3 * SE;
  k.sw = -s3 * SW;
  return k;
}

// (M u)_P / h^2 * 36 and (K u)_P for a real field with zero boundary values:
// neighbours outside the grid contribute nothing
template <typename T, typename Tin>
__device__ __forceinline__ void mk_apply(const Tin* __restrict__ u, const KStencil<T>& k, int m, int i1, int i2,
                                         T& mu36, T& ku) {
  const int s = i2 * m + i1;
  const bool w = i1 > 0, e = i1 < m - 1, so = i2 > 0, no = i2 < m - 1;
  // FP32 inputs widen on the integer pipes (cvt): GB300 runs F2F on its FP64 unit
  const T uc = cvt<T>(u[s]);
  const T uw = w ? cvt<T>(u[s - 1]) : T(0), ue = e ? cvt<T>(u[s + 1]) : T(0);
  const T us = so ? cvt<T>(u[s - m]) : T(0), un = no ? cvt<T>(u[s + m]) : T(0);
  const T usw = (so && w) ? cvt<T>(u[s - m - 1]) : T(0), use = (so && e) ? cvt<T>(u[s - m + 1]) : T(0);
  const T unw = (no && w) ? cvt<T>(u[s + m - 1]) : T(0), une = (no && e) ? cvt<T>(u[s + m + 1]) : T(0);
  mu36 = T(16) * uc + T(4) * (uw + ue + us + un) + (usw + use + unw + une);
  ku = k.c * uc + k.e * ue + k.w * uw + k.n * un + k.s * us + k.ne * une + k.nw * unw + k.se * use + k.sw * usw;
}

// out_p = cM M in_p + cK K in_p + beta out_p, FP64, `planes` fields of m^2 values
__global__ void __launch_bounds__(256) fevar_apply_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                          const double* __restrict__ E, int m, double h2, int planes,
                                                          double cM, double cK, double beta) {
  const int64_t np = (int64_t)m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (s >= np || p >= planes) return;
  const int i2 = (int)(s / m), i1 = (int)(s - (int64_t)i2 * m);
  const KStencil<double> k = k_stencil(E, m, i1, i2);
  double mu36, ku;
  mk_apply(in + p * np, k, m, i1, i2, mu36, ku);
  double v = cM * (h2 / 36.0) * mu36 + cK * ku;
  if (beta != 0.0) v = fma(beta, out[p * np + s], v);
  out[p * np + s] = v;
}

// All-at-once product A x (or A^T x) with A = [[alpha I(x)M, T^T], [-T, alpha I(x)M]],
// (T v)_j = M v_j - M v_{j-1} + tau K v_j.  One thread per spatial point and chunk of
// time blocks [j0, j1); M x1 at j0 - 1 and M x2 at j1 are formed at the chunk ends.
//   y1_j = alpha M x1_j + sg (M x2_j - M x2_{j+1} + tau K x2_j)
//   y2_j = alpha M x2_j - sg (M x1_j - M x1_{j-1} + tau K x1_j),   sg = -1 for A^T.
template <typename Tin, bool TRANSPOSE>
__global__ void __launch_bounds__(256) fevar_matvec_kernel(const Tin* __restrict__ x, double* __restrict__ y,
                                                           const double* __restrict__ E, int m, int n, int tj,
                                                           double h2, double alpha, double tau, size_t xstride,
                                                           size_t ystride, const int* __restrict__ jdev) {
  const int64_t np = (int64_t)m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  if (jdev) {  // device-resident Arnoldi index: x = Z_j, y = V_{j+1}
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int j0 = blockIdx.y * tj, j1 = min(n, j0 + tj);
  if (j0 >= n) return;
  const int i2 = (int)(s / m), i1 = (int)(s - (int64_t)i2 * m);
  const KStencil<double> k = k_stencil(E, m, i1, i2);
  const double mh = h2 / 36.0, sg = TRANSPOSE ? -1.0 : 1.0;
  const Tin* x1 = x;
  const Tin* x2 = x + (int64_t)n * np;
  double* y1 = y;
  double* y2 = y + (int64_t)n * np;
  double Mx1p = 0.0;  // M x1_{j-1}
  if (j0 > 0) {
    double mu, ku;
    mk_apply(x1 + (int64_t)(j0 - 1) * np, k, m, i1, i2, mu, ku);
    Mx1p = mh * mu;
  }
  double pMx1 = 0.0, pMx2 = 0.0, pKx2 = 0.0;  // block j - 1 of this chunk
  for (int j = j0; j < j1; ++j) {
    double mu1, ku1, mu2, ku2;
    mk_apply(x1 + (int64_t)j * np, k, m, i1, i2, mu1, ku1);
    mk_apply(x2 + (int64_t)j * np, k, m, i1, i2, mu2, ku2);
    const double Mx1 = mh * mu1, Mx2 = mh * mu2;
    y2[(int64_t)j * np + s] = alpha * Mx2 - sg * (Mx1 - Mx1p + tau * ku1);
    if (j > j0) y1[(int64_t)(j - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2 + tau * pKx2);
    Mx1p = Mx1;
    pMx1 = Mx1;
    pMx2 = Mx2;
    pKx2 = ku2;
  }
  double Mx2n = 0.0;  // M x2_{j1}
  if (j1 < n) {
    double mu, ku;
    mk_apply(x2 + (int64_t)j1 * np, k, m, i1, i2, mu, ku);
    Mx2n = mh * mu;
  }
  y1[(int64_t)(j1 - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2n + tau * pKx2);
}

}  // namespace

// ---------------------------------------------------------------------------
// Multigrid for (sigma M + tau K(a)): one Gauss-Seidel sweep from zero in colour
// order (colour c = (i1 & 1) + 2 (i2 & 1); points of one colour are not coupled),
// residual, restriction by P^T, recursion, bilinear correction (launch_mg_prolong),
// the one-point level solved by the sweep itself.
// ---------------------------------------------------------------------------
namespace {

// sum over the neighbours q of P selected by `take` of M_Pq u_q * 36 / h^2 and K_Pq u_q
template <typename Tc, typename Take>
__device__ __forceinline__ void mk_offdiag(const typename Cx<Tc>::t* __restrict__ u, const KStencil<Tc>& k, int m,
                                           int i1, int i2, Take take, typename Cx<Tc>::t& mu36,
                                           typename Cx<Tc>::t& ku) {
  typedef typename Cx<Tc>::t C;
  mu36 = czero<Tc>();
  ku = czero<Tc>();
  const int s = i2 * m + i1;
#pragma unroll
  for (int d2 = -1; d2 <= 1; ++d2)
#pragma unroll
    for (int d1 = -1; d1 <= 1; ++d1) {
      if (d1 == 0 && d2 == 0) continue;
      const int q1 = i1 + d1, q2 = i2 + d2;
      if (q1 < 0 || q1 >= m || q2 < 0 || q2 >= m || !take(d1, d2)) continue;
      const C v = u[s + d2 * m + d1];
      const Tc wm = (d1 != 0 && d2 != 0) ? Tc(1) : Tc(4);
      const Tc wk = d2 == 0 ? (d1 > 0 ? k.e : k.w)
                            : d1 == 0 ? (d2 > 0 ? k.n : k.s)
                                      : d2 > 0 ? (d1 > 0 ? k.ne : k.nw) : (d1 > 0 ? k.se : k.sw);
      mu36.x = fma(wm, v.x, mu36.x);
      mu36.y = fma(wm, v.y, mu36.y);
      ku.x = fma(wk, v.x, ku.x);
      ku.y = fma(wk, v.y, ku.y);
    }
}

// sigma * M-part + tau * K-part of a complex neighbour sum
template <typename Tc>
__device__ __forceinline__ typename Cx<Tc>::t shifted(typename Cx<Tc>::t sig, typename Cx<Tc>::t mu36, Tc mh,
                                                      typename Cx<Tc>::t ku, Tc tau) {
  typename Cx<Tc>::t r;
  r.x = mh * (sig.x * mu36.x - sig.y * mu36.y) + tau * ku.x;
  r.y = mh * (sig.x * mu36.y + sig.y * mu36.x) + tau * ku.y;
  return r;
}

// points of colour c: i1 = (c & 1) + 2 (t % nx), i2 = (c >> 1) + 2 (t / nx)
template <typename Tc>
__global__ void __launch_bounds__(256) fevar_smooth_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                           typename Cx<Tc>::t* __restrict__ u,
                                                           const Tc* __restrict__ E,
                                                           const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                           Tc h2, Tc tau, int colour, int planes) {
  typedef typename Cx<Tc>::t C;
  const int px = colour & 1, py = colour >> 1;
  const int nx = (m - px + 1) / 2, ny = (m - py + 1) / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (t >= nx * ny || p >= planes) return;
  const int i1 = px + 2 * (t % nx), i2 = py + 2 * (t / nx);
  const int64_t np = (int64_t)m * m;
  const C* rp = r + p * np;
  C* up = u + p * np;
  const KStencil<Tc> k = k_stencil(E, m, i1, i2);
  // a neighbour counts once its colour has been swept (the others are still zero)
  auto take = [&](int d1, int d2) { return (((px ^ (d1 & 1)) + 2 * (py ^ (d2 & 1))) < colour); };
  C mu36, ku;
  mk_offdiag<Tc>(up, k, m, i1, i2, take, mu36, ku);
  const C sig = sigma[p];
  const Tc mh = h2 / Tc(36);
  const C off = shifted<Tc>(sig, mu36, mh, ku, tau);
  const int s = i2 * m + i1;
  C acc = rp[s];
  acc.x -= off.x;
  acc.y -= off.y;
  C dg;
  dg.x = sig.x * (Tc(16) * mh) + tau * k.c;
  dg.y = sig.y * (Tc(16) * mh);
  up[s] = cmul(acc, cinv(dg));
}

// res = r - (sigma M + tau K) u at every point
template <typename Tc>
__global__ void __launch_bounds__(256) fevar_residual_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                             const typename Cx<Tc>::t* __restrict__ u,
                                                             typename Cx<Tc>::t* __restrict__ res,
                                                             const Tc* __restrict__ E,
                                                             const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                             Tc h2, Tc tau, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t np = (int64_t)m * m;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (s >= np || p >= planes) return;
  const int i2 = s / m, i1 = s - i2 * m;
  const C* up = u + p * np;
  const KStencil<Tc> k = k_stencil(E, m, i1, i2);
  C mu36, ku;
  mk_offdiag<Tc>(up, k, m, i1, i2, [](int, int) { return true; }, mu36, ku);
  const C uc = up[s];
  mu36.x = fma(Tc(16), uc.x, mu36.x);
  mu36.y = fma(Tc(16), uc.y, mu36.y);
  ku.x = fma(k.c, uc.x, ku.x);
  ku.y = fma(k.c, uc.y, ku.y);
  const C au = shifted<Tc>(sigma[p], mu36, h2 / Tc(36), ku, tau);
  const C rv = r[p * np + s];
  res[p * np + s] = rv - au;
}

// rc(I, J) = sum_{o1, o2 in -1..1} w(o1) w(o2) res(2I+1+o1, 2J+1+o2), w(0) = 1,
// w(+-1) = 1/2: the transpose of bilinear interpolation
template <typename Tc>
__global__ void __launch_bounds__(256) fevar_restrict_kernel(const typename Cx<Tc>::t* __restrict__ res,
                                                             typename Cx<Tc>::t* __restrict__ rc, int m, int planes) {
  typedef typename Cx<Tc>::t C;
  const int mc = (m - 1) / 2;
  const int sc = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (sc >= mc * mc || p >= planes) return;
  const int J = sc / mc, I = sc - J * mc;
  const C* rp = res + (int64_t)p * m * m;
  C acc = czero<Tc>();
#pragma unroll
  for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
    for (int o1 = -1; o1 <= 1; ++o1) {
      const Tc wt = (o1 == 0 ? Tc(1) : Tc(0.5)) * (o2 == 0 ? Tc(1) : Tc(0.5));
      const C v = rp[(2 * J + 1 + o2) * m + 2 * I + 1 + o1];
      acc.x = fma(wt, v.x, acc.x);
      acc.y = fma(wt, v.y, acc.y);
    }
  rc[(int64_t)p * mc * mc + sc] = acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// Gradient and objective with element matrices
// ---------------------------------------------------------------------------
namespace {

// value of field u (m^2 per time block) at grid node (g1, g2) of the grid with boundary
__device__ __forceinline__ double node_val(const double* __restrict__ u, int m, int g1, int g2) {
  return (g1 >= 1 && g1 <= m && g2 >= 1 && g2 <= m) ? u[(g2 - 1) * m + (g1 - 1)] : 0.0;
}

// u_e^T K_e v_e for the element with lower-left grid node (k1, k2), K_e of a = 1:
// 1/6 [4 on the diagonal, -1 between corners sharing an edge, -2 between opposite ones]
__device__ __forceinline__ double elem_form(const double* __restrict__ u, const double* __restrict__ v, int m, int k1,
                                            int k2) {
  const double u0 = node_val(u, m, k1, k2), u1 = node_val(u, m, k1 + 1, k2);
  const double u2 = node_val(u, m, k1, k2 + 1), u3 = node_val(u, m, k1 + 1, k2 + 1);
  const double v0 = node_val(v, m, k1, k2), v1 = node_val(v, m, k1 + 1, k2);
  const double v2 = node_val(v, m, k1, k2 + 1), v3 = node_val(v, m, k1 + 1, k2 + 1);
  const double diag = u0 * v0 + u1 * v1 + u2 * v2 + u3 * v3;
  const double edge = u0 * (v1 + v2) + u1 * (v0 + v3) + u2 * (v0 + v3) + u3 * (v1 + v2);
  const double opp = u0 * v3 + u3 * v0 + u1 * v2 + u2 * v1;
  return (4.0 * diag - edge - 2.0 * opp) / 6.0;
}

// part[c][e] = sum_{j in chunk c} (lam1_j^T K_e x2_j - lam2_j^T K_e x1_j)
__global__ void __launch_bounds__(256) fevar_grad_elem_kernel(const double* __restrict__ x,
                                                              const double* __restrict__ lam, int m, int n, int tj,
                                                              double* __restrict__ part) {
  const int me = m + 1;
  const int el = blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= me * me) return;
  const int k2 = el / me, k1 = el - k2 * me;
  const int64_t np = (int64_t)m * m;
  const int j0 = blockIdx.y * tj, j1 = min(n, j0 + tj);
  double acc = 0.0;
  for (int j = j0; j < j1; ++j) {
    const double* x1 = x + (int64_t)j * np;
    const double* x2 = x + ((int64_t)n + j) * np;
    const double* l1 = lam + (int64_t)j * np;
    const double* l2 = lam + ((int64_t)n + j) * np;
    acc += elem_form(l1, x2, m, k1, k2) - elem_form(l2, x1, m, k1, k2);
  }
  part[(int64_t)blockIdx.y * me * me + el] = acc;
}

// grad_P = -tau a_P / 4 sum over the four elements around P and the chunks
__global__ void __launch_bounds__(256) fevar_grad_node_kernel(const double* __restrict__ part, int nchunks, int m,
                                                              double tau, const double* __restrict__ a_int,
                                                              double* __restrict__ grad) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m * m) return;
  const int i2 = s / m, i1 = s - i2 * m;
  const int me = m + 1;
  double acc = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const double* pc = part + (int64_t)c * me * me;
    acc += pc[i2 * me + i1] + pc[i2 * me + i1 + 1] + pc[(i2 + 1) * me + i1] + pc[(i2 + 1) * me + i1 + 1];
  }
  grad[s] = -0.25 * tau * a_int[s] * acc;
}

// (M u)_s for u = x1/sqrt(gamma) - g (sel 0), x2 (sel 1), on time block j
__device__ __forceinline__ double m_err(const double* __restrict__ x1, const double* __restrict__ g, double isg,
                                        int m, int i1, int i2) {
  double acc = 0.0;
#pragma unroll
  for (int d2 = -1; d2 <= 1; ++d2)
#pragma unroll
    for (int d1 = -1; d1 <= 1; ++d1) {
      const int q1 = i1 + d1, q2 = i2 + d2;
      if (q1 < 0 || q1 >= m || q2 < 0 || q2 >= m) continue;
      const int q = q2 * m + q1;
      const double w = (d1 == 0 && d2 == 0) ? 16.0 : (d1 == 0 || d2 == 0) ? 4.0 : 1.0;
      acc = fma(w, g ? fma(x1[q], isg, -g[q]) : x1[q], acc);
    }
  return acc;
}

// partial[b] = sum over the block's points of e (M e) + p (M p) / gamma (times 36 / h^2)
__global__ void __launch_bounds__(256) fevar_objective_kernel(const double* __restrict__ x,
                                                              const double* __restrict__ g, int m, int n, double isg,
                                                              double igam, double* __restrict__ partial) {
  __shared__ double red[8];
  const int64_t np = (int64_t)m * m, tot = np * n;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / np);
    const int s = (int)(t - (int64_t)j * np);
    const int i2 = s / m, i1 = s - i2 * m;
    const double* x1 = x + (int64_t)j * np;
    const double* x2 = x + ((int64_t)n + j) * np;
    const double* gj = g + (int64_t)j * np;
    const double e = fma(x1[s], isg, -gj[s]);
    acc = fma(e, m_err(x1, gj, isg, m, i1, i2), acc);
    acc = fma(igam * x2[s], m_err(x2, nullptr, 0.0, m, i1, i2), acc);
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

__global__ void fevar_objective_finish_kernel(const double* __restrict__ partial, int nb, double c,
                                              double* __restrict__ J) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) acc += partial[b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) *J = 0.5 * c * acc;
}

// gJ times: dJ/dx1 = c M e / sqrt(gamma), dJ/dx2 = c M p / gamma, dJ/dg = -c M e
// (c = tau h^2 / 36 with the integer mass stencil)
__global__ void __launch_bounds__(256) fevar_objective_grad_kernel(const double* __restrict__ x,
                                                                   const double* __restrict__ g, int m, int n,
                                                                   double isg, double igam, double c,
                                                                   const double* __restrict__ gJ,
                                                                   double* __restrict__ gx, double* __restrict__ gg) {
  const int64_t np = (int64_t)m * m, tot = np * n;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int j = (int)(t / np);
  const int s = (int)(t - (int64_t)j * np);
  const int i2 = s / m, i1 = s - i2 * m;
  const double sc = c * (gJ ? *gJ : 1.0);
  const double* x1 = x + (int64_t)j * np;
  const double* x2 = x + ((int64_t)n + j) * np;
  const double Me = m_err(x1, g + (int64_t)j * np, isg, m, i1, i2);
  if (gx) {
    gx[t] = sc * Me * isg;
    gx[tot + t] = sc * igam * m_err(x2, nullptr, 0.0, m, i1, i2);
  }
  if (gg) gg[t] = -sc * Me;
}

// element coefficients of the level whose node I is node stride * I of the finest
// grid with boundary (M0 nodes per axis): the mean of each element's corner values
__global__ void __launch_bounds__(256) fevar_level_elements_kernel(const double* __restrict__ a_nodes, int M0,
                                                                   int stride, int m, double* __restrict__ e64,
                                                                   float* __restrict__ e32) {
  const int me = m + 1;
  const int el = blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= me * me) return;
  const int k2 = el / me, k1 = el - k2 * me;
  auto at = [&](int n1, int n2) { return a_nodes[(size_t)(n2 * stride) * M0 + (size_t)n1 * stride]; };
  const double v = 0.25 * (at(k1, k2) + at(k1 + 1, k2) + at(k1, k2 + 1) + at(k1 + 1, k2 + 1));
  e64[el] = v;
  e32[el] = (float)v;
}

}  // namespace

// ---------------------------------------------------------------------------
// Element product of an FP32 vector (the inner product of flexible GMRES) in
// double-float arithmetic: the nine K entries of a point are split once into FP32
// (hi, lo) pairs; per time block and half, M u (integer weights on FP32 values, every
// term exact) and K u (exact products hi * u by FMA, lo * u rounded) are summed with
// Knuth's TwoSum into (sum, error) pairs, widened on the integer pipes and combined
// in FP64 (a few FP64 operations per output instead of ~45).  Relative error of a
// sum: about 2^-44 of the sum of the magnitudes of its terms.
// ---------------------------------------------------------------------------
namespace {

struct DF {
  float hi, lo;
};

// (hi, lo) += x exactly (TwoSum; no contraction into FMA)
__device__ __forceinline__ void df_add(DF& a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

// (hi, lo) += (kh + kl) u
__device__ __forceinline__ void df_add_prod(DF& a, float kh, float kl, float u) {
  const float p = __fmul_rn(kh, u);
  const float e = fmaf(kh, u, -p);
  df_add(a, p);
  a.lo = __fadd_rn(a.lo, fmaf(kl, u, e));
}

__device__ __forceinline__ double df_val(const DF& a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }

struct KSplit {
  float h[9], l[9];  // centre, e, w, n, s, ne, nw, se, sw
};

__device__ __forceinline__ void mk_apply_df(const float* __restrict__ u, const KSplit& k, int m, int i1, int i2,
                                            double& mu36, double& ku) {
  const int s = i2 * m + i1;
  const bool w = i1 > 0, e = i1 < m - 1, so = i2 > 0, no = i2 < m - 1;
  const float v[9] = {u[s], e ? u[s + 1] : 0.0f, w ? u[s - 1] : 0.0f, no ? u[s + m] : 0.0f,
                      so ? u[s - m] : 0.0f, (no && e) ? u[s + m + 1] : 0.0f, (no && w) ? u[s + m - 1] : 0.0f,
                      (so && e) ? u[s - m + 1] : 0.0f, (so && w) ? u[s - m - 1] : 0.0f};
  DF am{__fmul_rn(16.0f, v[0]), 0.0f};
#pragma unroll
  for (int q = 1; q < 5; ++q) df_add(am, __fmul_rn(4.0f, v[q]));
#pragma unroll
  for (int q = 5; q < 9; ++q) df_add(am, v[q]);
  DF ak{0.0f, 0.0f};
#pragma unroll
  for (int q = 0; q < 9; ++q) df_add_prod(ak, k.h[q], k.l[q], v[q]);
  mu36 = df_val(am);
  ku = df_val(ak);
}

template <bool TRANSPOSE>
__global__ void __launch_bounds__(256) fevar_matvec_df_kernel(const float* __restrict__ x, double* __restrict__ y,
                                                              const double* __restrict__ E, int m, int n, int tj,
                                                              double h2, double alpha, double tau, size_t xstride,
                                                              size_t ystride, const int* __restrict__ jdev) {
  const int64_t np = (int64_t)m * m;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  if (jdev) {  // device-resident Arnoldi index: x = Z_j, y = V_{j+1}
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int j0 = blockIdx.y * tj, j1 = min(n, j0 + tj);
  if (j0 >= n) return;
  const int i2 = (int)(s / m), i1 = (int)(s - (int64_t)i2 * m);
  KSplit k;
  {
    const KStencil<double> kd = k_stencil(E, m, i1, i2);
    const double kv[9] = {kd.c, kd.e, kd.w, kd.n, kd.s, kd.ne, kd.nw, kd.se, kd.sw};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      k.h[q] = f64_to_f32(kv[q]);
      k.l[q] = f64_to_f32(kv[q] - f32_to_f64(k.h[q]));
    }
  }
  const double mh = h2 / 36.0, sg = TRANSPOSE ? -1.0 : 1.0;
  const float* x1 = x;
  const float* x2 = x + (int64_t)n * np;
  double* y1 = y;
  double* y2 = y + (int64_t)n * np;
  double Mx1p = 0.0;
  if (j0 > 0) {
    double mu, ku;
    mk_apply_df(x1 + (int64_t)(j0 - 1) * np, k, m, i1, i2, mu, ku);
    Mx1p = mh * mu;
  }
  double pMx1 = 0.0, pMx2 = 0.0, pKx2 = 0.0;
  for (int j = j0; j < j1; ++j) {
    double mu1, ku1, mu2, ku2;
    mk_apply_df(x1 + (int64_t)j * np, k, m, i1, i2, mu1, ku1);
    mk_apply_df(x2 + (int64_t)j * np, k, m, i1, i2, mu2, ku2);
    const double Mx1 = mh * mu1, Mx2 = mh * mu2;
    y2[(int64_t)j * np + s] = alpha * Mx2 - sg * (Mx1 - Mx1p + tau * ku1);
    if (j > j0) y1[(int64_t)(j - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2 + tau * pKx2);
    Mx1p = Mx1;
    pMx1 = Mx1;
    pMx2 = Mx2;
    pKx2 = ku2;
  }
  double Mx2n = 0.0;
  if (j1 < n) {
    double mu, ku;
    mk_apply_df(x2 + (int64_t)j1 * np, k, m, i1, i2, mu, ku);
    Mx2n = mh * mu;
  }
  y1[(int64_t)(j1 - 1) * np + s] = alpha * pMx1 + sg * (pMx2 - Mx2n + tau * pKx2);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static dim3 grid2(int64_t count, int y) { return dim3((unsigned)((count + 255) / 256), (unsigned)y); }

cudaError_t launch_fevar_apply(Launch& L, int m, int planes, double h2, const double* E, double cM, double cK,
                               const double* in, double beta, double* out) {
  const double np = (double)m * m * planes;
  L.begin(KC_FE_APPLY);
  fevar_apply_kernel<<<grid2((int64_t)m * m, planes), 256, 0, L.stream>>>(in, out, E, m, h2, planes, cM, cK, beta);
  return L.end(KC_FE_APPLY, np * (beta != 0.0 ? 24.0 : 16.0), np * 40.0);
}

template <typename Tin>
cudaError_t launch_matvec_fevar(Launch& L, int m, int n, double h2, double alpha, double tau, const double* E,
                                const Tin* x, double* y, bool transpose, size_t xstride, size_t ystride,
                                const int* jdev) {
  const int tj = n < 16 ? n : 16;
  const dim3 grid = grid2((int64_t)m * m, (n + tj - 1) / tj);
  const double tot = 2.0 * n * (double)m * m;
  L.begin(KC_MATVEC);
  if constexpr (std::is_same<Tin, float>::value) {
    if (transpose)
      fevar_matvec_df_kernel<true><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, h2, alpha, tau, xstride, ystride,
                                                               jdev);
    else
      fevar_matvec_df_kernel<false><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, h2, alpha, tau, xstride, ystride,
                                                                jdev);
    return L.end(KC_MATVEC, tot * (sizeof(Tin) + 8.0), tot * 160.0);
  }
  if (transpose)
    fevar_matvec_kernel<Tin, true><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, h2, alpha, tau, xstride, ystride,
                                                               jdev);
  else
    fevar_matvec_kernel<Tin, false><<<grid, 256, 0, L.stream>>>(x, y, E, m, n, tj, h2, alpha, tau, xstride, ystride,
                                                                jdev);
  return L.end(KC_MATVEC, tot * (sizeof(Tin) + 8.0), tot * 40.0);
}

template <typename Tc>
cudaError_t launch_fevar_smooth(Launch& L, int m, int planes, Tc h2, Tc tau, const Tc* E,
                                const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, typename Cx<Tc>::t* u) {
  const double cs = sizeof(typename Cx<Tc>::t);
  L.begin(KC_MG_SMOOTH);
  for (int c = 0; c < 4; ++c) {
    const int nx = (m - (c & 1) + 1) / 2, ny = (m - (c >> 1) + 1) / 2;
    if (nx * ny == 0) continue;
    fevar_smooth_kernel<Tc><<<grid2((int64_t)nx * ny, planes), 256, 0, L.stream>>>(r, u, E, sigma, m, h2, tau, c,
                                                                                  planes);
  }
  return L.end(KC_MG_SMOOTH, (double)m * m * planes * 3.0 * cs, (double)m * m * planes * 60.0);
}

template <typename Tc>
cudaError_t launch_fevar_resid_restrict(Launch& L, int m, int planes, Tc h2, Tc tau, const Tc* E,
                                        const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r,
                                        const typename Cx<Tc>::t* u, typename Cx<Tc>::t* res,
                                        typename Cx<Tc>::t* rc) {
  const double cs = sizeof(typename Cx<Tc>::t);
  const int mc = (m - 1) / 2;
  L.begin(KC_MG_RESID_RESTRICT);
  fevar_residual_kernel<Tc><<<grid2((int64_t)m * m, planes), 256, 0, L.stream>>>(r, u, res, E, sigma, m, h2, tau,
                                                                                 planes);
  fevar_restrict_kernel<Tc><<<grid2((int64_t)mc * mc, planes), 256, 0, L.stream>>>(res, rc, m, planes);
  return L.end(KC_MG_RESID_RESTRICT, (double)m * m * planes * 4.0 * cs, (double)m * m * planes * 60.0);
}

cudaError_t launch_fevar_grad(Launch& L, int m, int n, double tau, const double* a_int, const double* x,
                              const double* lam, double* part, int max_chunks, double* grad) {
  int tj = 1;
  while ((n + tj - 1) / tj > max_chunks) tj *= 2;
  const int nchunks = (n + tj - 1) / tj;
  const int me = m + 1;
  L.begin(KC_GRAD);
  fevar_grad_elem_kernel<<<grid2((int64_t)me * me, nchunks), 256, 0, L.stream>>>(x, lam, m, n, tj, part);
  fevar_grad_node_kernel<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, L.stream>>>(part, nchunks, m, tau,
                                                                                       a_int, grad);
  return L.end(KC_GRAD, 32.0 * n * (double)m * m, 100.0 * n * (double)m * m);
}

cudaError_t launch_fevar_objective(Launch& L, int m, int n, double h2, double tau, double gamma, const double* x,
                                   const double* g, double* partial, int max_partial, double* J) {
  const int64_t tot = (int64_t)m * m * n;
  int nb = (int)std::min<int64_t>((tot + 255) / 256, 1216);
  if (nb > max_partial) nb = max_partial;
  if (nb < 1) return cudaErrorInvalidValue;
  L.begin(KC_REDUCE);
  fevar_objective_kernel<<<nb, 256, 0, L.stream>>>(x, g, m, n, 1.0 / sqrt(gamma), 1.0 / gamma, partial);
  fevar_objective_finish_kernel<<<1, 32, 0, L.stream>>>(partial, nb, tau * h2 / 36.0, J);
  return L.end(KC_REDUCE, 24.0 * tot, 40.0 * tot);
}

cudaError_t launch_fevar_objective_grad(Launch& L, int m, int n, double h2, double tau, double gamma,
                                        const double* x, const double* g, const double* gJ, double* gx, double* gg) {
  const int64_t tot = (int64_t)m * m * n;
  L.begin(KC_GRAD);
  fevar_objective_grad_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(
      x, g, m, n, 1.0 / sqrt(gamma), 1.0 / gamma, tau * h2 / 36.0, gJ, gx, gg);
  return L.end(KC_GRAD, (24.0 + (gx ? 16.0 : 0.0) + (gg ? 8.0 : 0.0)) * tot, 40.0 * tot);
}

cudaError_t launch_fevar_level_elements(Launch& L, const double* a_nodes, int M0, int stride, int m, double* e64,
                                        float* e32) {
  const int64_t ne = (int64_t)(m + 1) * (m + 1);
  fevar_level_elements_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, L.stream>>>(a_nodes, M0, stride, m, e64, e32);
  return cudaGetLastError();
}

template cudaError_t launch_matvec_fevar<double>(Launch&, int, int, double, double, double, const double*,
                                                 const double*, double*, bool, size_t, size_t, const int*);
template cudaError_t launch_matvec_fevar<float>(Launch&, int, int, double, double, double, const double*,
                                                const float*, double*, bool, size_t, size_t, const int*);
#define PCOPT_INST_FEVAR(Tc)                                                                                    \
  template cudaError_t launch_fevar_smooth<Tc>(Launch&, int, int, Tc, Tc, const Tc*, const Cx<Tc>::t*,          \
                                               const Cx<Tc>::t*, Cx<Tc>::t*);                                   \
  template cudaError_t launch_fevar_resid_restrict<Tc>(Launch&, int, int, Tc, Tc, const Tc*, const Cx<Tc>::t*,  \
                                                       const Cx<Tc>::t*, const Cx<Tc>::t*, Cx<Tc>::t*, Cx<Tc>::t*);
PCOPT_INST_FEVAR(float)
PCOPT_INST_FEVAR(double)
#undef PCOPT_INST_FEVAR

}  // namespace pcopt
