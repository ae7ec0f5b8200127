// Finite elements in space (Section 1 with a mass matrix M != I): conforming
// bilinear (2D) / trilinear (3D) elements on the uniform grid, constant
// coefficient c.  Both matrices are Kronecker products of the 1D element matrices
//   M_1 = h/6 [1 4 1],   K_1 = 1/h [-1 2 -1],
// so with the unscaled 1D stencils S = [1 4 1] and D = [-1 2 -1]
//   M = wM * S (x) S [(x) S],            wM = (h/6)^dim,
//   K = wK * sum_axis D_axis (x) S_others,  wK = c (h/6)^(dim-1) / h.
// Every stencil is evaluated separably: a thread forms the column sums over the
// x2 (and x3) neighbours of its own x1 position,
//   q = S (x) S [..] v,   r = (D_x2 (x) S_x3 + S_x2 (x) D_x3) v   (2D: q = S v, r = D v),
// and the x1 direction then needs only the neighbouring columns:
//   M v = wM (q_-1 + 4 q_0 + q_+1),
//   K v = wK (2 q_0 - q_-1 - q_+1 + r_-1 + 4 r_0 + r_+1).
// In the all-at-once product these columns come from the warp's neighbouring
// lanes (shuffles); a warp spans 32 consecutive x1 columns and writes the 30
// inner ones.
#include <type_traits>

#include "common.cuh"

namespace pcopt {

namespace {

constexpr int kFeOut = 30;       // outputs per warp; lanes 0 and 31 hold the x1 halo
constexpr int kFeRowsPerCta = 8; // warps (grid rows) per 256-thread CTA
constexpr unsigned kFull = 0xffffffffu;

// column sums q, r at the point p (value at p = centre) from its x2 (and x3)
// neighbours; the flags say which neighbours are interior nodes
template <int DIM, typename Tin>
__device__ __forceinline__ void fe_column(const Tin* __restrict__ p, int64_t m, int64_t mm, bool e2m, bool e2p,
                                          bool e3m, bool e3p, double& q, double& r) {
  const double x0 = cvt<double>(p[0]);
  const double xs = cvt<double>(e2m ? p[-m] : Tin(0)), xn = cvt<double>(e2p ? p[m] : Tin(0));
  if (DIM == 2) {
    q = fma(4.0, x0, xs + xn);
    r = fma(6.0, x0, -q);  // 2 x0 - xs - xn
  } else {
    const double xb = cvt<double>(e3m ? p[-mm] : Tin(0)), xt = cvt<double>(e3p ? p[mm] : Tin(0));
    const double c = cvt<double>(e2m && e3m ? p[-m - mm] : Tin(0)) + cvt<double>(e2p && e3m ? p[m - mm] : Tin(0)) +
                     cvt<double>(e2m && e3p ? p[-m + mm] : Tin(0)) + cvt<double>(e2p && e3p ? p[m + mm] : Tin(0));
    const double e = (xs + xn) + (xb + xt);
    // S(x)S weights: 16 centre, 4 edges, 1 corners; D(x)S + S(x)D: 16 centre, -2 elsewhere
    q = fma(16.0, x0, fma(4.0, e, c));
    r = fma(16.0, x0, -2.0 * (c + e));
  }
}

// y = A x (or A^T x) with A = [[alpha I(x)M, T^T], [-T, alpha I(x)M]], T = B_n(x)M + tau I(x)K.
// wM and tKw = tau * wK scale the unscaled stencils.
template <typename Tin, int DIM, bool TRANSPOSE>
__global__ void __launch_bounds__(256) matvec_fe_kernel(const Tin* __restrict__ x, double* __restrict__ y, int m,
                                                        int64_t ms, int64_t rows, int segs, int n, int tj,
                                                        double alpha, double wM, double tKw, size_t xstride,
                                                        size_t ystride, const int* __restrict__ jdev) {
  if (jdev) {  // device-resident Arnoldi index: x = Z_j, y = V_{j+1}
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int lane = threadIdx.x & 31;
  const int seg = (int)(blockIdx.x % (unsigned)segs);
  const int64_t row = (int64_t)(blockIdx.x / (unsigned)segs) * kFeRowsPerCta + (threadIdx.x >> 5);
  if (row >= rows) return;  // whole warps leave together
  const int j0 = blockIdx.y * tj;
  const int j1 = min(n, j0 + tj);
  const int i1 = seg * kFeOut - 1 + lane;
  const bool has = i1 >= 0 && i1 < m;
  const bool out = has && lane >= 1 && lane <= kFeOut;
  const int i2 = (int)(DIM == 2 ? row : row % m);
  const int i3 = (int)(DIM == 3 ? row / m : 0);
  const bool e2m = i2 > 0, e2p = i2 < m - 1;
  const bool e3m = DIM == 3 && i3 > 0, e3p = DIM == 3 && i3 < m - 1;
  const int64_t mm = (int64_t)m * m;
  const int64_t s = row * m + (has ? i1 : 0);
  const Tin* x1 = x;
  const Tin* x2 = x + (int64_t)n * ms;
  double* y1 = y;
  double* y2 = y + (int64_t)n * ms;

  // unscaled M v and K v of time block j at this lane's point
  auto stencils = [&](const Tin* v, int j, double& mt, double& kt) {
    double q = 0.0, r = 0.0;
    if (has) fe_column<DIM>(v + (int64_t)j * ms + s, m, mm, e2m, e2p, e3m, e3p, q, r);
    const double ql = __shfl_up_sync(kFull, q, 1), qr = __shfl_down_sync(kFull, q, 1);
    const double rl = __shfl_up_sync(kFull, r, 1), rr = __shfl_down_sync(kFull, r, 1);
    const double sq = ql + qr;
    mt = fma(4.0, q, sq);
    kt = fma(4.0, r, rl + rr) + fma(2.0, q, -sq);
  };
  auto mass = [&](const Tin* v, int j) -> double {
    double q = 0.0, r = 0.0;
    if (has) fe_column<DIM>(v + (int64_t)j * ms + s, m, mm, e2m, e2p, e3m, e3p, q, r);
    const double ql = __shfl_up_sync(kFull, q, 1), qr = __shfl_down_sync(kFull, q, 1);
    return fma(4.0, q, ql + qr);
  };

  // y1_j = wM (alpha m1_j + sg (m2_j - m2_{j+1})) + sg tKw k2_j
  // y2_j = wM (alpha m2_j - sg (m1_j - m1_{j-1})) - sg tKw k1_j,   sg = -1 for A^T
  const double sg = TRANSPOSE ? -1.0 : 1.0;
  double m1p = j0 > 0 ? mass(x1, j0 - 1) : 0.0;
  double pm = 0.0, pk = 0.0;  // alpha m1 + sg m2 and k2 of the previous time block
  for (int j = j0; j < j1; ++j) {
    double m1, k1, m2, k2;
    stencils(x1, j, m1, k1);
    stencils(x2, j, m2, k2);
    const int64_t idx = (int64_t)j * ms + s;
    if (out) {
      if (j > j0) y1[idx - ms] = fma(wM, fma(-sg, m2, pm), sg * tKw * pk);
      y2[idx] = fma(wM, fma(alpha, m2, -sg * (m1 - m1p)), -sg * tKw * k1);
    }
    pm = fma(alpha, m1, sg * m2);
    pk = k2;
    m1p = m1;
  }
  const double m2n = j1 < n ? mass(x2, j1) : 0.0;
  if (out) y1[(int64_t)(j1 - 1) * ms + s] = fma(wM, fma(-sg, m2n, pm), sg * tKw * pk);
}

// ---------------------------------------------------------------------------
// The same product for an FP32 input z (the flexible-GMRES basis) in double-float
// arithmetic on the FP32 units: every quantity is an unevaluated sum hi + lo of two
// floats.  The stencil weights are small integers, so the column and row sums are
// exact TwoSum chains of scaled inputs; the FP64 scale factors (alpha, wM, tau wK)
// are split into float pairs and multiplied with an FMA error term.  Sums are not
// renormalised: every rounding error lands in `lo`, whose own rounding is then of
// order 2^-48 of the terms, and only the final hi + lo becomes an FP64 value.
// GB300's FP64 unit bounds the FP64 kernel above; this one runs on the FP32 pipes.
//
// The x1 direction uses D = 6 I - S:  with q the column sums as above and u the
// cross sums u = (I(x)S + S(x)I) v in the x2-x3 plane (2D: u = v),
//   M v / wM = S1 q,   K v / wK = 6 (q + S1 u) - dim S1 q.
struct DF {
  float hi, lo;
};

// a + b = s + err exactly (Knuth); the _rn intrinsics keep each operation separately
// rounded (no FMA contraction, which would break the exactness)
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return DF{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ DF df_scale2(DF a, float p2) { return DF{a.hi * p2, a.lo * p2}; }  // exact: p2 = 2^k
// c * v for a split FP64 constant c
__device__ __forceinline__ DF df_mul(DF c, DF v) {
  const float p = __fmul_rn(c.hi, v.hi);
  return DF{p, __fadd_rn(fmaf(c.hi, v.hi, -p), __fadd_rn(__fmul_rn(c.hi, v.lo), __fmul_rn(c.lo, v.hi)))};
}
__device__ __forceinline__ double df_to_f64(DF a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }
__device__ __forceinline__ DF df_shfl_up(DF a) {
  return DF{__shfl_up_sync(kFull, a.hi, 1), __shfl_up_sync(kFull, a.lo, 1)};
}
__device__ __forceinline__ DF df_shfl_down(DF a) {
  return DF{__shfl_down_sync(kFull, a.hi, 1), __shfl_down_sync(kFull, a.lo, 1)};
}
// a + b + 4 c from exact floats (S applied to a neighbour pair and a centre)
__device__ __forceinline__ DF s_sum(float a, float b, float c) {
  const DF t = two_sum(a, b);
  const DF q = two_sum(t.hi, 4.0f * c);
  return DF{q.hi, __fadd_rn(q.lo, t.lo)};
}

// column sums at p: q = S(x)S[..] v, and (3D) u = (I(x)S + S(x)I) v; 2D returns u = v
template <int DIM>
__device__ __forceinline__ void fe_column_df(const float* __restrict__ p, int64_t m, int64_t mm, bool e2m, bool e2p,
                                             bool e3m, bool e3p, DF& q, DF& u) {
  const float x0 = p[0];
  const float xs = e2m ? p[-m] : 0.0f, xn = e2p ? p[m] : 0.0f;
  if (DIM == 2) {
    q = s_sum(xs, xn, x0);
    u = DF{x0, 0.0f};
  } else {
    const float xb = e3m ? p[-mm] : 0.0f, xt = e3p ? p[mm] : 0.0f;
    const float c1 = e2m && e3m ? p[-m - mm] : 0.0f, c2 = e2p && e3m ? p[m - mm] : 0.0f;
    const float c3 = e2m && e3p ? p[-m + mm] : 0.0f, c4 = e2p && e3p ? p[m + mm] : 0.0f;
    const DF e = df_add(two_sum(xs, xn), two_sum(xb, xt));   // edges
    const DF c = df_add(two_sum(c1, c2), two_sum(c3, c4));   // corners
    q = df_add(df_add(DF{16.0f * x0, 0.0f}, df_scale2(e, 4.0f)), c);  // 16 x0 + 4 e + c
    u = df_add(e, DF{8.0f * x0, 0.0f});                            // 8 x0 + e
  }
}

template <int DIM>
__global__ void __launch_bounds__(256) matvec_fe_df_kernel(const float* __restrict__ x, double* __restrict__ y, int m,
                                                           int64_t ms, int64_t rows, int segs, int n, int tj,
                                                           DF alpha, DF wM, DF tKw, size_t xstride, size_t ystride,
                                                           const int* __restrict__ jdev) {
  if (jdev) {
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int lane = threadIdx.x & 31;
  const int seg = (int)(blockIdx.x % (unsigned)segs);
  const int64_t row = (int64_t)(blockIdx.x / (unsigned)segs) * kFeRowsPerCta + (threadIdx.x >> 5);
  if (row >= rows) return;  // whole warps leave together
  const int j0 = blockIdx.y * tj;
  const int j1 = min(n, j0 + tj);
  const int i1 = seg * kFeOut - 1 + lane;
  const bool has = i1 >= 0 && i1 < m;
  const bool out = has && lane >= 1 && lane <= kFeOut;
  const int i2 = (int)(DIM == 2 ? row : row % m);
  const int i3 = (int)(DIM == 3 ? row / m : 0);
  const bool e2m = i2 > 0, e2p = i2 < m - 1;
  const bool e3m = DIM == 3 && i3 > 0, e3p = DIM == 3 && i3 < m - 1;
  const int64_t mm = (int64_t)m * m;
  const int64_t s = row * m + (has ? i1 : 0);
  const float* x1 = x;
  const float* x2 = x + (int64_t)n * ms;
  double* y1 = y;
  double* y2 = y + (int64_t)n * ms;
  const DF zero{0.0f, 0.0f};

  // unscaled M v (mt) and K v (kt) of time block j
  auto stencils = [&](const float* v, int j, DF& mt, DF& kt) {
    DF q = zero, u = zero;
    if (has) fe_column_df<DIM>(v + (int64_t)j * ms + s, m, mm, e2m, e2p, e3m, e3p, q, u);
    mt = df_add(df_add(df_shfl_up(q), df_shfl_down(q)), df_scale2(q, 4.0f));  // S1 q
    DF su;                                                                   // S1 u
    if (DIM == 2) {
      su = s_sum(__shfl_up_sync(kFull, u.hi, 1), __shfl_down_sync(kFull, u.hi, 1), u.hi);
    } else {
      su = df_add(df_add(df_shfl_up(u), df_shfl_down(u)), df_scale2(u, 4.0f));
    }
    const DF w = df_add(q, su);
    // 6 w - DIM mt = 4 w + 2 w - 2 mt (- mt in 3D)
    DF k = df_sub(df_add(df_scale2(w, 4.0f), df_scale2(w, 2.0f)), df_scale2(mt, 2.0f));
    if (DIM == 3) k = df_sub(k, mt);
    kt = k;
  };
  auto mass = [&](const float* v, int j) -> DF {
    DF q = zero, u = zero;
    if (has) fe_column_df<DIM>(v + (int64_t)j * ms + s, m, mm, e2m, e2p, e3m, e3p, q, u);
    return df_add(df_add(df_shfl_up(q), df_shfl_down(q)), df_scale2(q, 4.0f));
  };

  // y1_j = wM (alpha m1_j + m2_j - m2_{j+1}) + tKw k2_j,  y2_j = wM (alpha m2_j - m1_j + m1_{j-1}) - tKw k1_j
  DF m1p = j0 > 0 ? mass(x1, j0 - 1) : zero;
  DF pm = zero, pk = zero;  // alpha m1 + m2 and tKw k2 of the previous time block
  for (int j = j0; j < j1; ++j) {
    DF m1, k1, m2, k2;
    stencils(x1, j, m1, k1);
    stencils(x2, j, m2, k2);
    const int64_t idx = (int64_t)j * ms + s;
    if (out) {
      if (j > j0) y1[idx - ms] = df_to_f64(df_add(df_mul(wM, df_sub(pm, m2)), pk));
      const DF t = df_add(df_mul(alpha, m2), df_sub(m1p, m1));
      y2[idx] = df_to_f64(df_sub(df_mul(wM, t), df_mul(tKw, k1)));
    }
    pm = df_add(df_mul(alpha, m1), m2);
    pk = df_mul(tKw, k2);
    m1p = m1;
  }
  const DF m2n = j1 < n ? mass(x2, j1) : zero;
  if (out) y1[(int64_t)(j1 - 1) * ms + s] = df_to_f64(df_add(df_mul(wM, df_sub(pm, m2n)), pk));
}

// out_p = cM (S(x)S..) in_p + cK (K stencil) in_p + beta out_p for every plane p
// (mass / stiffness products of single fields: right-hand side, end-point solves)
template <int DIM>
__global__ void __launch_bounds__(256) fe_apply_kernel(const double* __restrict__ in, double* __restrict__ outp,
                                                       int m, int64_t ms, int planes, double cM, double cK,
                                                       double beta) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ms * planes) return;
  const int64_t p = e / ms;
  const int64_t s = e - p * ms;
  const int i1 = (int)(s % m);
  const int64_t row = s / m;
  const int i2 = (int)(DIM == 2 ? row : row % m);
  const int i3 = (int)(DIM == 3 ? row / m : 0);
  const bool e2m = i2 > 0, e2p = i2 < m - 1;
  const bool e3m = DIM == 3 && i3 > 0, e3p = DIM == 3 && i3 < m - 1;
  const int64_t mm = (int64_t)m * m;
  const double* c = in + e;
  double q0, r0, ql = 0.0, rl = 0.0, qr = 0.0, rr = 0.0;
  fe_column<DIM>(c, m, mm, e2m, e2p, e3m, e3p, q0, r0);
  if (i1 > 0) fe_column<DIM>(c - 1, m, mm, e2m, e2p, e3m, e3p, ql, rl);
  if (i1 < m - 1) fe_column<DIM>(c + 1, m, mm, e2m, e2p, e3m, e3p, qr, rr);
  const double sq = ql + qr;
  const double mt = fma(4.0, q0, sq);
  const double kt = fma(4.0, r0, rl + rr) + fma(2.0, q0, -sq);
  double v = fma(cM, mt, cK * kt);
  if (beta != 0.0) v = fma(beta, outp[e], v);
  outp[e] = v;
}

}  // namespace

FeScale fe_scale(int dim, int m1, double c) {
  const double h = 1.0 / (m1 + 1);
  const double h6 = h / 6.0;
  FeScale f;
  f.wM = dim == 2 ? h6 * h6 : h6 * h6 * h6;
  f.wK = c * (dim == 2 ? h6 : h6 * h6) / h;
  return f;
}

template <typename Tin>
cudaError_t launch_matvec_fe(Launch& L, const Grid& g, int n, double alpha, FeScale fs, double tau, const Tin* x,
                             double* y, bool transpose, size_t xstride, size_t ystride, const int* jdev) {
  const int64_t rows = g.dim == 2 ? (int64_t)g.m : (int64_t)g.m * g.m;
  const int segs = (g.m + kFeOut - 1) / kFeOut;
  int tj = L.tiles && L.tiles->mv_tj > 0 ? L.tiles->mv_tj : 32;  // time blocks per thread
  tj = tj < n ? tj : n;
  dim3 grid((unsigned)(segs * ((rows + kFeRowsPerCta - 1) / kFeRowsPerCta)), (unsigned)((n + tj - 1) / tj));
  const double pts = (double)n * (double)g.np;
  const double bytes = 2.0 * pts * (sizeof(Tin) + sizeof(double));
  // per point and time block: two vectors' column sums and x1 stencils, two outputs
  const double flops = pts * (g.dim == 2 ? 48.0 : 64.0);
  const double tKw = tau * fs.wK;
  L.begin(KC_MATVEC);
  if constexpr (std::is_same<Tin, float>::value) {
    if (!transpose) {  // the flexible-GMRES product: double-float on the FP32 units
      auto split = [](double v) {
        const float hi = (float)v;
        return DF{hi, (float)(v - (double)hi)};
      };
      if (g.dim == 2)
        matvec_fe_df_kernel<2><<<grid, 256, 0, L.stream>>>(x, y, g.m, g.np, rows, segs, n, tj, split(alpha),
                                                           split(fs.wM), split(tKw), xstride, ystride, jdev);
      else
        matvec_fe_df_kernel<3><<<grid, 256, 0, L.stream>>>(x, y, g.m, g.np, rows, segs, n, tj, split(alpha),
                                                           split(fs.wM), split(tKw), xstride, ystride, jdev);
      return L.end(KC_MATVEC, jdev ? 0.0 : bytes, jdev ? 0.0 : flops);
    }
  }
#define PCOPT_FE_MV(D, TR)                                                                                    \
  matvec_fe_kernel<Tin, D, TR><<<grid, 256, 0, L.stream>>>(x, y, g.m, g.np, rows, segs, n, tj, alpha, fs.wM, \
                                                           tKw, xstride, ystride, jdev)
  if (g.dim == 2) {
    if (transpose) PCOPT_FE_MV(2, true);
    else PCOPT_FE_MV(2, false);
  } else {
    if (transpose) PCOPT_FE_MV(3, true);
    else PCOPT_FE_MV(3, false);
  }
#undef PCOPT_FE_MV
  return L.end(KC_MATVEC, jdev ? 0.0 : bytes, jdev ? 0.0 : flops);
}

template cudaError_t launch_matvec_fe<double>(Launch&, const Grid&, int, double, FeScale, double, const double*,
                                              double*, bool, size_t, size_t, const int*);
template cudaError_t launch_matvec_fe<float>(Launch&, const Grid&, int, double, FeScale, double, const float*, double*,
                                             bool, size_t, size_t, const int*);

cudaError_t launch_fe_apply(Launch& L, const Grid& g, int planes, double cM, double cK, const double* in, double beta,
                            double* out) {
  const int64_t tot = g.np * planes;
  if (tot == 0) return cudaSuccess;
  L.begin(KC_FE_APPLY);
  if (g.dim == 2)
    fe_apply_kernel<2><<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(in, out, g.m, g.np, planes, cM, cK, beta);
  else
    fe_apply_kernel<3><<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(in, out, g.m, g.np, planes, cM, cK, beta);
  return L.end(KC_FE_APPLY, (double)tot * (beta != 0.0 ? 24.0 : 16.0), (double)tot * (g.dim == 2 ? 30.0 : 70.0));
}

}  // namespace pcopt
