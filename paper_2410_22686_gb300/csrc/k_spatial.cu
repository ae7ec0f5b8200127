// Step 2 of the four-step apply of P_eps^{-1} (Section 2.1): for every
// spectral plane p (frequency k = p/2, shift sigma_p = lambda_k + alpha) solve
//     (sigma_p I + tau K) u_p = r_p
// either exactly by sine transforms (constant a, Example 1) or approximately
// by one V(1,0) multigrid cycle (variable a, Example 2: Gauss-Seidel
// pre-smoother, no post-smoother).  The multigrid reading: one red-black
// Gauss-Seidel sweep from zero (red = even sum of 1-based indices, first),
// full-weighting restriction, (bi/tri)linear prolongation, rediscretised
// coarse operators with the nodal coefficient injected, the same shift on
// every level, exact solve on the one-point level.
//
// Threads own one spatial point and loop over a chunk of planes, so the
// point's face weights and diagonal are read once and reused for every shift.
#include "common.cuh"

namespace pcopt {

namespace {

constexpr int kPlaneChunk = 8;

template <typename Tc>
__device__ __forceinline__ typename Cx<Tc>::t inv_diag(typename Cx<Tc>::t sig, Tc dg) {
  return cinv(cmk<Tc>(sig.x + dg, sig.y));
}

struct Coord {
  int i1, i2, i3;
};
__device__ __forceinline__ Coord coord_of(int64_t s, int m, int dim) {
  Coord c;
  c.i1 = (int)(s % m);
  int64_t r = s / m;
  if (dim == 2) {
    c.i2 = (int)r;
    c.i3 = 0;
  } else {
    c.i2 = (int)(r % m);
    c.i3 = (int)(r / m);
  }
  return c;
}

// ------------------------------------------------------------------- FST
template <typename Tc>
__global__ void fst_axis_kernel(const typename Cx<Tc>::t* __restrict__ in, typename Cx<Tc>::t* __restrict__ out,
                                const Tc* __restrict__ S, int m, int dim, int axis, int64_t np, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * planes) return;
  const int64_t p = e / np;
  const int64_t s = e - p * np;
  const Coord c = coord_of(s, m, dim);
  const int i = axis == 0 ? c.i1 : (axis == 1 ? c.i2 : c.i3);
  int64_t stride = 1;
  for (int a = 0; a < axis; ++a) stride *= m;
  const C* src = in + p * np + (s - (int64_t)i * stride);
  Tc ar = 0, ai = 0;
  for (int j = 0; j < m; ++j) {
    const Tc sij = S[i * m + j];
    const C v = src[(int64_t)j * stride];
    ar = fma(sij, v.x, ar);
    ai = fma(sij, v.y, ai);
  }
  out[e] = cmk<Tc>(ar, ai);
}

template <typename Tc>
__global__ void fst_divide_kernel(typename Cx<Tc>::t* __restrict__ buf, const Tc* __restrict__ lamK,
                                  const typename Cx<Tc>::t* __restrict__ sigma, int64_t np, int planes) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * planes) return;
  const int64_t p = e / np;
  const int64_t s = e - p * np;
  buf[e] = cmul(buf[e], inv_diag<Tc>(sigma[p], lamK[s]));
}

// ------------------------------------------------------------------- multigrid
// One red-black Gauss-Seidel sweep from u = 0, fused: a red point takes
// r/d; a black point takes (r + sum_k w_k u_red(nb_k))/d, where the red
// neighbour values are recomputed from r on the fly.
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_smooth_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                        TU* __restrict__ u,
                                                        const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                        const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                        int64_t np, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  const int p0 = blockIdx.y * kPlaneChunk;
  const int p1 = min(planes, p0 + kPlaneChunk);
  const Coord c = coord_of(s, m, DIM);
  const bool red = ((c.i1 + c.i2 + c.i3 + DIM) & 1) == 0;
  const Tc dg = diag[s];
  if (red) {
    for (int p = p0; p < p1; ++p) {
      const int64_t o = (int64_t)p * np + s;
      stc(u, o, cmul(r[o], inv_diag<Tc>(sigma[p], dg)));
    }
    return;
  }
  int64_t off[2 * DIM];
  bool ex[2 * DIM];
  Tc wv[2 * DIM], dn[2 * DIM];
  const int64_t mm = (int64_t)m * m;
  off[0] = -1;
  ex[0] = c.i1 > 0;
  off[1] = 1;
  ex[1] = c.i1 < m - 1;
  off[2] = -(int64_t)m;
  ex[2] = c.i2 > 0;
  off[3] = m;
  ex[3] = c.i2 < m - 1;
  if (DIM == 3) {
    off[4] = -mm;
    ex[4] = c.i3 > 0;
    off[5] = mm;
    ex[5] = c.i3 < m - 1;
  }
#pragma unroll
  for (int k = 0; k < 2 * DIM; ++k) {
    wv[k] = w[(int64_t)k * np + s];
    dn[k] = ex[k] ? diag[s + off[k]] : Tc(0);
  }
  for (int p = p0; p < p1; ++p) {
    const int64_t o = (int64_t)p * np + s;
    const C sig = sigma[p];
    C acc = r[o];
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k) {
      if (ex[k]) {
        const C ured = cmul(r[o + off[k]], inv_diag<Tc>(sig, dn[k]));
        acc.x = fma(wv[k], ured.x, acc.x);
        acc.y = fma(wv[k], ured.y, acc.y);
      }
    }
    stc(u, o, cmul(acc, inv_diag<Tc>(sig, dg)));
  }
}

// res = r - (sigma u + tau K u)
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_residual_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                          const TU* __restrict__ u,
                                                          typename Cx<Tc>::t* __restrict__ res,
                                                          const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                          const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                          int64_t np, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  const int p0 = blockIdx.y * kPlaneChunk;
  const int p1 = min(planes, p0 + kPlaneChunk);
  const Coord c = coord_of(s, m, DIM);
  int64_t off[2 * DIM];
  bool ex[2 * DIM];
  Tc wv[2 * DIM];
  const int64_t mm = (int64_t)m * m;
  off[0] = -1;
  ex[0] = c.i1 > 0;
  off[1] = 1;
  ex[1] = c.i1 < m - 1;
  off[2] = -(int64_t)m;
  ex[2] = c.i2 > 0;
  off[3] = m;
  ex[3] = c.i2 < m - 1;
  if (DIM == 3) {
    off[4] = -mm;
    ex[4] = c.i3 > 0;
    off[5] = mm;
    ex[5] = c.i3 < m - 1;
  }
#pragma unroll
  for (int k = 0; k < 2 * DIM; ++k) wv[k] = w[(int64_t)k * np + s];
  const Tc dg = diag[s];
  for (int p = p0; p < p1; ++p) {
    const int64_t o = (int64_t)p * np + s;
    const C sig = sigma[p];
    const C uc = ldc(u, o);
    // L u = (sigma + dg) u - sum_k w_k u_nb
    C lu = cmul(cmk<Tc>(sig.x + dg, sig.y), uc);
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k) {
      if (ex[k]) {
        const C un = ldc(u, o + off[k]);
        lu.x = fma(-wv[k], un.x, lu.x);
        lu.y = fma(-wv[k], un.y, lu.y);
      }
    }
    res[o] = r[o] - lu;
  }
}

// full weighting: coarse point I (1-based) on fine point 2I, weights prod_k w(o_k),
// w(0) = 1/2, w(+-1) = 1/4
template <typename Tc, int DIM>
__global__ void __launch_bounds__(256) mg_restrict_kernel(const typename Cx<Tc>::t* __restrict__ res,
                                                          typename Cx<Tc>::t* __restrict__ rc, int mf, int mc,
                                                          int64_t npf, int64_t npc, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t sc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sc >= npc) return;
  const int p0 = blockIdx.y * kPlaneChunk;
  const int p1 = min(planes, p0 + kPlaneChunk);
  const Coord c = coord_of(sc, mc, DIM);
  // 0-based fine centre of coarse (0-based) c is 2c+1
  const int f1 = 2 * c.i1 + 1, f2 = 2 * c.i2 + 1, f3 = 2 * c.i3 + 1;
  const Tc wt[3] = {Tc(0.25), Tc(0.5), Tc(0.25)};
  for (int p = p0; p < p1; ++p) {
    const C* rp = res + (int64_t)p * npf;
    C acc = czero<Tc>();
    for (int o3 = (DIM == 3 ? -1 : 0); o3 <= (DIM == 3 ? 1 : 0); ++o3) {
      for (int o2 = -1; o2 <= 1; ++o2) {
        for (int o1 = -1; o1 <= 1; ++o1) {
          Tc wgt = wt[o1 + 1] * wt[o2 + 1];
          if (DIM == 3) wgt *= wt[o3 + 1];
          const int64_t q = (DIM == 3 ? ((int64_t)(f3 + o3) * mf + (f2 + o2)) * mf : (int64_t)(f2 + o2) * mf) + (f1 + o1);
          const C v = rp[q];
          acc.x = fma(wgt, v.x, acc.x);
          acc.y = fma(wgt, v.y, acc.y);
        }
      }
    }
    rc[(int64_t)p * npc + sc] = acc;
  }
}

// u_f += P e_c, P = tensor product of 1D linear interpolation
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_prolong_kernel(const TU* __restrict__ ec, TU* __restrict__ uf, int mf, int mc,
                                                         int64_t npf, int64_t npc, int planes) {
  typedef typename Cx<Tc>::t C;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= npf) return;
  const int p0 = blockIdx.y * kPlaneChunk;
  const int p1 = min(planes, p0 + kPlaneChunk);
  const Coord c = coord_of(s, mf, DIM);
  // per axis: up to two coarse indices with weights
  int ci[3][2];
  Tc cw[3][2];
  int cnt[3];
  const int fi[3] = {c.i1, c.i2, c.i3};
  for (int a = 0; a < DIM; ++a) {
    const int f = fi[a];
    if (f & 1) {
      ci[a][0] = (f - 1) >> 1;
      cw[a][0] = Tc(1);
      cnt[a] = 1;
    } else {
      cnt[a] = 0;
      const int lo = (f >> 1) - 1, hi = f >> 1;
      if (lo >= 0) {
        ci[a][cnt[a]] = lo;
        cw[a][cnt[a]] = Tc(0.5);
        cnt[a]++;
      }
      if (hi < mc) {
        ci[a][cnt[a]] = hi;
        cw[a][cnt[a]] = Tc(0.5);
        cnt[a]++;
      }
    }
  }
  if (DIM == 2) {
    cnt[2] = 1;
    ci[2][0] = 0;
    cw[2][0] = Tc(1);
  }
  for (int p = p0; p < p1; ++p) {
    const TU* ep = ec + (int64_t)p * npc;
    C acc = czero<Tc>();
    for (int a3 = 0; a3 < cnt[2]; ++a3)
      for (int a2 = 0; a2 < cnt[1]; ++a2)
        for (int a1 = 0; a1 < cnt[0]; ++a1) {
          const Tc wgt = cw[0][a1] * cw[1][a2] * cw[2][a3];
          const int64_t q = ((int64_t)ci[2][a3] * mc + ci[1][a2]) * mc + ci[0][a1];
          const C v = ldc(ep, q);
          acc.x = fma(wgt, v.x, acc.x);
          acc.y = fma(wgt, v.y, acc.y);
        }
    const int64_t o = (int64_t)p * npf + s;
    stc(uf, o, ldc(uf, o) + acc);
  }
}

template <typename Tc, typename TU>
__global__ void mg_coarsest_kernel(const Tc* __restrict__ diag, const typename Cx<Tc>::t* __restrict__ sigma,
                                   const typename Cx<Tc>::t* __restrict__ r, TU* __restrict__ u, int planes) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= planes) return;
  stc(u, p, cmul(r[p], inv_diag<Tc>(sigma[p], diag[0])));
}

dim3 plane_grid(int64_t np, int planes) {
  return dim3((unsigned)((np + 255) / 256), (unsigned)((planes + kPlaneChunk - 1) / kPlaneChunk));
}

}  // namespace

template <typename Tc>
cudaError_t launch_fst_axis(Launch& L, const Grid& g, int planes, int axis, const Tc* S,
                            const typename Cx<Tc>::t* in, typename Cx<Tc>::t* out) {
  const int64_t tot = g.np * planes;
  const double cs = sizeof(typename Cx<Tc>::t);
  L.begin(KC_FST_AXIS);
  fst_axis_kernel<Tc><<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(in, out, S, g.m, g.dim, axis, g.np, planes);
  return L.end(KC_FST_AXIS, 2.0 * tot * cs, 4.0 * tot * g.m);
}

template <typename Tc>
cudaError_t launch_fst_divide(Launch& L, const Grid& g, int planes, const Tc* lamK, const typename Cx<Tc>::t* sigma,
                              typename Cx<Tc>::t* buf) {
  const int64_t tot = g.np * planes;
  const double cs = sizeof(typename Cx<Tc>::t);
  L.begin(KC_FST_DIVIDE);
  fst_divide_kernel<Tc><<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(buf, lamK, sigma, g.np, planes);
  return L.end(KC_FST_DIVIDE, 2.0 * tot * cs, 12.0 * tot);
}

template <typename Tc, typename TU>
cudaError_t launch_mg_smooth(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                             const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u) {
  const double cs = 0.5 * (sizeof(typename Cx<Tc>::t) + sizeof(TU));
  const double tot = (double)g.np * planes;
  L.begin(KC_MG_SMOOTH);
  if (g.dim == 2)
    mg_smooth_kernel<Tc, TU, 2><<<plane_grid(g.np, planes), 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np,
                                                                            planes);
  else
    mg_smooth_kernel<Tc, TU, 3><<<plane_grid(g.np, planes), 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np,
                                                                            planes);
  return L.end(KC_MG_SMOOTH, 2.0 * tot * cs, tot * (12.0 + 10.0 * g.dim));
}

template <typename Tc, typename TU>
cudaError_t launch_mg_resid_restrict(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                                     const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, const TU* u,
                                     typename Cx<Tc>::t* res, typename Cx<Tc>::t* rc) {
  const double cs = sizeof(typename Cx<Tc>::t);
  const int mc = (g.m - 1) / 2;
  const int64_t npc = g.dim == 2 ? (int64_t)mc * mc : (int64_t)mc * mc * mc;
  const double tot = (double)g.np * planes;
  L.begin(KC_MG_RESID_RESTRICT);
  if (g.dim == 2)
    mg_residual_kernel<Tc, TU, 2><<<plane_grid(g.np, planes), 256, 0, L.stream>>>(r, u, res, st.w, st.diag, sigma, g.m,
                                                                              g.np, planes);
  else
    mg_residual_kernel<Tc, TU, 3><<<plane_grid(g.np, planes), 256, 0, L.stream>>>(r, u, res, st.w, st.diag, sigma, g.m,
                                                                              g.np, planes);
  cudaError_t e = L.end(KC_MG_RESID_RESTRICT, 3.0 * tot * cs, tot * (8.0 + 4.0 * g.dim));
  if (e != cudaSuccess) return e;
  L.begin(KC_MG_RESID_RESTRICT);
  if (g.dim == 2)
    mg_restrict_kernel<Tc, 2><<<plane_grid(npc, planes), 256, 0, L.stream>>>(res, rc, g.m, mc, g.np, npc, planes);
  else
    mg_restrict_kernel<Tc, 3><<<plane_grid(npc, planes), 256, 0, L.stream>>>(res, rc, g.m, mc, g.np, npc, planes);
  return L.end(KC_MG_RESID_RESTRICT, tot * cs + (double)npc * planes * cs, (double)npc * planes * (g.dim == 2 ? 36 : 108));
}

template <typename Tc, typename TU>
cudaError_t launch_mg_prolong(Launch& L, const Grid& gf, int planes, const TU* ec, TU* uf) {
  const double cs = sizeof(TU);
  const int mc = (gf.m - 1) / 2;
  const int64_t npc = gf.dim == 2 ? (int64_t)mc * mc : (int64_t)mc * mc * mc;
  const double tot = (double)gf.np * planes;
  L.begin(KC_MG_PROLONG);
  if (gf.dim == 2)
    mg_prolong_kernel<Tc, TU, 2><<<plane_grid(gf.np, planes), 256, 0, L.stream>>>(ec, uf, gf.m, mc, gf.np, npc, planes);
  else
    mg_prolong_kernel<Tc, TU, 3><<<plane_grid(gf.np, planes), 256, 0, L.stream>>>(ec, uf, gf.m, mc, gf.np, npc, planes);
  return L.end(KC_MG_PROLONG, 2.0 * tot * cs + (double)npc * planes * cs, tot * 8.0);
}

template <typename Tc, typename TU>
cudaError_t launch_mg_coarsest(Launch& L, int planes, const Tc* diag, const typename Cx<Tc>::t* sigma,
                               const typename Cx<Tc>::t* r, TU* u) {
  const double cs = sizeof(typename Cx<Tc>::t);
  L.begin(KC_MG_COARSEST);
  mg_coarsest_kernel<Tc, TU><<<(planes + 255) / 256, 256, 0, L.stream>>>(diag, sigma, r, u, planes);
  return L.end(KC_MG_COARSEST, 2.0 * planes * cs, 12.0 * planes);
}

#define PCOPT_INST_FST(Tc)                                                                                   \
  template cudaError_t launch_fst_axis<Tc>(Launch&, const Grid&, int, int, const Tc*, const Cx<Tc>::t*,          \
                                           Cx<Tc>::t*);                                                             \
  template cudaError_t launch_fst_divide<Tc>(Launch&, const Grid&, int, const Tc*, const Cx<Tc>::t*, Cx<Tc>::t*);
#define PCOPT_INST_MG(Tc, TU)                                                                                    \
  template cudaError_t launch_mg_smooth<Tc, TU>(Launch&, const Grid&, int, const Stencil<Tc>&, const Cx<Tc>::t*, \
                                                const Cx<Tc>::t*, TU*);                                             \
  template cudaError_t launch_mg_resid_restrict<Tc, TU>(Launch&, const Grid&, int, const Stencil<Tc>&,           \
                                                        const Cx<Tc>::t*, const Cx<Tc>::t*, const TU*, Cx<Tc>::t*, \
                                                        Cx<Tc>::t*);                                                \
  template cudaError_t launch_mg_prolong<Tc, TU>(Launch&, const Grid&, int, const TU*, TU*);                     \
  template cudaError_t launch_mg_coarsest<Tc, TU>(Launch&, int, const Tc*, const Cx<Tc>::t*, const Cx<Tc>::t*,   \
                                                  TU*);
PCOPT_INST_FST(float)
PCOPT_INST_FST(double)
PCOPT_INST_MG(float, float2)
PCOPT_INST_MG(double, double2)
PCOPT_INST_MG(float, __nv_bfloat162)
#undef PCOPT_INST_FST
#undef PCOPT_INST_MG

}  // namespace pcopt
