// Down leg of one multigrid level of the V(1,0) cycle (Section 2.1, step 2 of the
// apply of P_eps^{-1}, variable a) in one launch for 2D grids:
//
//   red-black Gauss-Seidel sweep from u = 0 on (sigma_p I + tau K) u = r,
//   residual  res = r - (sigma_p I + tau K) u,
//   full weighting  rc(I, J) = sum_{o1,o2 in -1..1} w(o1) w(o2) res(2I+1+o1, 2J+1+o2),
//   w(0) = 1/2, w(+-1) = 1/4,
//
// with the same arithmetic as the per-level kernels of k_spatial.cu, but r is read
// from HBM once and the residual never goes there: a CTA owns a CX x CX tile of
// coarse points (the fine points 2I, 2I+1 of each, the last tile also the fine
// point m-1), stages r on the fine window [2I0-2, 2I0+2CX+2]^2 in shared memory,
// takes red u on all of it, black u on [2I0-1, 2I0+2CX+1]^2 and the residual on
// [2I0, 2I0+2CX]^2, then restricts.  The face weights and diagonal of the window
// stay in shared memory for all the CTA's planes.  Points outside the grid hold
// r = u = 0 (homogeneous Dirichlet boundary).  Red = even i1 + i2 (0-based),
// swept first.  Values of u are rounded to the storage type TU before any later
// step reads them, so the BF16-storage variant smooths, takes residuals and is
// corrected on exactly what it stores.
#include "common.cuh"

namespace pcopt {

namespace {

template <typename TU, typename C>
__device__ __forceinline__ C stored(C v) {
  if constexpr (std::is_same<TU, __nv_bfloat162>::value) {
    return __bfloat1622float2(__float22bfloat162_rn(v));
  } else {
    return v;
  }
}

// 1 / z; in FP32 with the hardware-approximate divide (2 ulp, far inside what a
// smoother needs)
__device__ __forceinline__ float2 inv_shift(float2 z) {
  const float q = __fdividef(1.0f, fmaf(z.x, z.x, z.y * z.y));
  return make_float2(z.x * q, -z.y * q);
}
__device__ __forceinline__ double2 inv_shift(double2 z) { return cinv(z); }

template <typename Tc, typename TU, int CX>
__global__ void __launch_bounds__(256) mg_down2_kernel(const typename Cx<Tc>::t* __restrict__ r, TU* __restrict__ u,
                                                       typename Cx<Tc>::t* __restrict__ rc,
                                                       const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                       const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                       int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  constexpr int NT = 256;
  constexpr int WR = 2 * CX + 5;  // r window per axis
  constexpr int NW = WR * WR;
  constexpr int NB = WR - 2;      // black range [1, WR-2]
  constexpr int NPR = (NB + 1) / 2;
  constexpr int NRS = WR - 4;     // residual range [2, WR-3]
  constexpr int NPC = (NRS + 1) / 2;
  constexpr int SA = (NW + NT - 1) / NT;         // window slots per thread
  constexpr int SB = (NB * NPR + NT - 1) / NT;   // black slots
  constexpr int SC = (NRS * NPC + NT - 1) / NT;  // red residual slots
  // Residual of a sweep from zero: black points are solved exactly against their
  // red neighbours and red points against zero, so res_black = 0 and
  // res_red = sum_k w_k u_black(nb_k).  With BF16 storage the stored u no longer
  // satisfies this and the residual is formed explicitly from it.
  constexpr bool EXPLICIT = std::is_same<TU, __nv_bfloat162>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sR = reinterpret_cast<C*>(smem_raw);
  C* sU = sR + NW;
  Tc* sD = reinterpret_cast<Tc*>(sU + NW);
  Tc* sW = sD + NW;  // [4][NW]: faces -x, +x, -y, +y

  const int mc = (m - 1) / 2;
  const int64_t np = (int64_t)m * m;
  const int64_t npc = (int64_t)mc * mc;
  const int I0 = blockIdx.x * CX, J0 = blockIdx.y * CX;
  const int fx = 2 * I0 - 2, fy = 2 * J0 - 2;  // fine coordinates of window cell (0, 0)
  const int p0 = blockIdx.z * pch;
  const int p1 = min(planes, p0 + pch);
  // owned fine points: local [2, ex) x [2, ey)
  const int ex = (I0 + CX >= mc ? m : 2 * (I0 + CX)) - fx;
  const int ey = (J0 + CX >= mc ? m : 2 * (J0 + CX)) - fy;
  const int tid = threadIdx.x;

  // per-thread slots, the same for every plane: in-plane offset (-1 outside),
  // colour and ownership of the window cells; shared-memory index of the black
  // and red-residual points
  int goffA[SA];
  unsigned redA = 0, ownA = 0;
#pragma unroll
  for (int i = 0; i < SA; ++i) {
    const int e = tid + i * NT;
    const int a1 = e % WR, a2 = e / WR;
    const int f1 = fx + a1, f2 = fy + a2;
    const bool in = e < NW && f1 >= 0 && f1 < m && f2 >= 0 && f2 < m;
    goffA[i] = in ? f2 * m + f1 : -1;
    if (((f1 + f2) & 1) == 0) redA |= 1u << i;
    if (in && a1 >= 2 && a1 < ex && a2 >= 2 && a2 < ey) ownA |= 1u << i;
    if (e < NW) {
      sD[e] = in ? diag[goffA[i]] : Tc(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) sW[k * NW + e] = in ? w[(int64_t)k * np + goffA[i]] : Tc(0);
      sR[e] = czero<Tc>();
      sU[e] = czero<Tc>();
    }
  }
  int qB[SB];
  unsigned ownB = 0;
#pragma unroll
  for (int i = 0; i < SB; ++i) {
    const int e = tid + i * NT;
    const int a2 = 1 + e / NPR;
    int a1 = 1 + 2 * (e % NPR);
    if (((fx + a1 + fy + a2) & 1) == 0) ++a1;
    const int f1 = fx + a1, f2 = fy + a2;
    const bool ok = e < NB * NPR && a1 <= WR - 2 && f1 >= 0 && f1 < m && f2 >= 0 && f2 < m;
    qB[i] = ok ? a2 * WR + a1 : -1;
    if (ok && a1 >= 2 && a1 < ex && a2 >= 2 && a2 < ey) ownB |= 1u << i;
  }
  int qC[SC];
#pragma unroll
  for (int i = 0; i < SC; ++i) {
    const int e = tid + i * NT;
    const int a2 = 2 + e / NPC;
    int a1 = 2 + 2 * (e % NPC);
    if ((fx + a1 + fy + a2) & 1) ++a1;  // the red one of the pair
    const bool ok = e < NRS * NPC && a1 <= WR - 3 && fx + a1 < m && fy + a2 < m;
    qC[i] = ok ? a2 * WR + a1 : -1;
  }

  C pre[SA];
  auto fetch = [&](int p) {
    const C* rp = r + (int64_t)p * np;
#pragma unroll
    for (int i = 0; i < SA; ++i) pre[i] = goffA[i] >= 0 ? rp[goffA[i]] : czero<Tc>();
  };
  if (p0 < p1) fetch(p0);
  __syncthreads();

  for (int p = p0; p < p1; ++p) {
    const C sig = sigma[p];
    TU* up = u + (int64_t)p * np;
    // stage r; red points take u = r / (sigma + d)
#pragma unroll
    for (int i = 0; i < SA; ++i) {
      if (goffA[i] < 0) continue;
      const int e = tid + i * NT;
      sR[e] = pre[i];
      if (redA & (1u << i)) {
        const C uv = stored<TU>(cmul(pre[i], inv_shift(cmk<Tc>(sig.x + sD[e], sig.y))));
        sU[e] = uv;
        if (ownA & (1u << i)) stc(up, goffA[i], uv);
      }
    }
    __syncthreads();
    if (p + 1 < p1) fetch(p + 1);  // the next plane's window is in flight meanwhile
    // black points: u = (r + sum_k w_k u_red(nb_k)) / (sigma + d)
#pragma unroll
    for (int i = 0; i < SB; ++i) {
      const int q = qB[i];
      if (q < 0) continue;
      C acc = sR[q];
      const C ul = sU[q - 1], ur = sU[q + 1], ud = sU[q - WR], uu = sU[q + WR];
      const Tc w0 = sW[q], w1 = sW[NW + q], w2 = sW[2 * NW + q], w3 = sW[3 * NW + q];
      acc.x = fma(w0, ul.x, acc.x);
      acc.y = fma(w0, ul.y, acc.y);
      acc.x = fma(w1, ur.x, acc.x);
      acc.y = fma(w1, ur.y, acc.y);
      acc.x = fma(w2, ud.x, acc.x);
      acc.y = fma(w2, ud.y, acc.y);
      acc.x = fma(w3, uu.x, acc.x);
      acc.y = fma(w3, uu.y, acc.y);
      const C uv = stored<TU>(cmul(acc, inv_shift(cmk<Tc>(sig.x + sD[q], sig.y))));
      sU[q] = uv;
      if (ownB & (1u << i)) stc(up, (int64_t)(fy + q / WR) * m + fx + q % WR, uv);
    }
    __syncthreads();
    if constexpr (!EXPLICIT) {
      // red residuals, in place of r
#pragma unroll
      for (int i = 0; i < SC; ++i) {
        const int q = qC[i];
        if (q < 0) continue;
        const C ul = sU[q - 1], ur = sU[q + 1], ud = sU[q - WR], uu = sU[q + WR];
        const Tc w0 = sW[q], w1 = sW[NW + q], w2 = sW[2 * NW + q], w3 = sW[3 * NW + q];
        C res;
        res.x = w0 * ul.x;
        res.y = w0 * ul.y;
        res.x = fma(w1, ur.x, res.x);
        res.y = fma(w1, ur.y, res.y);
        res.x = fma(w2, ud.x, res.x);
        res.y = fma(w2, ud.y, res.y);
        res.x = fma(w3, uu.x, res.x);
        res.y = fma(w3, uu.y, res.y);
        sR[q] = res;
      }
    } else {
      // residual of the stored u at every point of the restriction windows
      for (int e = tid; e < NRS * NRS; e += NT) {
        const int a1 = 2 + e % NRS, a2 = 2 + e / NRS;
        if (fx + a1 >= m || fy + a2 >= m) continue;
        const int q = a2 * WR + a1;
        const C uc = sU[q];
        C lu = cmul(cmk<Tc>(sig.x + sD[q], sig.y), uc);
        const C ul = sU[q - 1], ur = sU[q + 1], ud = sU[q - WR], uu = sU[q + WR];
        const Tc w0 = sW[q], w1 = sW[NW + q], w2 = sW[2 * NW + q], w3 = sW[3 * NW + q];
        lu.x = fma(-w0, ul.x, lu.x);
        lu.y = fma(-w0, ul.y, lu.y);
        lu.x = fma(-w1, ur.x, lu.x);
        lu.y = fma(-w1, ur.y, lu.y);
        lu.x = fma(-w2, ud.x, lu.x);
        lu.y = fma(-w2, ud.y, lu.y);
        lu.x = fma(-w3, uu.x, lu.x);
        lu.y = fma(-w3, uu.y, lu.y);
        sR[q] = sR[q] - lu;
      }
    }
    __syncthreads();
    // full weighting onto the coarse tile; the edge points of each 3x3 window are
    // black (zero residual unless it was formed explicitly)
    for (int e = tid; e < CX * CX; e += NT) {
      const int I = I0 + e % CX, J = J0 + e / CX;
      if (I >= mc || J >= mc) continue;
      const int q = (2 * (J - J0) + 3) * WR + 2 * (I - I0) + 3;
      const C c0 = sR[q];
      const C k4 = sR[q - WR - 1] + sR[q - WR + 1] + sR[q + WR - 1] + sR[q + WR + 1];
      C acc;
      if constexpr (EXPLICIT) {
        const C e4 = sR[q - 1] + sR[q + 1] + sR[q - WR] + sR[q + WR];
        acc.x = fma(Tc(0.25), c0.x, fma(Tc(0.125), e4.x, Tc(0.0625) * k4.x));
        acc.y = fma(Tc(0.25), c0.y, fma(Tc(0.125), e4.y, Tc(0.0625) * k4.y));
      } else {
        acc.x = fma(Tc(0.25), c0.x, Tc(0.0625) * k4.x);
        acc.y = fma(Tc(0.25), c0.y, Tc(0.0625) * k4.y);
      }
      rc[(int64_t)p * npc + (int64_t)J * mc + I] = acc;
    }
    __syncthreads();
  }
}

template <typename Tc, typename TU, int CX>
cudaError_t down2(Launch& L, int m, int planes, int pch, const Tc* w, const Tc* diag,
                  const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u, typename Cx<Tc>::t* rc) {
  typedef typename Cx<Tc>::t C;
  constexpr int WR = 2 * CX + 5;
  const size_t smem = (size_t)WR * WR * (2 * sizeof(C) + 5 * sizeof(Tc));
  cudaError_t e = cudaFuncSetAttribute(mg_down2_kernel<Tc, TU, CX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int mc = (m - 1) / 2;
  const unsigned tiles = (unsigned)((mc + CX - 1) / CX);
  dim3 grid(tiles, tiles, (unsigned)((planes + pch - 1) / pch));
  mg_down2_kernel<Tc, TU, CX><<<grid, 256, smem, L.stream>>>(r, u, rc, w, diag, sigma, m, planes, pch);
  return cudaGetLastError();
}

}  // namespace

// default tile: 16 x 16 coarse points (FP32 window 37^2, 49 KB) or 8 x 8 in FP64;
// planes per CTA so that the grid holds about ctas_per_sm CTAs per SM (default 8)
int mg_down_default_cx(int tc_bytes) { return tc_bytes == 4 ? 16 : 8; }

int mg_down_default_pch(int m, int planes, int cx, int ctas_per_sm, int sms) {
  const int mc = (m - 1) / 2;
  const long tiles = (long)((mc + cx - 1) / cx) * ((mc + cx - 1) / cx);
  const long target = (long)(ctas_per_sm > 0 ? ctas_per_sm : 8) * (sms > 0 ? sms : 152);
  long pch = (tiles * planes + target - 1) / target;
  if (pch < 1) pch = 1;
  if (pch > 64) pch = 64;
  return (int)pch;
}

template <typename Tc, typename TU>
cudaError_t launch_mg_down(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                           const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u,
                           typename Cx<Tc>::t* rc, int cx, int pch) {
  if (g.dim != 2 || g.m < 3 || (g.m & 1) == 0) return cudaErrorInvalidValue;
  if (cx <= 0 && L.tiles) cx = L.tiles->mg_cx;
  if (cx <= 0) cx = mg_down_default_cx((int)sizeof(Tc));
  if (pch <= 0)
    pch = mg_down_default_pch(g.m, planes, cx, L.tiles ? L.tiles->mg_ctas : 0, L.tiles ? L.tiles->sms : 0);
  const double cs = sizeof(typename Cx<Tc>::t);
  const int mc = (g.m - 1) / 2;
  const double tot = (double)g.np * planes;
  // algorithmic bytes: read r, write u, write the coarse right-hand side
  const double bytes = tot * (cs + sizeof(TU)) + (double)mc * mc * planes * cs;
  L.begin(KC_MG_DOWN);
  cudaError_t e;
  if (cx == 8)
    e = down2<Tc, TU, 8>(L, g.m, planes, pch, st.w, st.diag, sigma, r, u, rc);
  else if (cx == 16)
    e = down2<Tc, TU, 16>(L, g.m, planes, pch, st.w, st.diag, sigma, r, u, rc);
  else
    e = cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  return L.end(KC_MG_DOWN, bytes, tot * 60.0);
}

#define PCOPT_INST_DOWN(Tc, TU)                                                                              \
  template cudaError_t launch_mg_down<Tc, TU>(Launch&, const Grid&, int, const Stencil<Tc>&, const Cx<Tc>::t*, \
                                              const Cx<Tc>::t*, TU*, Cx<Tc>::t*, int, int);
PCOPT_INST_DOWN(float, float2)
PCOPT_INST_DOWN(double, double2)
PCOPT_INST_DOWN(float, __nv_bfloat162)
#undef PCOPT_INST_DOWN

}  // namespace pcopt
