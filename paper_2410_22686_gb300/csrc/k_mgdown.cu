// Down leg of one multigrid level of the V(1,0) cycle (Section 2.1, step 2 of the
// apply of P_eps^{-1}, variable a) in one launch for 2D grids:
//
//   red-black Gauss-Seidel sweep from u = 0 on (sigma_p I + tau K) u = r,
//   residual  res = r - (sigma_p I + tau K) u,
//   full weighting  rc(I, J) = sum_{o1,o2 in -1..1} w(o1) w(o2) res(2I+1+o1, 2J+1+o2),
//   w(0) = 1/2, w(+-1) = 1/4,
//
// the operations of the per-level kernels of k_spatial.cu, but r is read from HBM
// once and the residual never goes there.  A CTA owns a CX x CX tile of coarse
// points (the fine points 2I, 2I+1 of each, the last tile also the fine point
// m-1), stages r on the fine window [2I0-2, 2I0+2CX+2]^2 in shared memory, takes
// red u on all of it, black u on [2I0-1, 2I0+2CX+1]^2 and the residual on
// [2I0, 2I0+2CX]^2, then restricts.  The face weights and diagonal of the window
// stay in shared memory for all the CTA's planes, and the next plane's window is
// loaded while the current one is swept.  Points outside the grid hold r = u = 0
// (homogeneous Dirichlet boundary).  Red = even i1 + i2 (0-based), swept first.
// Values of u are rounded to the storage type TU before any later step reads
// them, so the BF16-storage variant smooths, takes residuals and is corrected on
// exactly what it stores.
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

// the four face weights of one cell, loaded with one shared-memory access
template <typename T>
struct W4;
template <>
struct W4<float> {
  typedef float4 t;
};
template <>
struct W4<double> {
  typedef double4_32a t;
};

template <typename T>
__device__ __forceinline__ void cfma(typename Cx<T>::t& acc, T w, typename Cx<T>::t v) {
  acc.x = fma(w, v.x, acc.x);
  acc.y = fma(w, v.y, acc.y);
}

// Shared memory holds the window colour by colour: the window origin (2 I0 - 2,
// 2 J0 - 2) is even, so cell (a1, a2) is red iff a1 + a2 is even, and each colour
// of row a2 is a dense row of HW = (WR + 1) / 2 slots indexed k = a1 >> 1.  The
// four neighbours of a cell have the other colour and sit at k - p, k + 1 - p
// (same row) and k (rows a2 +- 1), with p = a2 & 1 for a black cell and 1 - p
// for a red one; consecutive lanes take consecutive k, so every access is
// unit-stride.
template <typename Tc, typename TU, int CX>
__global__ void __launch_bounds__(256) mg_down2_kernel(const typename Cx<Tc>::t* __restrict__ r, TU* __restrict__ u,
                                                       typename Cx<Tc>::t* __restrict__ rc,
                                                       const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                       const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                       int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  constexpr int NT = 256;
  constexpr int WR = 2 * CX + 5;   // r window per axis
  constexpr int HW = (WR + 1) / 2; // slots per row and colour
  constexpr int NH = WR * HW;      // slots per colour
  constexpr int SA = (2 * NH + NT - 1) / NT;       // window slots per thread (both colours)
  constexpr int NBR = WR - 2;                      // black rows [1, WR-2]
  constexpr int SB = (NBR * HW + NT - 1) / NT;     // black slots
  constexpr int NRR = WR - 4;                      // residual rows [2, WR-3]
  constexpr int SC = (NRR * HW + NT - 1) / NT;     // red residual slots
  // Residual of a sweep from zero: black points are solved exactly against their
  // red neighbours and red points against zero, so res_black = 0 and
  // res_red = sum_k w_k u_black(nb_k).  With BF16 storage the stored u no longer
  // satisfies this and the residual is formed explicitly from it.
  constexpr bool EXPLICIT = std::is_same<TU, __nv_bfloat162>::value;
  typedef typename W4<Tc>::t WV;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  WV* sWr = reinterpret_cast<WV*>(smem_raw);  // faces (-x, +x, -y, +y) of red cells
  WV* sWb = sWr + NH;
  C* sRr = reinterpret_cast<C*>(sWb + NH);    // r (then the red residual), red cells
  C* sRb = sRr + NH;                          // r (then the black residual), black cells
  C* sUr = sRb + NH;
  C* sUb = sUr + NH;
  Tc* sDr = reinterpret_cast<Tc*>(sUb + NH);
  Tc* sDb = sDr + NH;

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

  // window slots e in [0, 2 NH): colour c = e / NH (0 red), row a2, k; per slot the
  // in-plane offset (-1 outside the grid) and ownership
  int goffA[SA];
  unsigned ownA = 0;
#pragma unroll
  for (int i = 0; i < SA; ++i) {
    const int e = tid + i * NT;
    const int c = e >= NH ? 1 : 0;
    const int h = e - c * NH;
    const int a2 = h / HW, k = h - (h / HW) * HW;
    const int a1 = 2 * k + ((a2 & 1) ^ c);
    const int f1 = fx + a1, f2 = fy + a2;
    const bool in = e < 2 * NH && a1 < WR && f1 >= 0 && f1 < m && f2 >= 0 && f2 < m;
    goffA[i] = in ? f2 * m + f1 : -1;
    if (in && a1 >= 2 && a1 < ex && a2 >= 2 && a2 < ey) ownA |= 1u << i;
    if (e < 2 * NH) {
      (c ? sDb : sDr)[h] = in ? diag[goffA[i]] : Tc(0);
      WV wv;
      wv.x = in ? w[goffA[i]] : Tc(0);
      wv.y = in ? w[np + goffA[i]] : Tc(0);
      wv.z = in ? w[2 * np + goffA[i]] : Tc(0);
      wv.w = in ? w[3 * np + goffA[i]] : Tc(0);
      (c ? sWb : sWr)[h] = wv;
      (c ? sRb : sRr)[h] = czero<Tc>();
      (c ? sUb : sUr)[h] = czero<Tc>();
    }
  }
  // black cells of rows [1, WR-2] with a1 in [1, WR-2] inside the grid
  int hB[SB];
  unsigned ownB = 0;
#pragma unroll
  for (int i = 0; i < SB; ++i) {
    const int e = tid + i * NT;
    const int a2 = 1 + e / HW, k = e - (e / HW) * HW;
    const int a1 = 2 * k + ((a2 & 1) ^ 1);
    const int f1 = fx + a1, f2 = fy + a2;
    const bool ok = e < NBR * HW && a1 >= 1 && a1 <= WR - 2 && f1 >= 0 && f1 < m && f2 >= 0 && f2 < m;
    hB[i] = ok ? a2 * HW + k : -1;
    if (ok && a1 >= 2 && a1 < ex && a2 >= 2 && a2 < ey) ownB |= 1u << i;
  }
  // red cells of rows [2, WR-3] with a1 in [2, WR-3] inside the grid
  int hC[SC];
#pragma unroll
  for (int i = 0; i < SC; ++i) {
    const int e = tid + i * NT;
    const int a2 = 2 + e / HW, k = e - (e / HW) * HW;
    const int a1 = 2 * k + (a2 & 1);
    const bool ok = e < NRR * HW && a1 >= 2 && a1 <= WR - 3 && fx + a1 < m && fy + a2 < m;
    hC[i] = ok ? a2 * HW + k : -1;
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
      if (e < NH) {
        sRr[e] = pre[i];
        const C uv = stored<TU>(cmul(pre[i], inv_shift(cmk<Tc>(sig.x + sDr[e], sig.y))));
        sUr[e] = uv;
        if (ownA & (1u << i)) stc(up, goffA[i], uv);
      } else {
        sRb[e - NH] = pre[i];
      }
    }
    __syncthreads();
    if (p + 1 < p1) fetch(p + 1);  // the next plane's window is in flight meanwhile
    // black points: u = (r + sum_k w_k u_red(nb_k)) / (sigma + d)
#pragma unroll
    for (int i = 0; i < SB; ++i) {
      const int h = hB[i];
      if (h < 0) continue;
      const int a2 = h / HW;
      const int s = a2 & 1;  // left red neighbour at k - s, right at k + 1 - s
      C acc = sRb[h];
      const WV wv = sWb[h];
      cfma<Tc>(acc, wv.x, sUr[h - s]);
      cfma<Tc>(acc, wv.y, sUr[h + 1 - s]);
      cfma<Tc>(acc, wv.z, sUr[h - HW]);
      cfma<Tc>(acc, wv.w, sUr[h + HW]);
      const C uv = stored<TU>(cmul(acc, inv_shift(cmk<Tc>(sig.x + sDb[h], sig.y))));
      sUb[h] = uv;
      if (ownB & (1u << i)) {
        const int k = h - a2 * HW;
        stc(up, (int64_t)(fy + a2) * m + fx + 2 * k + (s ^ 1), uv);
      }
    }
    __syncthreads();
    if constexpr (!EXPLICIT) {
      // red residuals, in place of r
#pragma unroll
      for (int i = 0; i < SC; ++i) {
        const int h = hC[i];
        if (h < 0) continue;
        const int s = (h / HW) & 1;  // left black neighbour at k - 1 + s, right at k + s
        C res;
        const WV wv = sWr[h];
        const C ul = sUb[h - 1 + s];
        res.x = wv.x * ul.x;
        res.y = wv.x * ul.y;
        cfma<Tc>(res, wv.y, sUb[h + s]);
        cfma<Tc>(res, wv.z, sUb[h - HW]);
        cfma<Tc>(res, wv.w, sUb[h + HW]);
        sRr[h] = res;
      }
    } else {
      // residual of the stored u at every point of the restriction windows
      for (int e = tid; e < 2 * NRR * HW; e += NT) {
        const int c = e >= NRR * HW ? 1 : 0;
        const int g = e - c * NRR * HW;
        const int a2 = 2 + g / HW, k = g - (g / HW) * HW;
        const int sp = (a2 & 1) ^ c;  // a1 parity
        const int a1 = 2 * k + sp;
        if (a1 < 2 || a1 > WR - 3 || fx + a1 >= m || fy + a2 >= m) continue;
        const int h = a2 * HW + k;
        // neighbours have the other colour; same-row ones at k - 1 + sp and k + sp
        const C* U = c ? sUr : sUb;
        const WV wv = (c ? sWb : sWr)[h];
        const C uc = (c ? sUb : sUr)[h];
        C lu = cmul(cmk<Tc>(sig.x + (c ? sDb : sDr)[h], sig.y), uc);
        cfma<Tc>(lu, -wv.x, U[h - 1 + sp]);
        cfma<Tc>(lu, -wv.y, U[h + sp]);
        cfma<Tc>(lu, -wv.z, U[h - HW]);
        cfma<Tc>(lu, -wv.w, U[h + HW]);
        C* R = c ? sRb : sRr;
        R[h] = R[h] - lu;
      }
    }
    __syncthreads();
    // full weighting onto the coarse tile: centre and corners are red, edges black
    // (zero residual unless it was formed explicitly)
    for (int e = tid; e < CX * CX; e += NT) {
      const int I = I0 + e % CX, J = J0 + e / CX;
      if (I >= mc || J >= mc) continue;
      const int a1 = 2 * (I - I0) + 3, a2 = 2 * (J - J0) + 3;  // odd: k = (a1 - 1) / 2 in row a2
      const int h = a2 * HW + (a1 >> 1);
      // corners (a1 -+ 1, a2 -+ 1) are red cells of the even rows at k and k + 1
      const C c0 = sRr[h];
      const C k4 = sRr[h - HW] + sRr[h - HW + 1] + sRr[h + HW] + sRr[h + HW + 1];
      C acc;
      if constexpr (EXPLICIT) {
        // edges: black (a1 -+ 1, a2) at k, k + 1 in row a2; (a1, a2 -+ 1) at k in rows a2 -+ 1
        const C e4 = sRb[h] + sRb[h + 1] + sRb[h - HW] + sRb[h + HW];
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
  constexpr int NH = WR * ((WR + 1) / 2);  // slots per colour
  const size_t smem = (size_t)NH * (2 * sizeof(typename W4<Tc>::t) + 4 * sizeof(C) + 2 * sizeof(Tc));
  cudaError_t e = cudaFuncSetAttribute(mg_down2_kernel<Tc, TU, CX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // prefer shared memory in the unified L1 (the window is 50 KB per CTA in FP32)
  e = cudaFuncSetAttribute(mg_down2_kernel<Tc, TU, CX>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
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
