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
#include <algorithm>

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

// ---------------------------------------------------------------------------
// Register-marching variant (FP32 iterates): no shared memory, no barriers.  A warp
// owns one spectral plane, a strip of 64 fine columns (lane q: the column pair
// cA = 2 I0 - 2 + 2q, cB = cA + 1, which always holds one red and one black cell)
// and a segment of coarse rows [J0, J1); it walks the fine rows t = 2 J0 - 2 ...
// 2 J1 + 2 and at each step forms
//   red u of row t (from r and the shift alone),
//   black u of row t - 1 (red neighbours: the lane's own rows t - 2, t - 1, t and
//     the pair partner or the neighbouring lane's row t - 1 via a shuffle),
//   the red residual of row t - 2 (black neighbours likewise, the sweep-from-zero
//     identity: res_red = sum_k w_k u_black, res_black = 0),
//   and, when row t - 2 = 2J + 2 is even, the full-weighting value of coarse row J
//     from the residual rows 2J, 2J + 1, 2J + 2 (centre at cB, corners at cA and at
//     the next lane's cA).
// Lanes 1..29 own their pairs and coarse points; lanes 0, 30, 31 are the halo whose
// values only feed their neighbours.  Rows and columns outside the grid hold zero.
constexpr int kMarchPairs = 29;

__device__ __forceinline__ float2 shfl_dn(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_upc(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ void prefetch_l1(const void* ptr) { asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr)); }

// State of one lane between steps: red u of rows t-2, t-1 (R0, R1), black u of rows
// t-3, t-2 (B0, B1), the black r of row t-1, the last even-row restriction partial
// and the last odd-row residual; r of rows t .. t + kMarchAhead - 1 in flight.
constexpr int kMarchAhead = 2;  // (4 was slower: fewer resident warps)
struct MarchState {
  float2 R0, R1, B0, B1, rbp, Ep, ro;
  float2 nA[kMarchAhead], nB[kMarchAhead];
};

// One step at row t; EV = (t even).  Red cells: cA on even rows, cB on odd rows.
template <bool EV>
__device__ __forceinline__ void march_step(MarchState& S, int t, const float2* __restrict__ rp,
                                           float2* __restrict__ up, float2* __restrict__ rcp,
                                           const float4* __restrict__ w4, const float* __restrict__ diag,
                                           float2 sig, int m, int mc, int cA, bool inA, bool inB, bool own,
                                           bool ownc, int Ic, int k0, int k1, int J0, int J1) {
  const float2 z = make_float2(0.f, 0.f);
  const int cB = cA + 1;
  const float2 rA = S.nA[0], rB = S.nB[0];
#pragma unroll
  for (int i = 0; i + 1 < kMarchAhead; ++i) {
    S.nA[i] = S.nA[i + 1];
    S.nB[i] = S.nB[i + 1];
  }
  {  // r kMarchAhead rows ahead in flight, coefficients one row further into L1
    const int ta = t + kMarchAhead;
    const bool ok = ta >= 0 && ta < m;
    const int o = ta * m;
    S.nA[kMarchAhead - 1] = (ok && inA) ? rp[o + cA] : z;
    S.nB[kMarchAhead - 1] = (ok && inB) ? rp[o + cB] : z;
    const int tc = ta + 1;
    if (inA && tc >= 0 && tc < m) {
      prefetch_l1(w4 + tc * m + cA);
      prefetch_l1(diag + tc * m + cA);
    }
  }
  // red u of row t
  float2 R2 = z;
  {
    const int c = EV ? cA : cB;
    if ((EV ? inA : inB) && t >= 0 && t < m)
      R2 = cmul(EV ? rA : rB, inv_shift(make_float2(sig.x + diag[t * m + c], sig.y)));
  }
  // black u of row t - 1 (black at cB on even rows, at cA on odd rows)
  float2 B2 = z;
  {
    const int k = t - 1;  // parity opposite to t
    const float2 nb = EV ? shfl_upc(S.R1) : shfl_dn(S.R1);
    const float2 left = EV ? nb : S.R1, right = EV ? S.R1 : nb;
    const int c = EV ? cA : cB;
    if ((EV ? inA : inB) && k >= 0 && k < m) {
      const int o = k * m + c;
      const float4 wv = w4[o];
      float2 acc = S.rbp;
      cfma<float>(acc, wv.x, left);
      cfma<float>(acc, wv.y, right);
      cfma<float>(acc, wv.z, S.R0);
      cfma<float>(acc, wv.w, R2);
      B2 = cmul(acc, inv_shift(make_float2(sig.x + diag[o], sig.y)));
    }
    if (own && k >= k0 && k < k1) {
      const int o = k * m;
      if (inA) up[o + cA] = EV ? B2 : S.R1;
      if (inB) up[o + cB] = EV ? S.R1 : B2;
    }
  }
  // red residual of row t - 2 (same parity as t)
  {
    const int k2 = t - 2;
    const float2 nb = EV ? shfl_upc(S.B1) : shfl_dn(S.B1);
    const float2 left = EV ? nb : S.B1, right = EV ? S.B1 : nb;
    const int c = EV ? cA : cB;
    float2 res = z;
    if ((EV ? inA : inB) && k2 >= 0 && k2 < m) {
      const float4 wv = w4[k2 * m + c];
      res.x = wv.x * left.x;
      res.y = wv.x * left.y;
      cfma<float>(res, wv.y, right);
      cfma<float>(res, wv.z, S.B0);
      cfma<float>(res, wv.w, B2);
    }
    if (EV) {
      const float2 sdr = shfl_dn(res);
      const float2 E = make_float2(res.x + sdr.x, res.y + sdr.y);
      const int J = (k2 >> 1) - 1;  // coarse row whose last residual row is k2
      if (ownc && J >= J0 && J < J1) {
        float2 v;
        v.x = fmaf(0.25f, S.ro.x, 0.0625f * (S.Ep.x + E.x));
        v.y = fmaf(0.25f, S.ro.y, 0.0625f * (S.Ep.y + E.y));
        rcp[J * mc + Ic] = v;
      }
      S.Ep = E;
    } else {
      S.ro = res;
    }
  }
  S.R0 = S.R1;
  S.R1 = R2;
  S.B0 = S.B1;
  S.B1 = B2;
  S.rbp = EV ? rB : rA;  // black r of row t
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS) mg_down2_march_kernel(const float2* __restrict__ r,
                                                                    float2* __restrict__ u,
                                                                    float2* __restrict__ rc,
                                                                    const float4* __restrict__ w4,
                                                                    const float* __restrict__ diag,
                                                                    const float2* __restrict__ sigma, int m,
                                                                    int planes, int segj, int nstrips) {
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.y * WARPS + (threadIdx.x >> 5);
  if (p >= planes) return;  // whole warp
  const int mc = (m - 1) / 2;
  const int st = blockIdx.x % nstrips, sg = blockIdx.x / nstrips;
  const int I0 = st * kMarchPairs;
  const int J0 = sg * segj, J1 = min(mc, J0 + segj);
  const int k0 = 2 * J0, k1 = (J1 == mc) ? m : 2 * J1;
  const int cA = 2 * I0 - 2 + 2 * lane;
  const bool inA = cA >= 0 && cA < m, inB = cA + 1 >= 0 && cA + 1 < m;
  const bool own = lane >= 1 && lane <= kMarchPairs;
  const int Ic = I0 - 1 + lane;
  const bool ownc = own && Ic < mc;
  const int64_t np = (int64_t)m * m;
  const float2* rp = r + (int64_t)p * np;
  float2* up = u + (int64_t)p * np;
  float2* rcp = rc + (int64_t)p * mc * mc;
  const float2 sig = sigma[p];
  const float2 z = make_float2(0.f, 0.f);
  MarchState S;
  S.R0 = S.R1 = S.B0 = S.B1 = S.rbp = S.Ep = S.ro = z;
  // rows k0 - 2 (even) ... k0 - 3 + kMarchAhead in flight before the first step
#pragma unroll
  for (int i = 0; i < kMarchAhead; ++i) {
    const int ti = k0 - 2 + i;
    const bool ok = ti >= 0 && ti < m;
    S.nA[i] = (ok && inA) ? rp[ti * m + cA] : z;
    S.nB[i] = (ok && inB) ? rp[ti * m + cA + 1] : z;
  }
  const int tEnd = 2 * J1 + 2;  // even, like the first row k0 - 2
  int t = k0 - 2;
  for (; t + 1 <= tEnd; t += 2) {
    march_step<true>(S, t, rp, up, rcp, w4, diag, sig, m, mc, cA, inA, inB, own, ownc, Ic, k0, k1, J0, J1);
    march_step<false>(S, t + 1, rp, up, rcp, w4, diag, sig, m, mc, cA, inA, inB, own, ownc, Ic, k0, k1, J0, J1);
  }
  march_step<true>(S, t, rp, up, rcp, w4, diag, sig, m, mc, cA, inA, inB, own, ownc, Ic, k0, k1, J0, J1);
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
                           typename Cx<Tc>::t* rc, int cx, int pch, const float4* w4) {
  if (g.dim != 2 || g.m < 3 || (g.m & 1) == 0) return cudaErrorInvalidValue;
  if constexpr (std::is_same<Tc, float>::value && std::is_same<TU, float2>::value) {
    if (w4 && L.tiles && L.tiles->mg_march > 0) {
      constexpr int WARPS = 4;
      const int mc = (g.m - 1) / 2;
      const int nstrips = (mc + kMarchPairs - 1) / kMarchPairs;
      // the tuned segment length, shortened on small levels until the grid holds
      // about 32 warps per SM
      int segj = L.tiles->mg_seg > 0 ? L.tiles->mg_seg : 16;
      const long target = 32L * (L.tiles->sms > 0 ? L.tiles->sms : 152);
      const long need = (target + (long)nstrips * planes - 1) / ((long)nstrips * planes);
      if (need > 1) segj = std::min(segj, std::max(2, (int)(mc / need)));
      const int nsegs = (mc + segj - 1) / segj;
      const double tot = (double)g.np * planes;
      L.begin(KC_MG_DOWN);
      mg_down2_march_kernel<WARPS><<<dim3((unsigned)(nstrips * nsegs), (unsigned)((planes + WARPS - 1) / WARPS)),
                                     32 * WARPS, 0, L.stream>>>(r, u, rc, w4, st.diag, sigma, g.m, planes, segj,
                                                                nstrips);
      return L.end(KC_MG_DOWN, tot * (sizeof(float2) + sizeof(float2)) + (double)mc * mc * planes * sizeof(float2),
                   tot * 60.0);
    }
  }
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
                                              const Cx<Tc>::t*, TU*, Cx<Tc>::t*, int, int, const float4*);
PCOPT_INST_DOWN(float, float2)
PCOPT_INST_DOWN(double, double2)
PCOPT_INST_DOWN(float, __nv_bfloat162)
#undef PCOPT_INST_DOWN

}  // namespace pcopt
