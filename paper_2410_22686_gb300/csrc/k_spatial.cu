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
#include <type_traits>

#include "common.cuh"

namespace pcopt {

namespace {

constexpr int kPlaneChunk = 8;  // default planes per CTA

// 1 / (sigma + d); FP32 with the hardware-approximate divide (2 ulp, far inside what
// a smoother needs), FP64 exact
__device__ __forceinline__ float2 inv_shift_c(float2 sig, float d) {
  const float a = sig.x + d;
  const float q = __fdividef(1.0f, fmaf(a, a, sig.y * sig.y));
  return make_float2(a * q, -sig.y * q);
}
__device__ __forceinline__ double2 inv_shift_c(double2 sig, double d) { return inv_diag<double>(sig, d); }

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
                                  const Tc* __restrict__ rmass, const typename Cx<Tc>::t* __restrict__ sigma,
                                  int64_t np, int planes) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * planes) return;
  const int64_t p = e / np;
  const int64_t s = e - p * np;
  typename Cx<Tc>::t v = buf[e];
  if (rmass) v = cscale(v, rmass[s]);  // finite elements: 1 / eigenvalue of M
  buf[e] = cmul(v, inv_diag<Tc>(sigma[p], lamK[s]));
}

// ------------------------------------------------------------------- multigrid
// One red-black Gauss-Seidel sweep from u = 0: a red point takes r/d; a black point
// takes (r + sum_k w_k u_red(nb_k))/d.  MODE 0 does both colours in one pass and
// recomputes the red neighbour values from r (one reciprocal per neighbour, cheap in
// FP32); MODE 1 writes the red points only and MODE 2 the black ones from the stored
// red values (two passes, one reciprocal per point: FP64, whose reciprocal is costly).
// MODE 0 with one thread per pair of x1-neighbours (i1 = 2q, 2q+1): one point of the
// pair is red and one black, so every lane does one red and one black update (a thread
// per point splits each warp between the cheap red and the expensive black update) and
// the black point takes its partner's red value without recomputing it.
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_smooth_pair_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                             TU* __restrict__ u, const Tc* __restrict__ w,
                                                             const Tc* __restrict__ diag,
                                                             const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                             int64_t np, int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  const int half = (m + 1) / 2;  // pairs per grid row (the last one may hold a single point)
  const int64_t rows = np / m;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * half) return;
  const int p0 = blockIdx.y * pch;
  const int p1 = min(planes, p0 + pch);
  const int64_t row = t / half;
  const int q = (int)(t - row * half);
  const int i2 = (int)(DIM == 2 ? row : row % m);
  const int i3 = (int)(DIM == 3 ? row / m : 0);
  const int ia = 2 * q;
  const bool hasb = ia + 1 < m;
  const bool a_red = ((ia + i2 + i3 + DIM) & 1) == 0;
  const int64_t sa = row * m + ia;
  // the black point of the pair (absent when the pair holds only a red point)
  const bool has_black = !a_red || hasb;
  const bool has_red = a_red || hasb;
  const int64_t sr = a_red ? sa : sa + 1;
  const int64_t sk = a_red ? sa + 1 : sa;
  const int ik = a_red ? ia + 1 : ia;  // x1 index of the black point
  const Tc dr = has_red ? diag[sr] : Tc(1);
  // neighbours of the black point: x1 -/+ (one of them is the red partner), x2 -/+, x3 -/+
  int64_t off[2 * DIM];
  bool ex[2 * DIM];
  bool partner[2 * DIM];
  Tc wv[2 * DIM], dn[2 * DIM];
  const int64_t mm = (int64_t)m * m;
  off[0] = -1;
  ex[0] = ik > 0;
  off[1] = 1;
  ex[1] = ik < m - 1;
  off[2] = -(int64_t)m;
  ex[2] = i2 > 0;
  off[3] = m;
  ex[3] = i2 < m - 1;
  if (DIM == 3) {
    off[4] = -mm;
    ex[4] = i3 > 0;
    off[5] = mm;
    ex[5] = i3 < m - 1;
  }
#pragma unroll
  for (int k = 0; k < 2 * DIM; ++k) partner[k] = has_red && (k == (a_red ? 0 : 1));
  Tc dk = Tc(1);
  if (has_black) {
    dk = diag[sk];
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k) {
      wv[k] = w[(int64_t)k * np + sk];
      dn[k] = (ex[k] && !partner[k]) ? diag[sk + off[k]] : Tc(0);
    }
  }
  for (int p = p0; p < p1; ++p) {
    const int64_t base = (int64_t)p * np;
    const C sig = sigma[p];
    C ur = czero<Tc>();
    if (has_red) {
      ur = cmul(r[base + sr], inv_shift_c(sig, dr));
      stc(u, base + sr, ur);
    }
    if (has_black) {
      const int64_t o = base + sk;
      C acc = r[o];
#pragma unroll
      for (int k = 0; k < 2 * DIM; ++k) {
        if (ex[k]) {
          const C v = partner[k] ? ur : cmul(r[o + off[k]], inv_shift_c(sig, dn[k]));
          acc.x = fma(wv[k], v.x, acc.x);
          acc.y = fma(wv[k], v.y, acc.y);
        }
      }
      stc(u, o, cmul(acc, inv_shift_c(sig, dk)));
    }
  }
}

template <typename Tc, typename TU, int DIM, int MODE>
__global__ void __launch_bounds__(256) mg_smooth_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                        TU* __restrict__ u,
                                                        const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                        const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                        int64_t np, int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  const int p0 = blockIdx.y * pch;
  const int p1 = min(planes, p0 + pch);
  const Coord c = coord_of(s, m, DIM);
  const bool red = ((c.i1 + c.i2 + c.i3 + DIM) & 1) == 0;
  const Tc dg = diag[s];
  if (red) {
    if (MODE == 2) return;
    for (int p = p0; p < p1; ++p) {
      const int64_t o = (int64_t)p * np + s;
      stc(u, o, cmul(r[o], inv_shift_c(sigma[p], dg)));
    }
    return;
  }
  if (MODE == 1) return;
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
        const C ured = MODE == 2 ? ldc(u, o + off[k]) : cmul(r[o + off[k]], inv_shift_c(sig, dn[k]));
        acc.x = fma(wv[k], ured.x, acc.x);
        acc.y = fma(wv[k], ured.y, acc.y);
      }
    }
    stc(u, o, cmul(acc, inv_shift_c(sig, dg)));
  }
}

// res = r - (sigma u + tau K u)
// Gauss-Seidel sweep from zero in the natural order (x1 fastest): u_P = (r_P + sum over
// the lower neighbours Q of w_PQ u_Q) / (sigma + d_P); the other neighbours are still
// zero.  Points with equal index sum i1 + i2 (+ i3) do not depend on each other, so one
// CTA per spectral plane walks these diagonals in order, a barrier between two (the
// values of the previous diagonal come back through the CTA's own global writes).
// This is the paper-reproduction option of the smoother; the red-black sweep is the
// parallel default.
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_smooth_lex_kernel(const typename Cx<Tc>::t* __restrict__ r, TU* u,
                                                            const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                            const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                            int64_t np) {
  typedef typename Cx<Tc>::t C;
  const int p = blockIdx.x;
  const C sig = sigma[p];
  const C* rp = r + (int64_t)p * np;
  TU* up = u + (int64_t)p * np;
  const int64_t mm = (int64_t)m * m;
  const int tmax = DIM * (m - 1);
  for (int t = 0; t <= tmax; ++t) {
    if (DIM == 2) {
      const int lo = max(0, t - (m - 1)), hi = min(m - 1, t);
      for (int i2 = lo + (int)threadIdx.x; i2 <= hi; i2 += blockDim.x) {
        const int i1 = t - i2;
        const int64_t s = (int64_t)i2 * m + i1;
        C acc = rp[s];
        if (i1 > 0) {
          const C v = ldc(up, s - 1);
          const Tc wk = w[s];  // towards -x1
          acc.x = fma(wk, v.x, acc.x);
          acc.y = fma(wk, v.y, acc.y);
        }
        if (i2 > 0) {
          const C v = ldc(up, s - m);
          const Tc wk = w[2 * np + s];  // towards -x2
          acc.x = fma(wk, v.x, acc.x);
          acc.y = fma(wk, v.y, acc.y);
        }
        stc(up, s, cmul(acc, inv_diag<Tc>(sig, diag[s])));
      }
    } else {
      // (i2, i3) pairs of the diagonal: i1 = t - i2 - i3 in [0, m)
      const int lo3 = max(0, t - 2 * (m - 1)), hi3 = min(m - 1, t);
      const int n3 = hi3 - lo3 + 1;
      for (int q = (int)threadIdx.x; q < n3 * m; q += blockDim.x) {
        const int i3 = lo3 + q / m, i2 = q - (q / m) * m;
        const int i1 = t - i2 - i3;
        if (i1 < 0 || i1 >= m) continue;
        const int64_t s = (int64_t)i3 * mm + (int64_t)i2 * m + i1;
        C acc = rp[s];
        if (i1 > 0) {
          const C v = ldc(up, s - 1);
          const Tc wk = w[s];
          acc.x = fma(wk, v.x, acc.x);
          acc.y = fma(wk, v.y, acc.y);
        }
        if (i2 > 0) {
          const C v = ldc(up, s - m);
          const Tc wk = w[2 * np + s];
          acc.x = fma(wk, v.x, acc.x);
          acc.y = fma(wk, v.y, acc.y);
        }
        if (i3 > 0) {
          const C v = ldc(up, s - mm);
          const Tc wk = w[4 * np + s];  // towards -x3
          acc.x = fma(wk, v.x, acc.x);
          acc.y = fma(wk, v.y, acc.y);
        }
        stc(up, s, cmul(acc, inv_diag<Tc>(sig, diag[s])));
      }
    }
    __syncthreads();
  }
}

// Residual after the red-black sweep from zero, from the sweep's identity: zero at
// black points (their update solved their own equation) and sum_k w_k u_black at red
// ones (the red update used zero neighbours).  One thread per red/black pair along x1.
// Iterates stored in the compute type only (BF16 storage breaks the identity).
template <typename Tc, int DIM>
__global__ void __launch_bounds__(256) mg_residual_pair_kernel(const typename Cx<Tc>::t* __restrict__ u,
                                                               typename Cx<Tc>::t* __restrict__ res,
                                                               const Tc* __restrict__ w, int m, int64_t np,
                                                               int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  const int half = (m + 1) / 2;
  const int64_t rows = np / m;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * half) return;
  const int p0 = blockIdx.y * pch;
  const int p1 = min(planes, p0 + pch);
  const int64_t row = t / half;
  const int q = (int)(t - row * half);
  const int i2 = (int)(DIM == 2 ? row : row % m);
  const int i3 = (int)(DIM == 3 ? row / m : 0);
  const int ia = 2 * q;
  const bool hasb = ia + 1 < m;
  const bool a_red = ((ia + i2 + i3 + DIM) & 1) == 0;
  const int64_t sa = row * m + ia;
  const bool has_red = a_red || hasb;
  const bool has_black = !a_red || hasb;
  const int64_t sr = a_red ? sa : sa + 1;
  const int64_t sk = a_red ? sa + 1 : sa;
  const int ir = a_red ? ia : ia + 1;
  int64_t off[2 * DIM];
  bool ex[2 * DIM];
  Tc wv[2 * DIM];
  const int64_t mm = (int64_t)m * m;
  off[0] = -1;
  ex[0] = ir > 0;
  off[1] = 1;
  ex[1] = ir < m - 1;
  off[2] = -(int64_t)m;
  ex[2] = i2 > 0;
  off[3] = m;
  ex[3] = i2 < m - 1;
  if (DIM == 3) {
    off[4] = -mm;
    ex[4] = i3 > 0;
    off[5] = mm;
    ex[5] = i3 < m - 1;
  }
  if (has_red) {
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k) wv[k] = w[(int64_t)k * np + sr];
  }
  for (int p = p0; p < p1; ++p) {
    const int64_t base = (int64_t)p * np;
    if (has_black) res[base + sk] = czero<Tc>();
    if (has_red) {
      const int64_t o = base + sr;
      C acc = czero<Tc>();
#pragma unroll
      for (int k = 0; k < 2 * DIM; ++k) {
        if (ex[k]) {
          const C un = u[o + off[k]];
          acc.x = fma(wv[k], un.x, acc.x);
          acc.y = fma(wv[k], un.y, acc.y);
        }
      }
      res[o] = acc;
    }
  }
}

template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_residual_kernel(const typename Cx<Tc>::t* __restrict__ r,
                                                          const TU* __restrict__ u,
                                                          typename Cx<Tc>::t* __restrict__ res,
                                                          const Tc* __restrict__ w, const Tc* __restrict__ diag,
                                                          const typename Cx<Tc>::t* __restrict__ sigma, int m,
                                                          int64_t np, int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  const int p0 = blockIdx.y * pch;
  const int p1 = min(planes, p0 + pch);
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
                                                          int64_t npf, int64_t npc, int planes, int pch) {
  typedef typename Cx<Tc>::t C;
  const int64_t sc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sc >= npc) return;
  const int p0 = blockIdx.y * pch;
  const int p1 = min(planes, p0 + pch);
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

// u_f += P e_c (P = tensor product of 1D linear interpolation), one thread per coarse cell: cell (I[,J[,K]]), each index in
// [-1, mc-1], owns the fine points 2I+1 and 2I+2 per axis (0-based; 2I+1 sits on
// coarse point I, 2I+2 halfway between I and I+1), so every fine point is written
// exactly once; the 2^d corner values are loaded once and coarse values outside
// [0, mc) are the zero boundary.
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(256) mg_prolong_cell_kernel(const TU* __restrict__ ec, TU* __restrict__ uf, int mf,
                                                              int mc, int64_t npf, int64_t npc, int planes,
                                                              int pch) {
  typedef typename Cx<Tc>::t C;
  const int mc1 = mc + 1;
  const int64_t ncell = DIM == 2 ? (int64_t)mc1 * mc1 : (int64_t)mc1 * mc1 * mc1;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  const int p0 = blockIdx.y * pch;
  const int p1 = min(planes, p0 + pch);
  const int I = (int)(cell % mc1) - 1;
  const int J = (int)((cell / mc1) % mc1) - 1;
  const int K = DIM == 3 ? (int)(cell / ((int64_t)mc1 * mc1)) - 1 : 0;
  const Tc hf = Tc(0.5);
  for (int p = p0; p < p1; ++p) {
    const TU* ep = ec + (int64_t)p * npc;
    TU* up = uf + (int64_t)p * npf;
    C c[2][2][2];
#pragma unroll
    for (int a3 = 0; a3 < (DIM == 3 ? 2 : 1); ++a3)
#pragma unroll
      for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
        for (int a1 = 0; a1 < 2; ++a1) {
          const int i1 = I + a1, i2 = J + a2, i3 = K + a3;
          const bool in = i1 >= 0 && i1 < mc && i2 >= 0 && i2 < mc && (DIM == 2 || (i3 >= 0 && i3 < mc));
          c[a3][a2][a1] = in ? ldc(ep, DIM == 2 ? (int64_t)i2 * mc + i1 : ((int64_t)i3 * mc + i2) * mc + i1)
                             : czero<Tc>();
        }
    // interpolate along x1, then x2, then x3: e[o3][o2][o1], o = 0 -> coincident, 1 -> midpoint
    C e1[2][2][2];
#pragma unroll
    for (int a3 = 0; a3 < (DIM == 3 ? 2 : 1); ++a3)
#pragma unroll
      for (int a2 = 0; a2 < 2; ++a2) {
        e1[a3][a2][0] = c[a3][a2][0];
        e1[a3][a2][1] = cscale(c[a3][a2][0] + c[a3][a2][1], hf);
      }
    C e2[2][2][2];
#pragma unroll
    for (int a3 = 0; a3 < (DIM == 3 ? 2 : 1); ++a3)
#pragma unroll
      for (int o1 = 0; o1 < 2; ++o1) {
        e2[a3][0][o1] = e1[a3][0][o1];
        e2[a3][1][o1] = cscale(e1[a3][0][o1] + e1[a3][1][o1], hf);
      }
#pragma unroll
    for (int o3 = 0; o3 < (DIM == 3 ? 2 : 1); ++o3) {
      const int f3 = DIM == 3 ? 2 * K + 1 + o3 : 0;
      if (DIM == 3 && f3 < 0) continue;
#pragma unroll
      for (int o2 = 0; o2 < 2; ++o2) {
        const int f2 = 2 * J + 1 + o2;
        if (f2 < 0) continue;
#pragma unroll
        for (int o1 = 0; o1 < 2; ++o1) {
          const int f1 = 2 * I + 1 + o1;
          if (f1 < 0) continue;
          C v = e2[0][o2][o1];
          if (DIM == 3) v = o3 == 0 ? e2[0][o2][o1] : cscale(e2[0][o2][o1] + e2[1][o2][o1], hf);
          const int64_t q = DIM == 2 ? (int64_t)f2 * mf + f1 : ((int64_t)f3 * mf + f2) * mf + f1;
          stc(up, q, ldc(up, q) + v);
        }
      }
    }
  }
}

template <typename Tc, typename TU>
__global__ void mg_coarsest_kernel(const Tc* __restrict__ diag, const typename Cx<Tc>::t* __restrict__ sigma,
                                   const typename Cx<Tc>::t* __restrict__ r, TU* __restrict__ u, int planes) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= planes) return;
  stc(u, p, cmul(r[p], inv_diag<Tc>(sigma[p], diag[0])));
}

dim3 plane_grid(int64_t np, int planes, int pch) {
  return dim3((unsigned)((np + 255) / 256), (unsigned)((planes + pch - 1) / pch));
}

int plane_chunk(const Launch& L) {
  const int v = L.tiles ? L.tiles->pro_pch : 0;
  return v > 0 ? v : kPlaneChunk;
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
cudaError_t launch_fst_divide(Launch& L, const Grid& g, int planes, const Tc* lamK, const Tc* rmass,
                              const typename Cx<Tc>::t* sigma,
                              typename Cx<Tc>::t* buf) {
  const int64_t tot = g.np * planes;
  const double cs = sizeof(typename Cx<Tc>::t);
  L.begin(KC_FST_DIVIDE);
  fst_divide_kernel<Tc><<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(buf, lamK, rmass, sigma, g.np, planes);
  return L.end(KC_FST_DIVIDE, 2.0 * tot * cs, 12.0 * tot);
}

template <typename Tc, typename TU>
cudaError_t launch_mg_smooth(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                             const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u) {
  const int pch = plane_chunk(L);
  const double cs = 0.5 * (sizeof(typename Cx<Tc>::t) + sizeof(TU));
  const double tot = (double)g.np * planes;
  const dim3 grid = plane_grid(g.np, planes, pch);
  L.begin(KC_MG_SMOOTH);
  if (sizeof(Tc) == 8) {  // two passes: one reciprocal per point
    if (g.dim == 2) {
      mg_smooth_kernel<Tc, TU, 2, 1><<<grid, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np, planes, pch);
      mg_smooth_kernel<Tc, TU, 2, 2><<<grid, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np, planes, pch);
    } else {
      mg_smooth_kernel<Tc, TU, 3, 1><<<grid, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np, planes, pch);
      mg_smooth_kernel<Tc, TU, 3, 2><<<grid, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np, planes, pch);
    }
  } else {
    const int64_t pairs = (g.np / g.m) * ((g.m + 1) / 2);
    const dim3 pgrid((unsigned)((pairs + 255) / 256), (unsigned)((planes + pch - 1) / pch));
    if (g.dim == 2)
      mg_smooth_pair_kernel<Tc, TU, 2><<<pgrid, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np, planes, pch);
    else
      mg_smooth_pair_kernel<Tc, TU, 3><<<pgrid, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np, planes, pch);
  }
  return L.end(KC_MG_SMOOTH, 2.0 * tot * cs, tot * (12.0 + 10.0 * g.dim));
}

template <typename Tc, typename TU>
cudaError_t launch_mg_smooth_lex(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                                 const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u) {
  const double cs = 0.5 * (sizeof(typename Cx<Tc>::t) + sizeof(TU));
  const double tot = (double)g.np * planes;
  L.begin(KC_MG_SMOOTH);
  if (g.dim == 2)
    mg_smooth_lex_kernel<Tc, TU, 2><<<planes, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np);
  else
    mg_smooth_lex_kernel<Tc, TU, 3><<<planes, 256, 0, L.stream>>>(r, u, st.w, st.diag, sigma, g.m, g.np);
  return L.end(KC_MG_SMOOTH, 2.0 * tot * cs, tot * (6.0 + 4.0 * g.dim));
}

template <typename Tc, typename TU>
cudaError_t launch_mg_resid_restrict(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                                     const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, const TU* u,
                                     typename Cx<Tc>::t* res, typename Cx<Tc>::t* rc, bool rb_sweep) {
  const int pch = plane_chunk(L);
  const double cs = sizeof(typename Cx<Tc>::t);
  const int mc = (g.m - 1) / 2;
  const int64_t npc = g.dim == 2 ? (int64_t)mc * mc : (int64_t)mc * mc * mc;
  const double tot = (double)g.np * planes;
  L.begin(KC_MG_RESID_RESTRICT);
  double rbytes = 3.0 * tot * cs;
  bool done = false;
  if constexpr (std::is_same<TU, typename Cx<Tc>::t>::value) {
    if (rb_sweep) {
      // u is the red-black sweep from zero just made: its residual follows from the sweep's identity
      const int64_t pairs = (g.np / g.m) * ((g.m + 1) / 2);
      const dim3 pgrid((unsigned)((pairs + 255) / 256), (unsigned)((planes + pch - 1) / pch));
      if (g.dim == 2)
        mg_residual_pair_kernel<Tc, 2><<<pgrid, 256, 0, L.stream>>>(u, res, st.w, g.m, g.np, planes, pch);
      else
        mg_residual_pair_kernel<Tc, 3><<<pgrid, 256, 0, L.stream>>>(u, res, st.w, g.m, g.np, planes, pch);
      rbytes = 2.0 * tot * cs;
      done = true;
    }
  }
  if (!done) {
    if (g.dim == 2)
      mg_residual_kernel<Tc, TU, 2><<<plane_grid(g.np, planes, pch), 256, 0, L.stream>>>(r, u, res, st.w, st.diag,
                                                                                        sigma, g.m, g.np, planes, pch);
    else
      mg_residual_kernel<Tc, TU, 3><<<plane_grid(g.np, planes, pch), 256, 0, L.stream>>>(r, u, res, st.w, st.diag,
                                                                                        sigma, g.m, g.np, planes, pch);
  }
  cudaError_t e = L.end(KC_MG_RESID_RESTRICT, rbytes, tot * (8.0 + 4.0 * g.dim));
  if (e != cudaSuccess) return e;
  L.begin(KC_MG_RESID_RESTRICT);
  if (g.dim == 2)
    mg_restrict_kernel<Tc, 2><<<plane_grid(npc, planes, pch), 256, 0, L.stream>>>(res, rc, g.m, mc, g.np, npc, planes, pch);
  else
    mg_restrict_kernel<Tc, 3><<<plane_grid(npc, planes, pch), 256, 0, L.stream>>>(res, rc, g.m, mc, g.np, npc, planes, pch);
  return L.end(KC_MG_RESID_RESTRICT, tot * cs + (double)npc * planes * cs, (double)npc * planes * (g.dim == 2 ? 36 : 108));
}

template <typename Tc, typename TU>
cudaError_t launch_mg_prolong(Launch& L, const Grid& gf, int planes, const TU* ec, TU* uf) {
  const int pch = plane_chunk(L);
  const double cs = sizeof(TU);
  const int mc = (gf.m - 1) / 2;
  const int64_t npc = gf.dim == 2 ? (int64_t)mc * mc : (int64_t)mc * mc * mc;
  const double tot = (double)gf.np * planes;
  const int64_t ncell = gf.dim == 2 ? (int64_t)(mc + 1) * (mc + 1) : (int64_t)(mc + 1) * (mc + 1) * (mc + 1);
  L.begin(KC_MG_PROLONG);
  if (gf.dim == 2)
    mg_prolong_cell_kernel<Tc, TU, 2><<<plane_grid(ncell, planes, pch), 256, 0, L.stream>>>(ec, uf, gf.m, mc, gf.np, npc,
                                                                                      planes, pch);
  else
    mg_prolong_cell_kernel<Tc, TU, 3><<<plane_grid(ncell, planes, pch), 256, 0, L.stream>>>(ec, uf, gf.m, mc, gf.np, npc,
                                                                                      planes, pch);
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
  template cudaError_t launch_fst_divide<Tc>(Launch&, const Grid&, int, const Tc*, const Tc*, const Cx<Tc>::t*, Cx<Tc>::t*);
#define PCOPT_INST_MG(Tc, TU)                                                                                    \
  template cudaError_t launch_mg_smooth<Tc, TU>(Launch&, const Grid&, int, const Stencil<Tc>&, const Cx<Tc>::t*, \
                                                const Cx<Tc>::t*, TU*);                                             \
  template cudaError_t launch_mg_smooth_lex<Tc, TU>(Launch&, const Grid&, int, const Stencil<Tc>&,              \
                                                    const Cx<Tc>::t*, const Cx<Tc>::t*, TU*);                       \
  template cudaError_t launch_mg_resid_restrict<Tc, TU>(Launch&, const Grid&, int, const Stencil<Tc>&,           \
                                                        const Cx<Tc>::t*, const Cx<Tc>::t*, const TU*, Cx<Tc>::t*, \
                                                        Cx<Tc>::t*, bool);                                          \
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

// ---------------------------------------------------------------------------
// Coarse part of the V(1,0) cycle in one kernel.  From level l0 (the first one
// with few enough points) down to the one-point level and back, the cycle is
// launch- and latency-bound when run level by level; here one CTA owns one
// spectral plane and keeps every coarse level in shared memory.  The
// arithmetic is that of the per-level kernels above: red-black sweep from zero,
// residual, full weighting, exact one-point solve, linear prolongation.
// ---------------------------------------------------------------------------
namespace pcopt {
namespace {

template <int DIM>
__device__ __forceinline__ int64_t lin(int i1, int i2, int i3, int m) {
  return DIM == 2 ? (int64_t)i2 * m + i1 : ((int64_t)i3 * m + i2) * m + i1;
}

// one plane per CTA; in FP32, 1024 threads give about one point per thread on the
// largest coarse level (31^2), so each of the cycle's ~20 dependent phases is short
// (FP64 is bound by its arithmetic and runs faster with 256)
template <typename Tc>
constexpr int coarse_threads() {
  return sizeof(Tc) == 4 ? 1024 : 256;
}

// For odd m the parity of the linear index s = i1 + m i2 (+ m^2 i3) is that of
// i1 + i2 (+ i3), so red points (i1 + i2 + i3 + DIM even) are s = DIM mod 2,
// DIM mod 2 + 2, ... and each colour is swept without idle threads.  With `stage`
// the coarse levels' face weights and diagonals are copied into shared memory once.
template <typename Tc, typename TU, int DIM>
__global__ void __launch_bounds__(1024) mg_coarse_cycle_kernel(const CoarseLevels<Tc> lv,
                                                              const typename Cx<Tc>::t* __restrict__ r0,
                                                              TU* __restrict__ u0,
                                                              const typename Cx<Tc>::t* __restrict__ sigma,
                                                              int stage) {
  typedef typename Cx<Tc>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const C sig = sigma[p];
  C* rl[kMaxCoarseLevels];
  TU* ul[kMaxCoarseLevels];
  C* resl[kMaxCoarseLevels];
  const Tc* wl[kMaxCoarseLevels];
  const Tc* dl[kMaxCoarseLevels];
  {
    unsigned char* q = smem_raw;
    for (int l = 0; l < lv.count; ++l) {
      const int np = (int)lv.np[l];
      rl[l] = reinterpret_cast<C*>(q);
      q += (size_t)np * sizeof(C);
      resl[l] = reinterpret_cast<C*>(q);
      q += (size_t)np * sizeof(C);
      ul[l] = reinterpret_cast<TU*>(q);
      q += (((size_t)np * sizeof(TU) + 15) / 16) * 16;
    }
    for (int l = 0; l < lv.count; ++l) {
      const int np = (int)lv.np[l];
      if (stage) {
        Tc* w = reinterpret_cast<Tc*>(q);
        q += (((size_t)(2 * DIM + 1) * np * sizeof(Tc) + 15) / 16) * 16;
        for (int e = tid; e < 2 * DIM * np; e += nt) w[e] = lv.w[l][e];
        for (int e = tid; e < np; e += nt) w[2 * DIM * np + e] = lv.diag[l][e];
        wl[l] = w;
        dl[l] = w + 2 * DIM * np;
      } else {
        wl[l] = lv.w[l];
        dl[l] = lv.diag[l];
      }
    }
  }
  // level 0 of the coarse part comes from global memory
  const int np0 = (int)lv.np[0];
  for (int s = tid; s < np0; s += nt) rl[0][s] = r0[(int64_t)p * np0 + s];
  __syncthreads();
  constexpr int red0 = DIM & 1;
  for (int l = 0; l + 1 < lv.count; ++l) {
    const int m = lv.m[l];
    const int np = (int)lv.np[l];
    const Tc* w = wl[l];
    const Tc* dg = dl[l];
    // red points: u = r / d ; black points wait for them
    for (int s = red0 + 2 * tid; s < np; s += 2 * nt) stc(ul[l], s, cmul(rl[l][s], inv_shift_c(sig, dg[s])));
    __syncthreads();
    for (int s = 1 - red0 + 2 * tid; s < np; s += 2 * nt) {
      const int i1 = s % m;
      const int rr = s / m;
      const int i2 = DIM == 2 ? rr : rr % m;
      const int i3 = DIM == 3 ? rr / m : 0;
      const int off[6] = {-1, 1, -m, m, -m * m, m * m};
      const bool ex[6] = {i1 > 0, i1 < m - 1, i2 > 0, i2 < m - 1, i3 > 0, i3 < m - 1};
      C acc = rl[l][s];
#pragma unroll
      for (int k = 0; k < 2 * DIM; ++k) {
        if (ex[k]) {
          const C ured = ldc(ul[l], s + off[k]);
          const Tc wk = w[k * np + s];
          acc.x = fma(wk, ured.x, acc.x);
          acc.y = fma(wk, ured.y, acc.y);
        }
      }
      stc(ul[l], s, cmul(acc, inv_shift_c(sig, dg[s])));
    }
    __syncthreads();
    // residual res = r - (sigma u + tau K u)
    for (int s = tid; s < np; s += nt) {
      const int i1 = s % m;
      const int rr = s / m;
      const int i2 = DIM == 2 ? rr : rr % m;
      const int i3 = DIM == 3 ? rr / m : 0;
      const int off[6] = {-1, 1, -m, m, -m * m, m * m};
      const bool ex[6] = {i1 > 0, i1 < m - 1, i2 > 0, i2 < m - 1, i3 > 0, i3 < m - 1};
      const C uc = ldc(ul[l], s);
      C lu = cmul(cmk<Tc>(sig.x + dg[s], sig.y), uc);
#pragma unroll
      for (int k = 0; k < 2 * DIM; ++k) {
        if (ex[k]) {
          const C un = ldc(ul[l], s + off[k]);
          const Tc wk = w[k * np + s];
          lu.x = fma(-wk, un.x, lu.x);
          lu.y = fma(-wk, un.y, lu.y);
        }
      }
      resl[l][s] = rl[l][s] - lu;
    }
    __syncthreads();
    // full weighting onto level l + 1
    const int mc = lv.m[l + 1];
    const int npc = (int)lv.np[l + 1];
    const Tc wt[3] = {Tc(0.25), Tc(0.5), Tc(0.25)};
    for (int sc = tid; sc < npc; sc += nt) {
      const int c1 = sc % mc;
      const int rr = sc / mc;
      const int c2 = DIM == 2 ? rr : rr % mc;
      const int c3 = DIM == 3 ? rr / mc : 0;
      const int f1 = 2 * c1 + 1, f2 = 2 * c2 + 1, f3 = 2 * c3 + 1;
      C acc = czero<Tc>();
      for (int o3 = (DIM == 3 ? -1 : 0); o3 <= (DIM == 3 ? 1 : 0); ++o3)
#pragma unroll
        for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
          for (int o1 = -1; o1 <= 1; ++o1) {
            Tc wgt = wt[o1 + 1] * wt[o2 + 1];
            if (DIM == 3) wgt *= wt[o3 + 1];
            const C v = resl[l][(int)lin<DIM>(f1 + o1, f2 + o2, f3 + o3, m)];
            acc.x = fma(wgt, v.x, acc.x);
            acc.y = fma(wgt, v.y, acc.y);
          }
      rl[l + 1][sc] = acc;
    }
    __syncthreads();
  }
  // one-point level
  {
    const int l = lv.count - 1;
    if (tid == 0) stc(ul[l], 0, cmul(rl[l][0], inv_shift_c(sig, dl[l][0])));
    __syncthreads();
  }
  // prolongation and correction back up
  for (int l = lv.count - 2; l >= 0; --l) {
    const int mf = lv.m[l], mc = lv.m[l + 1];
    const int npf = (int)lv.np[l];
    for (int s = tid; s < npf; s += nt) {
      const int fi[3] = {s % mf, DIM == 2 ? s / mf : (s / mf) % mf, DIM == 3 ? s / mf / mf : 0};
      int ci[3][2];
      Tc cw[3][2];
      int cnt[3] = {1, 1, 1};
      ci[2][0] = 0;
      cw[2][0] = Tc(1);
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
      C acc = czero<Tc>();
      for (int a3 = 0; a3 < cnt[2]; ++a3)
        for (int a2 = 0; a2 < cnt[1]; ++a2)
          for (int a1 = 0; a1 < cnt[0]; ++a1) {
            const Tc wgt = cw[0][a1] * cw[1][a2] * cw[2][a3];
            const C v = ldc(ul[l + 1], (int)lin<DIM>(ci[0][a1], ci[1][a2], ci[2][a3], mc));
            acc.x = fma(wgt, v.x, acc.x);
            acc.y = fma(wgt, v.y, acc.y);
          }
      stc(ul[l], s, ldc(ul[l], s) + acc);
    }
    __syncthreads();
  }
  for (int s = tid; s < np0; s += nt) stc(u0, (int64_t)p * np0 + s, ldc(ul[0], s));
}

}  // namespace

template <typename Tc, typename TU>
size_t mg_coarse_cycle_smem(const CoarseLevels<Tc>& lv) {
  size_t b = 0;
  for (int l = 0; l < lv.count; ++l)
    b += 2 * (size_t)lv.np[l] * sizeof(typename Cx<Tc>::t) + (((size_t)lv.np[l] * sizeof(TU) + 15) / 16) * 16;
  return b;
}

// shared memory of the staged face weights and diagonals of all coarse levels
template <typename Tc>
static size_t coarse_coef_smem(const CoarseLevels<Tc>& lv, int dim) {
  size_t b = 0;
  for (int l = 0; l < lv.count; ++l) b += (((size_t)(2 * dim + 1) * lv.np[l] * sizeof(Tc) + 15) / 16) * 16;
  return b;
}

template <typename Tc, typename TU>
cudaError_t launch_mg_coarse_cycle(Launch& L, int dim, int planes, const CoarseLevels<Tc>& lv,
                                   const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r0, TU* u0) {
  // stage the coefficients too when everything fits beside the levels
  const size_t base = mg_coarse_cycle_smem<Tc, TU>(lv);
  const size_t coef = coarse_coef_smem<Tc>(lv, dim);
  const int stage = base + coef <= 200 * 1024 ? 1 : 0;
  const size_t smem = base + (stage ? coef : 0);
  cudaError_t e;
  if (dim == 2)
    e = cudaFuncSetAttribute(mg_coarse_cycle_kernel<Tc, TU, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else
    e = cudaFuncSetAttribute(mg_coarse_cycle_kernel<Tc, TU, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  double pts = 0;
  for (int l = 0; l < lv.count; ++l) pts += (double)lv.np[l];
  const double cs = sizeof(typename Cx<Tc>::t);
  L.begin(KC_MG_COARSE);
  if (dim == 2)
    mg_coarse_cycle_kernel<Tc, TU, 2><<<planes, coarse_threads<Tc>(), smem, L.stream>>>(lv, r0, u0, sigma, stage);
  else
    mg_coarse_cycle_kernel<Tc, TU, 3><<<planes, coarse_threads<Tc>(), smem, L.stream>>>(lv, r0, u0, sigma, stage);
  return L.end(KC_MG_COARSE, (double)planes * lv.np[0] * (cs + sizeof(TU)), (double)planes * pts * 60.0);
}

#define PCOPT_INST_CC(Tc, TU)                                                                              \
  template cudaError_t launch_mg_coarse_cycle<Tc, TU>(Launch&, int, int, const CoarseLevels<Tc>&,         \
                                                      const Cx<Tc>::t*, const Cx<Tc>::t*, TU*);            \
  template size_t mg_coarse_cycle_smem<Tc, TU>(const CoarseLevels<Tc>&);
PCOPT_INST_CC(float, float2)
PCOPT_INST_CC(double, double2)
PCOPT_INST_CC(float, __nv_bfloat162)
#undef PCOPT_INST_CC

}  // namespace pcopt
