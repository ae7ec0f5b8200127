// Scaled FFT along time: steps 1 and 3-4 of the four-step apply of
// P_eps^{-1} (Section 2.1), with C_{eps,n} = D^{-1} F Lambda F^* D
// (Eq. decomposition_eps), D = diag(eps^{j/n}), lambda_k = 1 - eps^{1/n} theta^{-k}.
//
// C_{eps,n} is Toeplitz, so its transpose is C^T = J C J with J the reversal of the
// time index, and (C^T + alpha I)^{-1} v1 = J (C + alpha I)^{-1} J v1: both halves go
// through the same transform,
//   half 1 (block C_eps^T + alpha I):  hat v1 = fft(D J v1), shifts lambda_k + alpha,
//   half 2 (block C_eps   + alpha I):  hat v2 = fft(D v2),   shifts lambda_k + alpha,
// inverted by D^{-1} ifft(.) (and J again for half 1).  The two real halves are
// packed into one complex sequence z = D J v1 + i D v2 (two-for-one) and only the
// Hermitian half k = 0..n/2 is kept: spectral plane 2k holds hat v2[k], plane 2k+1
// hat v1[k], and both planes of a pair share sigma_k = lambda_k + alpha.  The two
// parts of z carry the same scaling eps^{j/n} at every j, so the packing costs no
// accuracy.  (Packing D^{-1} v1 with D v2 instead, the form C^T = D F conj(Lambda)
// F^* D^{-1} suggests, mixes parts whose ratio reaches eps^{-2}: the smaller part then
// keeps only about u / eps^2 of relative accuracy, which ruins an FP32 transform at
// the paper's eps = tau/2.)
//
// One CTA owns TS consecutive spatial points and the whole time axis: it
// reads n rows of TS values per half (coalesced along space), runs an
// in-place radix-2 FFT of length n in shared memory for all TS columns
// (threads of a warp work on consecutive columns: conflict-free), and writes
// frequency-major planes (the time<->space transpose happens in shared memory).
#include <algorithm>

#include "common.cuh"
#include "regfft.cuh"

namespace pcopt {

namespace {

__device__ __forceinline__ int bitrev(int j, int logn) { return logn ? (int)(__brev((unsigned)j) >> (32 - logn)) : 0; }

// Parents of fine point s in the next coarser level and their linear weights,
// per axis: odd f sits on coarse point (f-1)/2 (weight 1), even f halfway between
// f/2-1 and f/2 (1/2 each, a parent outside [0, mc) is the zero boundary).
template <typename Tc, typename TU>
struct Parents {
  int o[3][2];
  Tc wt[3][2];
  __device__ __forceinline__ void init(const FineCorrection<TU>& fc, int64_t s) {
    int f[3];
    f[0] = (int)(s % fc.mf);
    const int64_t r = s / fc.mf;
    f[1] = (int)(fc.dim == 2 ? r : r % fc.mf);
    f[2] = fc.dim == 3 ? (int)(r / fc.mf) : 0;
    int stride = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= fc.dim) {
        o[a][0] = o[a][1] = 0;
        wt[a][0] = Tc(1);
        wt[a][1] = Tc(0);
        continue;
      }
      if (f[a] & 1) {
        o[a][0] = o[a][1] = ((f[a] - 1) >> 1) * stride;
        wt[a][0] = Tc(1);
        wt[a][1] = Tc(0);
      } else {
        int lo = (f[a] >> 1) - 1, hi = f[a] >> 1;
        wt[a][0] = lo >= 0 ? Tc(0.5) : Tc(0);
        wt[a][1] = hi < fc.mc ? Tc(0.5) : Tc(0);
        if (lo < 0) lo = hi;
        if (hi >= fc.mc) hi = lo;
        o[a][0] = lo * stride;
        o[a][1] = hi * stride;
      }
      stride *= fc.mc;
    }
  }
  __device__ __forceinline__ typename Cx<Tc>::t at(const FineCorrection<TU>& fc, int p) const {
    typedef typename Cx<Tc>::t C;
    const TU* e = fc.ec + (int64_t)p * fc.npc;
    C acc = czero<Tc>();
    for (int c2 = 0; c2 < (fc.dim == 3 ? 2 : 1); ++c2)
#pragma unroll
      for (int c1 = 0; c1 < 2; ++c1)
#pragma unroll
        for (int c0 = 0; c0 < 2; ++c0) {
          const Tc w = wt[2][c2] * wt[1][c1] * wt[0][c0];
          if (w != Tc(0)) {
            const C v = ldc(e, o[2][c2] + o[1][c1] + o[0][c0]);
            acc.x = fma(w, v.x, acc.x);
            acc.y = fma(w, v.y, acc.y);
          }
        }
    return acc;
  }
};

template <typename Tc, bool INVERSE>
__device__ __forceinline__ void fft_columns(typename Cx<Tc>::t* z, const typename Cx<Tc>::t* __restrict__ tw, int n,
                                            int TS) {
  typedef typename Cx<Tc>::t C;
  for (int half = 1, st = n >> 1; half < n; half <<= 1, st >>= 1) {
    const int nb = (n >> 1) * TS;
    for (int e = threadIdx.x; e < nb; e += blockDim.x) {
      const int bi = e / TS;
      const int c = e - bi * TS;
      const int pos = bi & (half - 1);
      const int i0 = ((bi - pos) << 1) + pos;
      const int i1 = i0 + half;
      C W = tw[pos * st];
      if (INVERSE) W.y = -W.y;
      const C a = z[i0 * TS + c];
      const C b = cmul(W, z[i1 * TS + c]);
      z[i0 * TS + c] = a + b;
      z[i1 * TS + c] = a - b;
    }
    __syncthreads();
  }
}

template <typename Tc, typename Tin>
__global__ void __launch_bounds__(256) tfft_forward_kernel(const Tin* __restrict__ v, const Tc* __restrict__ dpow,
                                                           const typename Cx<Tc>::t* __restrict__ tw,
                                                           typename Cx<Tc>::t* __restrict__ spec, int64_t ms, int n,
                                                           int logn, int TS) {
  typedef typename Cx<Tc>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* z = reinterpret_cast<C*>(smem_raw);
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const Tin* v1 = v;
  const Tin* v2 = v + (int64_t)n * ms;
  for (int e = threadIdx.x; e < n * TS; e += blockDim.x) {
    const int j = e / TS;
    const int c = e - j * TS;
    const int64_t s = s0 + c;
    Tc a = Tc(0), b = Tc(0);
    if (s < ms) {
      const Tc d = dpow[j];
      a = cvt<Tc>(v1[(int64_t)(n - 1 - j) * ms + s]) * d;  // D J v1
      b = cvt<Tc>(v2[(int64_t)j * ms + s]) * d;            // D v2
    }
    z[bitrev(j, logn) * TS + c] = cmk<Tc>(a, b);
  }
  __syncthreads();
  fft_columns<Tc, false>(z, tw, n, TS);
  const int nf = n / 2 + 1;
  const Tc hf = Tc(0.5);
  for (int e = threadIdx.x; e < nf * TS; e += blockDim.x) {
    const int k = e / TS;
    const int c = e - k * TS;
    const int64_t s = s0 + c;
    if (s >= ms) continue;
    const C Z = z[k * TS + c];
    const C W = z[((n - k) & (n - 1)) * TS + c];
    // hat v2[k] = (Z[k] - conj Z[n-k]) / (2i);  hat v1[k] = (Z[k] + conj Z[n-k]) / 2
    spec[(int64_t)(2 * k) * ms + s] = cmk<Tc>((Z.y + W.y) * hf, (W.x - Z.x) * hf);
    spec[(int64_t)(2 * k + 1) * ms + s] = cmk<Tc>((Z.x + W.x) * hf, (Z.y - W.y) * hf);
  }
}

template <typename Tc, typename TU, typename Tout>
__global__ void __launch_bounds__(256) tfft_inverse_kernel(const TU* __restrict__ spec,
                                                           const Tc* __restrict__ dpow,
                                                           const typename Cx<Tc>::t* __restrict__ tw,
                                                           Tout* __restrict__ w, int64_t ms, int n, int logn,
                                                           int TS, FineCorrection<TU> fc) {
  typedef typename Cx<Tc>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* z = reinterpret_cast<C*>(smem_raw);
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const int nf = n / 2 + 1;
  for (int e = threadIdx.x; e < nf * TS; e += blockDim.x) {
    const int k = e / TS;
    const int c = e - k * TS;
    const int64_t s = s0 + c;
    C sa = czero<Tc>(), sb = czero<Tc>();
    if (s < ms) {
      sa = ldc(spec, (int64_t)(2 * k) * ms + s);      // hat w2[k]
      sb = ldc(spec, (int64_t)(2 * k + 1) * ms + s);  // hat w1[k]
      if (fc.ec) {
        Parents<Tc, TU> par;
        par.init(fc, s);
        sa = sa + par.at(fc, 2 * k);
        sb = sb + par.at(fc, 2 * k + 1);
      }
    }
    // Y[k] = hat w1[k] + i hat w2[k] with hat w1[k] = sb, hat w2[k] = sa
    z[bitrev(k, logn) * TS + c] = cmk<Tc>(sb.x - sa.y, sb.y + sa.x);
    if (k > 0 && 2 * k < n) {
      // Y[n-k] = conj(hat w1[k]) + i conj(hat w2[k]) (real halves)
      z[bitrev(n - k, logn) * TS + c] = cmk<Tc>(sb.x + sa.y, sa.x - sb.y);
    }
  }
  __syncthreads();
  fft_columns<Tc, true>(z, tw, n, TS);
  const Tc inv_n = Tc(1) / Tc(n);
  Tout* w1 = w;
  Tout* w2 = w + (int64_t)n * ms;
  for (int e = threadIdx.x; e < n * TS; e += blockDim.x) {
    const int j = e / TS;
    const int c = e - j * TS;
    const int64_t s = s0 + c;
    if (s >= ms) continue;
    const int jr = n - 1 - j;
    const Tc wt1 = (z[jr * TS + c].x * inv_n) / dpow[jr];  // J D^{-1} ifft(hat w1)
    const Tc wt2 = (z[j * TS + c].y * inv_n) / dpow[j];    // D^{-1} ifft(hat w2)
    w1[(int64_t)j * ms + s] = cvt<Tout>(wt1 - wt2);   // step 4: [[I, -I], [I, I]]
    w2[(int64_t)j * ms + s] = cvt<Tout>(wt1 + wt2);
  }
}

// ---------------------------------------------------------------------------
// Four-step FFT in registers (n = N1 * N2 <= 1024): the kernels used in practice.
// Forward X[k] = sum_j x[j] w^{jk}, w = exp(-2 pi i / n), j = j1 + N1 j2,
// k = k2 + N2 k1:  (A) an N2-point DFT over j2 per j1, (B) the twiddle
// w^{j1 k2}, (C) an N1-point DFT over j1 per k2.  The inverse uses the same
// split with k = k1 + N1 k2, j = j2 + N2 j1 and conjugate twiddles.  Each of
// the N1 thread rows of a CTA owns one j1 (then one k2) of COLS = 256/N1
// spatial columns: two register FFTs and one shared-memory exchange instead of
// log2(n) shared-memory radix-2 stages.
// Forward transform of one tile of COLS = 256 / N1 columns.  ld(j, a, b) gives
// v1[n-1-j] and v2[j] of the thread's column (zero outside the grid).  Returns after
// the spectrum stores; the caller's barrier orders the reuse of `sm`.
template <typename Tc, int N1, int N2, typename Ld>
__device__ __forceinline__ void fwd4_body(Ld&& ld, const Tc* __restrict__ dpow, const Tc* __restrict__ dinv,
                                          const typename Cx<Tc>::t* __restrict__ tw,
                                          typename Cx<Tc>::t* __restrict__ spec, typename Cx<Tc>::t* sm,
                                          int64_t ms, int64_t s, bool valid, int r, int c) {
  typedef typename Cx<Tc>::t C;
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  // (A) rows j = r + N1 j2: z = D J v1 + i D v2, N2-point DFT over j2
  C x[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    const int j = r + N1 * j2;
    Tc a, b;
    PC_DOK(j < n && c < COLS && (!valid || s < ms), 301);
    ld(j, a, b);
    x[j2] = cmk<Tc>(a * dpow[j], b * dpow[j]);
  }
  reg_fft<N2, false>(x, tw, N1);
  // (B) twiddle w^{j1 k2}, stored as Y[k2][j1]
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const C y = (k2 == 0 || r == 0) ? x[k2] : cmul(tw[r * k2], x[k2]);
    sm[(k2 * N1 + r) * COLS + c] = y;
  }
  __syncthreads();
  // (C) row k2 = r (< N2): N1-point DFT over j1, X[k2 + N2 k1]
  C y[N1];
  if (r < N2) {
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) y[j1] = sm[(r * N1 + j1) * COLS + c];
  }
  __syncthreads();
  if (r < N2) {
    reg_fft<N1, false>(y, tw, N2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) sm[(r + N2 * k1) * COLS + c] = y[k1];
  }
  __syncthreads();
  if (valid) {
    // Hermitian split of the two-for-one spectrum, k = 0..n/2
    const Tc hf = Tc(0.5);
    constexpr int NI = (n / 2) / N1 + 1;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int k = r + N1 * i;
      if (k <= n / 2) {
        const C Z = sm[k * COLS + c];
        const C W = sm[((n - k) & (n - 1)) * COLS + c];
        // hat v2[k] = (Z[k] - conj Z[n-k]) / (2i),  hat v1[k] = (Z[k] + conj Z[n-k]) / 2
        spec[(int64_t)(2 * k) * ms + s] = cmk<Tc>((Z.y + W.y) * hf, (W.x - Z.x) * hf);
        spec[(int64_t)(2 * k + 1) * ms + s] = cmk<Tc>((Z.x + W.x) * hf, (Z.y - W.y) * hf);
      }
    }
  }
}

// Inverse transform, D scalings and the [[I, -I], [I, I]] butterfly of one tile.
// ld(k, sa, sb) gives spectral planes 2k and 2k+1 of the thread's column (zero
// outside the grid).  Returns after the output stores.
template <typename Tc, typename Tout, int N1, int N2, typename Ld>
__device__ __forceinline__ void inv4_body(Ld&& ld, const Tc* __restrict__ dpow, const Tc* __restrict__ dinv,
                                          const typename Cx<Tc>::t* __restrict__ tw, Tout* __restrict__ w,
                                          typename Cx<Tc>::t* sm, int64_t ms, int64_t s, bool valid, int r,
                                          int c) {
  typedef typename Cx<Tc>::t C;
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  // Y[k] = hat w1[k] + i hat w2[k] for all k from the half spectrum (a fixed trip
  // count, so all of a thread's loads are in flight together)
  constexpr int NI = (n / 2) / N1 + 1;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int k = r + N1 * i;
    if (k <= n / 2) {
      C sa, sb;
      ld(k, sa, sb);
      // Y[k] = hat w1[k] + i hat w2[k] (sb = hat w1[k], sa = hat w2[k]);
      // Y[n-k] = conj(hat w1[k]) + i conj(hat w2[k]) (real halves)
      sm[k * COLS + c] = cmk<Tc>(sb.x - sa.y, sb.y + sa.x);
      if (k > 0 && 2 * k < n) sm[(n - k) * COLS + c] = cmk<Tc>(sb.x + sa.y, sa.x - sb.y);
    }
  }
  __syncthreads();
  // (A) row k1 = r: N2-point inverse DFT over k2 of Y[k1 + N1 k2], twiddle w^{-k1 j2}
  C x[N2];
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) x[k2] = sm[(r + N1 * k2) * COLS + c];
  __syncthreads();
  reg_fft<N2, true>(x, tw, N1);
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    C t = tw[r * j2];
    t.y = -t.y;
    sm[(j2 * N1 + r) * COLS + c] = (j2 == 0 || r == 0) ? x[j2] : cmul(t, x[j2]);
  }
  __syncthreads();
  // (C) row j2 = r: N1-point inverse DFT over k1 -> z[j2 + N2 j1]
  C y[N1];
  if (r < N2) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) y[k1] = sm[(r * N1 + k1) * COLS + c];
  }
  __syncthreads();  // every read of the exchange is done before sm is rewritten
  if (r < N2) {
    reg_fft<N1, true>(y, tw, N2);
    const Tc inv_n = Tc(1) / Tc(n);
    // half 1 belongs to time n-1-j (J D^{-1} ifft(hat w1)), half 2 to time j
    // (D^{-1} ifft(hat w2)): meet in shared memory for the butterfly
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int j = r + N2 * j1;
      sm[(n - 1 - j) * COLS + c].x = dinv[j] * (y[j1].x * inv_n);
      sm[j * COLS + c].y = dinv[j] * (y[j1].y * inv_n);
    }
  }
  __syncthreads();
  if (r < N2 && valid) {
    Tout* w1 = w;
    Tout* w2 = w + (int64_t)n * ms;
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int j = r + N2 * j1;
      const C t = sm[j * COLS + c];
      w1[(int64_t)j * ms + s] = cvt<Tout>(t.x - t.y);  // step 4: [[I, -I], [I, I]]
      w2[(int64_t)j * ms + s] = cvt<Tout>(t.x + t.y);
    }
  }
}

// FP64 transforms of up to 256 points are compiled for two CTAs per SM (128 registers):
// their arithmetic bounds them, and a second CTA hides the FP64 and shared-memory latency
template <typename Tc, int NP>
constexpr int tfft_fp64_blocks() {
  return (sizeof(Tc) == 8 && NP <= 256) ? 2 : 1;
}

// one CTA per tile, inputs loaded straight into registers
template <typename Tin, typename Tc, int N1, int N2>
__global__ void __launch_bounds__(256) tfft4_forward_kernel(const Tin* __restrict__ v, const Tc* __restrict__ dpow,
                                                            const Tc* __restrict__ dinv,
                                                            const typename Cx<Tc>::t* __restrict__ tw,
                                                            typename Cx<Tc>::t* __restrict__ spec, int64_t ms,
                                                            size_t vstride, const int* __restrict__ jdev) {
  typedef typename Cx<Tc>::t C;
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);  // [n][COLS]
  const int c = threadIdx.x % COLS;
  const int r = threadIdx.x / COLS;  // 0..N1-1
  const int64_t s = (int64_t)blockIdx.x * COLS + c;
  const bool valid = s < ms;
  if (jdev) v += (size_t)(*jdev) * vstride;  // input = basis vector j (device-resident index)
  const Tin* v1 = v;
  const Tin* v2 = v + (int64_t)n * ms;
  fwd4_body<Tc, N1, N2>(
      [&](int j, Tc& a, Tc& b) {
        a = valid ? cvt<Tc>(v1[(int64_t)(n - 1 - j) * ms + s]) : Tc(0);
        b = valid ? cvt<Tc>(v2[(int64_t)j * ms + s]) : Tc(0);
      },
      dpow, dinv, tw, spec, sm, ms, s, valid, r, c);
}

// the same for FP64 transforms of up to 256 points, compiled for two CTAs per SM
// (128 registers): their FP64 arithmetic bounds them, and a second CTA hides latency
template <typename Tin, int N1, int N2>
__global__ void __launch_bounds__(256, 2) tfft4_forward_f64_kernel(const Tin* __restrict__ v,
                                                                   const double* __restrict__ dpow,
                                                                   const double* __restrict__ dinv,
                                                                   const double2* __restrict__ tw,
                                                                   double2* __restrict__ spec, int64_t ms,
                                                                   size_t vstride, const int* __restrict__ jdev) {
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sm = reinterpret_cast<double2*>(smem_raw);  // [n][COLS]
  const int c = threadIdx.x % COLS;
  const int r = threadIdx.x / COLS;
  const int64_t s = (int64_t)blockIdx.x * COLS + c;
  const bool valid = s < ms;
  if (jdev) v += (size_t)(*jdev) * vstride;
  const Tin* v1 = v;
  const Tin* v2 = v + (int64_t)n * ms;
  fwd4_body<double, N1, N2>(
      [&](int j, double& a, double& b) {
        a = valid ? cvt<double>(v1[(int64_t)(n - 1 - j) * ms + s]) : 0.0;
        b = valid ? cvt<double>(v2[(int64_t)j * ms + s]) : 0.0;
      },
      dpow, dinv, tw, spec, sm, ms, s, valid, r, c);
}

// Persistent streaming variant: each CTA walks tiles blockIdx.x, + gridDim.x, ...
// and copies the next tile's 2n x COLS inputs into a second shared-memory stage
// with cp.async while it transforms the current one.
template <typename Tin, typename Tc, int N1, int N2>
__global__ void __launch_bounds__(256) tfft4s_forward_kernel(const Tin* __restrict__ v, const Tc* __restrict__ dpow,
                                                             const Tc* __restrict__ dinv,
                                                             const typename Cx<Tc>::t* __restrict__ tw,
                                                             typename Cx<Tc>::t* __restrict__ spec, int64_t ms,
                                                             int ntiles, size_t vstride, const int* __restrict__ jdev) {
  typedef typename Cx<Tc>::t C;
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  constexpr int TILE = 2 * n * COLS;  // rows 0..n-1: v1, n..2n-1: v2 (v2 = v1 + n ms)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tin* stage = reinterpret_cast<Tin*>(smem_raw);  // [2][2n][COLS]
  C* sm = reinterpret_cast<C*>(stage + 2 * TILE);  // [n][COLS]
  const int c = threadIdx.x % COLS;
  const int r = threadIdx.x / COLS;
  if (jdev) v += (size_t)(*jdev) * vstride;
  auto issue = [&](int tile, int buf) {
    Tin* dst = stage + buf * TILE;
    const int64_t s0 = (int64_t)tile * COLS;
    for (int e = threadIdx.x; e < TILE; e += 256) {
      const int cc = e % COLS;
      const int row = e / COLS;
      const bool ok = s0 + cc < ms;
      cp_async<sizeof(Tin)>(dst + e, v + (int64_t)row * ms + (ok ? s0 + cc : 0), ok);
    }
    cp_async_commit();
  };
  if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  int buf = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    if (t + (int)gridDim.x < ntiles)
      issue(t + gridDim.x, buf ^ 1);
    else
      cp_async_commit();  // empty group: the wait below always leaves one pending
    cp_async_wait<1>();
    __syncthreads();
    const Tin* st = stage + buf * TILE;
    const int64_t s = (int64_t)t * COLS + c;
    fwd4_body<Tc, N1, N2>(
        [&](int j, Tc& a, Tc& b) {
          a = cvt<Tc>(st[(n - 1 - j) * COLS + c]);
          b = cvt<Tc>(st[(n + j) * COLS + c]);
        },
        dpow, dinv, tw, spec, sm, ms, s, s < ms, r, c);
    __syncthreads();  // stage[buf] and sm are rewritten next
  }
  cp_async_wait<0>();
}

template <typename Tc, typename TU, typename Tout, int N1, int N2>
__global__ void __launch_bounds__(256, (sizeof(Tc) == 4 && N1 * N2 <= 256) ? 4 : tfft_fp64_blocks<Tc, N1 * N2>()) tfft4_inverse_kernel(const TU* __restrict__ spec, const Tc* __restrict__ dpow,
                                                            const Tc* __restrict__ dinv,
                                                            const typename Cx<Tc>::t* __restrict__ tw,
                                                            Tout* __restrict__ w, int64_t ms, size_t wstride,
                                                            const int* __restrict__ jdev, FineCorrection<TU> fc) {
  typedef typename Cx<Tc>::t C;
  constexpr int COLS = 256 / N1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);  // [n][COLS]
  const int c = threadIdx.x % COLS;
  const int r = threadIdx.x / COLS;
  const int64_t s = (int64_t)blockIdx.x * COLS + c;
  const bool valid = s < ms;
  if (jdev) w += (size_t)(*jdev) * wstride;  // output = basis vector j
  Parents<Tc, TU> par;
  if (fc.ec && valid) par.init(fc, s);
  inv4_body<Tc, Tout, N1, N2>(
      [&](int k, C& sa, C& sb) {
        sa = czero<Tc>();
        sb = czero<Tc>();
        if (valid) {
          sa = ldc(spec, (int64_t)(2 * k) * ms + s);
          sb = ldc(spec, (int64_t)(2 * k + 1) * ms + s);
          if (fc.ec) {
            sa = sa + par.at(fc, 2 * k);
            sb = sb + par.at(fc, 2 * k + 1);
          }
        }
      },
      dpow, dinv, tw, w, sm, ms, s, valid, r, c);
}

// Persistent streaming inverse: the next tile's 2 (n/2 + 1) spectral planes are
// copied into a second stage with cp.async while the current tile is transformed.
template <typename Tc, typename TU, typename Tout, int N1, int N2>
__global__ void __launch_bounds__(256) tfft4s_inverse_kernel(const TU* __restrict__ spec, const Tc* __restrict__ dpow,
                                                             const Tc* __restrict__ dinv,
                                                             const typename Cx<Tc>::t* __restrict__ tw,
                                                             Tout* __restrict__ w, int64_t ms, int ntiles,
                                                             size_t wstride, const int* __restrict__ jdev,
                                                             FineCorrection<TU> fc) {
  typedef typename Cx<Tc>::t C;
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  constexpr int NP = 2 * (n / 2 + 1);  // spectral planes
  constexpr int TILE = NP * COLS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TU* stage = reinterpret_cast<TU*>(smem_raw);                                // [2][NP][COLS]
  C* sm = reinterpret_cast<C*>(smem_raw + ((2 * TILE * sizeof(TU) + 15) / 16) * 16);  // [n][COLS]
  const int c = threadIdx.x % COLS;
  const int r = threadIdx.x / COLS;
  if (jdev) w += (size_t)(*jdev) * wstride;
  auto issue = [&](int tile, int buf) {
    TU* dst = stage + buf * TILE;
    const int64_t s0 = (int64_t)tile * COLS;
    for (int e = threadIdx.x; e < TILE; e += 256) {
      const int cc = e % COLS;
      const int p = e / COLS;
      const bool ok = s0 + cc < ms;
      cp_async<sizeof(TU)>(dst + e, spec + (int64_t)p * ms + (ok ? s0 + cc : 0), ok);
    }
    cp_async_commit();
  };
  if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  int buf = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    if (t + (int)gridDim.x < ntiles)
      issue(t + gridDim.x, buf ^ 1);
    else
      cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const TU* st = stage + buf * TILE;
    const int64_t s = (int64_t)t * COLS + c;
    const bool valid = s < ms;
    Parents<Tc, TU> par;
    if (fc.ec && valid) par.init(fc, s);
    inv4_body<Tc, Tout, N1, N2>(
        [&](int k, C& sa, C& sb) {
          sa = ldc(st, (2 * k) * COLS + c);
          sb = ldc(st, (2 * k + 1) * COLS + c);
          if (fc.ec && valid) {
            sa = sa + par.at(fc, 2 * k);
            sb = sb + par.at(fc, 2 * k + 1);
          }
        },
        dpow, dinv, tw, w, sm, ms, s, valid, r, c);
    __syncthreads();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Direct DFT along time for lengths that are not powers of two (the paper's own
// runs use n = 2^k - 1): a CTA holds TS columns of all n time samples in shared
// memory and forms each needed frequency as a plain sum with the twiddle index
// advanced incrementally modulo n.  n^2 work per column.
template <typename Tc, typename Tin>
__global__ void __launch_bounds__(256) tdft_forward_kernel(const Tin* __restrict__ v, const Tc* __restrict__ dpow,
                                                           const Tc* __restrict__ dinv,
                                                           const typename Cx<Tc>::t* __restrict__ tw,
                                                           typename Cx<Tc>::t* __restrict__ spec, int64_t ms, int n,
                                                           int TS) {
  typedef typename Cx<Tc>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* z = reinterpret_cast<C*>(smem_raw);  // [n][TS]
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const Tin* v1 = v;
  const Tin* v2 = v + (int64_t)n * ms;
  for (int e = threadIdx.x; e < n * TS; e += blockDim.x) {
    const int j = e / TS, c = e - (e / TS) * TS;
    const int64_t s = s0 + c;
    Tc a = Tc(0), b = Tc(0);
    if (s < ms) {
      a = cvt<Tc>(v1[(int64_t)(n - 1 - j) * ms + s]) * dpow[j];  // D J v1
      b = cvt<Tc>(v2[(int64_t)j * ms + s]) * dpow[j];            // D v2
    }
    z[j * TS + c] = cmk<Tc>(a, b);
  }
  __syncthreads();
  const int nf = n / 2 + 1;
  const Tc hf = Tc(0.5);
  for (int e = threadIdx.x; e < nf * TS; e += blockDim.x) {
    const int k = e / TS, c = e - (e / TS) * TS;
    const int64_t s = s0 + c;
    const int kn = (n - k) % n;
    C Z = czero<Tc>(), W = czero<Tc>();
    int ik = 0, ikn = 0;  // (j k) mod n and (j (n-k)) mod n
    for (int j = 0; j < n; ++j) {
      const C x = z[j * TS + c];
      const C a = tw[ik], b = tw[ikn];
      Z.x = fma(a.x, x.x, fma(-a.y, x.y, Z.x));
      Z.y = fma(a.x, x.y, fma(a.y, x.x, Z.y));
      W.x = fma(b.x, x.x, fma(-b.y, x.y, W.x));
      W.y = fma(b.x, x.y, fma(b.y, x.x, W.y));
      ik += k;
      if (ik >= n) ik -= n;
      ikn += kn;
      if (ikn >= n) ikn -= n;
    }
    if (s >= ms) continue;
    spec[(int64_t)(2 * k) * ms + s] = cmk<Tc>((Z.y + W.y) * hf, (W.x - Z.x) * hf);  // hat v2[k]
    spec[(int64_t)(2 * k + 1) * ms + s] = cmk<Tc>((Z.x + W.x) * hf, (Z.y - W.y) * hf);  // hat v1[k]
  }
}

template <typename Tc, typename TU, typename Tout>
__global__ void __launch_bounds__(256) tdft_inverse_kernel(const TU* __restrict__ spec, const Tc* __restrict__ dpow,
                                                           const Tc* __restrict__ dinv,
                                                           const typename Cx<Tc>::t* __restrict__ tw,
                                                           Tout* __restrict__ w, int64_t ms, int n, int TS,
                                                           FineCorrection<TU> fc) {
  typedef typename Cx<Tc>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* z = reinterpret_cast<C*>(smem_raw);  // [n][TS]
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const int nf = n / 2 + 1;
  for (int e = threadIdx.x; e < nf * TS; e += blockDim.x) {
    const int k = e / TS, c = e - (e / TS) * TS;
    const int64_t s = s0 + c;
    C sa = czero<Tc>(), sb = czero<Tc>();
    if (s < ms) {
      sa = ldc(spec, (int64_t)(2 * k) * ms + s);
      sb = ldc(spec, (int64_t)(2 * k + 1) * ms + s);
      if (fc.ec) {
        Parents<Tc, TU> par;
        par.init(fc, s);
        sa = sa + par.at(fc, 2 * k);
        sb = sb + par.at(fc, 2 * k + 1);
      }
    }
    // Y[k] = hat w1[k] + i hat w2[k], Y[n-k] = conj(hat w1[k]) + i conj(hat w2[k])
    z[k * TS + c] = cmk<Tc>(sb.x - sa.y, sb.y + sa.x);
    if (k > 0 && 2 * k < n) z[(n - k) * TS + c] = cmk<Tc>(sb.x + sa.y, sa.x - sb.y);
  }
  __syncthreads();
  const Tc inv_n = Tc(1) / Tc(n);
  C* o = z + (size_t)n * TS;  // [n][TS]: half 1 in .x, half 2 in .y, both at their own time
  for (int e = threadIdx.x; e < n * TS; e += blockDim.x) {
    const int j = e / TS, c = e - (e / TS) * TS;
    C y = czero<Tc>();
    int ij = 0;  // (j k) mod n, conjugate twiddles
    for (int k = 0; k < n; ++k) {
      const C x = z[k * TS + c];
      const C a = tw[ij];
      y.x = fma(a.x, x.x, fma(a.y, x.y, y.x));
      y.y = fma(a.x, x.y, fma(-a.y, x.x, y.y));
      ij += j;
      if (ij >= n) ij -= n;
    }
    o[(n - 1 - j) * TS + c].x = dinv[j] * (y.x * inv_n);  // J D^{-1} ifft(hat w1)
    o[j * TS + c].y = dinv[j] * (y.y * inv_n);            // D^{-1} ifft(hat w2)
  }
  __syncthreads();
  Tout* w1 = w;
  Tout* w2 = w + (int64_t)n * ms;
  for (int e = threadIdx.x; e < n * TS; e += blockDim.x) {
    const int j = e / TS, c = e - (e / TS) * TS;
    const int64_t s = s0 + c;
    if (s >= ms) continue;
    const C t = o[j * TS + c];
    w1[(int64_t)j * ms + s] = cvt<Tout>(t.x - t.y);  // step 4: [[I, -I], [I, I]]
    w2[(int64_t)j * ms + s] = cvt<Tout>(t.x + t.y);
  }
}

template <typename Tc>
int pick_ts_dft(int n) {
  // n*TS complex values within 96 KB of shared memory, TS a power of two in [1, 64]
  const int budget = 98304 / (int)sizeof(typename Cx<Tc>::t);
  int ts = 64;
  while (ts > 1 && n * ts > budget) ts >>= 1;
  return ts;
}

template <typename Tc>
int pick_ts(int n) {
  // keep n*TS complex values within 64 KB of shared memory, TS a power of two in [1, 256]
  const int budget = 65536 / (int)sizeof(typename Cx<Tc>::t);
  int ts = 256;
  while (ts > 1 && n * ts > budget) ts >>= 1;
  return ts;
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace

template <typename Tin, typename Tc, int N1, int N2>
cudaError_t fwd4(Launch& L, int64_t ms, const Tin* v, const Tc* dpow, const Tc* dinv, const typename Cx<Tc>::t* tw,
                 typename Cx<Tc>::t* spec, size_t vstride, const int* jdev) {
  constexpr int COLS = 256 / N1;
  const size_t smem = (size_t)N1 * N2 * COLS * sizeof(typename Cx<Tc>::t);
  const unsigned blocks = (unsigned)((ms + COLS - 1) / COLS);
  if constexpr (tfft_fp64_blocks<Tc, N1 * N2>() == 2) {
    auto kern = tfft4_forward_f64_kernel<Tin, N1, N2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, 256, smem, L.stream>>>(v, dpow, dinv, tw, spec, ms, vstride, jdev);
  } else {
    auto kern = tfft4_forward_kernel<Tin, Tc, N1, N2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, 256, smem, L.stream>>>(v, dpow, dinv, tw, spec, ms, vstride, jdev);
  }
  return cudaGetLastError();
}

template <typename Tc, typename TU, typename Tout, int N1, int N2>
cudaError_t inv4(Launch& L, int64_t ms, const TU* spec, const Tc* dpow, const Tc* dinv, const typename Cx<Tc>::t* tw,
                 Tout* w, size_t wstride, const int* jdev, const FineCorrection<TU>& fc) {
  constexpr int COLS = 256 / N1;
  const size_t smem = (size_t)N1 * N2 * COLS * sizeof(typename Cx<Tc>::t);
  cudaError_t e = cudaFuncSetAttribute(tfft4_inverse_kernel<Tc, TU, Tout, N1, N2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tfft4_inverse_kernel<Tc, TU, Tout, N1, N2><<<(unsigned)((ms + COLS - 1) / COLS), 256, smem, L.stream>>>(
      spec, dpow, dinv, tw, w, ms, wstride, jdev, fc);
  return cudaGetLastError();
}

static int sm_count(const Launch& L) { return L.tiles && L.tiles->sms > 0 ? L.tiles->sms : 152; }

template <typename Tin, typename Tc, int N1, int N2>
cudaError_t fwd4s(Launch& L, int64_t ms, const Tin* v, const Tc* dpow, const Tc* dinv,
                  const typename Cx<Tc>::t* tw, typename Cx<Tc>::t* spec, size_t vstride, const int* jdev) {
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  const size_t smem = (size_t)2 * 2 * n * COLS * sizeof(Tin) + (size_t)n * COLS * sizeof(typename Cx<Tc>::t);
  if (smem > 227 * 1024) return fwd4<Tin, Tc, N1, N2>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
  auto kern = tfft4s_forward_kernel<Tin, Tc, N1, N2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem)) != cudaSuccess) return e;
  const int ntiles = (int)((ms + COLS - 1) / COLS);
  const int grid = std::min(ntiles, std::max(1, per_sm) * sm_count(L));
  kern<<<grid, 256, smem, L.stream>>>(v, dpow, dinv, tw, spec, ms, ntiles, vstride, jdev);
  return cudaGetLastError();
}

template <typename Tc, typename TU, typename Tout, int N1, int N2>
cudaError_t inv4s(Launch& L, int64_t ms, const TU* spec, const Tc* dpow, const Tc* dinv,
                  const typename Cx<Tc>::t* tw, Tout* w, size_t wstride, const int* jdev,
                  const FineCorrection<TU>& fc) {
  constexpr int n = N1 * N2;
  constexpr int COLS = 256 / N1;
  constexpr int NP = 2 * (n / 2 + 1);
  const size_t smem = (((size_t)2 * NP * COLS * sizeof(TU) + 15) / 16) * 16 +
                      (size_t)n * COLS * sizeof(typename Cx<Tc>::t);
  if (smem > 227 * 1024) return inv4<Tc, TU, Tout, N1, N2>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
  auto kern = tfft4s_inverse_kernel<Tc, TU, Tout, N1, N2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem)) != cudaSuccess) return e;
  const int ntiles = (int)((ms + COLS - 1) / COLS);
  const int grid = std::min(ntiles, std::max(1, per_sm) * sm_count(L));
  kern<<<grid, 256, smem, L.stream>>>(spec, dpow, dinv, tw, w, ms, ntiles, wstride, jdev, fc);
  return cudaGetLastError();
}

// largest n handled by the four-step kernels (register pressure bounds FP64)
template <typename Tc>
constexpr int four_step_max() {
  return sizeof(Tc) == 4 ? 1024 : 256;
}

template <typename Tin, typename Tc>
cudaError_t fwd4_dispatch(Launch& L, int64_t ms, int n, const Tin* v, const Tc* dpow, const Tc* dinv,
                          const typename Cx<Tc>::t* tw, typename Cx<Tc>::t* spec, size_t vstride, const int* jdev) {
  const bool stream = L.tiles && L.tiles->fft_stream > 0;
  switch (n) {
    case 1: return stream ? fwd4s<Tin, Tc, 1, 1>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 1, 1>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 2: return stream ? fwd4s<Tin, Tc, 2, 1>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 2, 1>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 4: return stream ? fwd4s<Tin, Tc, 2, 2>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 2, 2>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 8: return stream ? fwd4s<Tin, Tc, 4, 2>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 4, 2>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 16: return stream ? fwd4s<Tin, Tc, 4, 4>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 4, 4>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 32: return stream ? fwd4s<Tin, Tc, 8, 4>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 8, 4>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 64: return stream ? fwd4s<Tin, Tc, 8, 8>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 8, 8>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 128: return stream ? fwd4s<Tin, Tc, 16, 8>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 16, 8>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 256: return stream ? fwd4s<Tin, Tc, 16, 16>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 16, 16>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
    case 512:
      if constexpr (sizeof(Tc) == 4) return stream ? fwd4s<Tin, Tc, 32, 16>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 32, 16>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
      break;
    case 1024:
      if constexpr (sizeof(Tc) == 4) return stream ? fwd4s<Tin, Tc, 32, 32>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev)
                    : fwd4<Tin, Tc, 32, 32>(L, ms, v, dpow, dinv, tw, spec, vstride, jdev);
      break;
  }
  return cudaErrorInvalidValue;
}

template <typename Tc, typename TU, typename Tout>
cudaError_t inv4_dispatch(Launch& L, int64_t ms, int n, const TU* spec, const Tc* dpow, const Tc* dinv,
                          const typename Cx<Tc>::t* tw, Tout* w, size_t wstride, const int* jdev,
                          const FineCorrection<TU>& fc) {
  const bool stream = L.tiles && L.tiles->fft_stream > 0;
  switch (n) {
    case 1: return stream ? inv4s<Tc, TU, Tout, 1, 1>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 1, 1>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 2: return stream ? inv4s<Tc, TU, Tout, 2, 1>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 2, 1>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 4: return stream ? inv4s<Tc, TU, Tout, 2, 2>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 2, 2>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 8: return stream ? inv4s<Tc, TU, Tout, 4, 2>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 4, 2>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 16: return stream ? inv4s<Tc, TU, Tout, 4, 4>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 4, 4>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 32: return stream ? inv4s<Tc, TU, Tout, 8, 4>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 8, 4>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 64: return stream ? inv4s<Tc, TU, Tout, 8, 8>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 8, 8>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 128: return stream ? inv4s<Tc, TU, Tout, 16, 8>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 16, 8>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 256: return stream ? inv4s<Tc, TU, Tout, 16, 16>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 16, 16>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    case 512:
      if constexpr (sizeof(Tc) == 4) return stream ? inv4s<Tc, TU, Tout, 32, 16>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 32, 16>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
      break;
    case 1024:
      if constexpr (sizeof(Tc) == 4) return stream ? inv4s<Tc, TU, Tout, 32, 32>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc)
                    : inv4<Tc, TU, Tout, 32, 32>(L, ms, spec, dpow, dinv, tw, w, wstride, jdev, fc);
      break;
  }
  return cudaErrorInvalidValue;
}

template <typename Tc, typename Tin>
cudaError_t launch_tfft_forward(Launch& L, int64_t ms, int n, const Tin* v, const Tc* dpow, const Tc* dinv,
                                const typename Cx<Tc>::t* tw, typename Cx<Tc>::t* spec, size_t vstride,
                                const int* jdev) {
  const bool pow2 = (n & (n - 1)) == 0;
  if (jdev && (n > four_step_max<Tc>() || !pow2)) return cudaErrorNotSupported;
  if (!pow2) {
    const int TS = pick_ts_dft<Tc>(n);
    const size_t smem = (size_t)n * TS * sizeof(typename Cx<Tc>::t);
    cudaError_t e = cudaFuncSetAttribute(tdft_forward_kernel<Tc, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nf = n / 2 + 1;
    L.begin(KC_TFFT_FWD);
    tdft_forward_kernel<Tc, Tin><<<(unsigned)((ms + TS - 1) / TS), 256, smem, L.stream>>>(v, dpow, dinv, tw, spec, ms, n, TS);
    return L.end(KC_TFFT_FWD, 2.0 * n * ms * sizeof(Tin) + 2.0 * nf * ms * sizeof(typename Cx<Tc>::t),
                 16.0 * (double)nf * n * ms);
  }
  if (n <= four_step_max<Tc>()) {
    const int nf = n / 2 + 1;
    const double bytes = 2.0 * n * ms * sizeof(Tin) + 2.0 * nf * ms * sizeof(typename Cx<Tc>::t);
    const double flops = (double)ms * (5.0 * n * ilog2(n) + 2.0 * n);
    L.begin(KC_TFFT_FWD);
    fwd4_dispatch<Tin, Tc>(L, ms, n, v, dpow, dinv, tw, spec, vstride, jdev);
    return L.end(KC_TFFT_FWD, bytes, flops);
  }
  const int TS = pick_ts<Tc>(n);
  const size_t smem = (size_t)n * TS * sizeof(typename Cx<Tc>::t);
  cudaError_t e = cudaFuncSetAttribute(tfft_forward_kernel<Tc, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ms + TS - 1) / TS);
  const int nf = n / 2 + 1;
  const double bytes = 2.0 * n * ms * sizeof(Tin) + 2.0 * nf * ms * sizeof(typename Cx<Tc>::t);
  const double flops = (double)ms * (5.0 * n * ilog2(n) + 2.0 * n);
  L.begin(KC_TFFT_FWD);
  tfft_forward_kernel<Tc, Tin><<<blocks, 256, smem, L.stream>>>(v, dpow, tw, spec, ms, n, ilog2(n), TS);
  return L.end(KC_TFFT_FWD, bytes, flops);
}

template <typename Tc, typename TU, typename Tout>
cudaError_t launch_tfft_inverse(Launch& L, int64_t ms, int n, const TU* spec, const Tc* dpow, const Tc* dinv,
                                const typename Cx<Tc>::t* tw, Tout* w, size_t wstride, const int* jdev,
                                FineCorrection<TU> fc) {
  // bytes of the fused correction: the coarse planes once
  const double cbytes = fc.ec ? (double)(n / 2 + 1) * 2.0 * fc.npc * sizeof(TU) : 0.0;
  const bool pow2 = (n & (n - 1)) == 0;
  if (jdev && (n > four_step_max<Tc>() || !pow2)) return cudaErrorNotSupported;
  if (!pow2) {
    const int TS = pick_ts_dft<Tc>(n);
    // the spectrum and, after the sums, both halves at their own times: two [n][TS] arrays
    const size_t smem = 2 * (size_t)n * TS * sizeof(typename Cx<Tc>::t);
    cudaError_t e =
        cudaFuncSetAttribute(tdft_inverse_kernel<Tc, TU, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nf = n / 2 + 1;
    L.begin(KC_TFFT_INV);
    tdft_inverse_kernel<Tc, TU, Tout><<<(unsigned)((ms + TS - 1) / TS), 256, smem, L.stream>>>(spec, dpow, dinv, tw, w,
                                                                                            ms, n, TS, fc);
    return L.end(KC_TFFT_INV, 2.0 * nf * ms * sizeof(TU) + 2.0 * n * ms * sizeof(Tout) + cbytes,
                 8.0 * (double)n * n * ms);
  }
  if (n <= four_step_max<Tc>()) {
    const int nf = n / 2 + 1;
    const double bytes = 2.0 * nf * ms * sizeof(TU) + 2.0 * n * ms * sizeof(Tout) + cbytes;
    const double flops = (double)ms * (5.0 * n * ilog2(n) + 4.0 * n);
    L.begin(KC_TFFT_INV);
    inv4_dispatch<Tc, TU, Tout>(L, ms, n, spec, dpow, dinv, tw, w, wstride, jdev, fc);
    return L.end(KC_TFFT_INV, bytes, flops);
  }
  const int TS = pick_ts<Tc>(n);
  const size_t smem = (size_t)n * TS * sizeof(typename Cx<Tc>::t);
  cudaError_t e =
      cudaFuncSetAttribute(tfft_inverse_kernel<Tc, TU, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ms + TS - 1) / TS);
  const int nf = n / 2 + 1;
  const double bytes = 2.0 * nf * ms * sizeof(TU) + 2.0 * n * ms * sizeof(Tout) + cbytes;
  const double flops = (double)ms * (5.0 * n * ilog2(n) + 4.0 * n);
  L.begin(KC_TFFT_INV);
  tfft_inverse_kernel<Tc, TU, Tout><<<blocks, 256, smem, L.stream>>>(spec, dpow, tw, w, ms, n, ilog2(n), TS, fc);
  return L.end(KC_TFFT_INV, bytes, flops);
}

template cudaError_t launch_tfft_forward<double, double>(Launch&, int64_t, int, const double*, const double*,
                                                         const double*, const double2*, double2*, size_t, const int*);
template cudaError_t launch_tfft_forward<float, double>(Launch&, int64_t, int, const double*, const float*,
                                                        const float*, const float2*, float2*, size_t, const int*);
template cudaError_t launch_tfft_forward<float, float>(Launch&, int64_t, int, const float*, const float*,
                                                       const float*, const float2*, float2*, size_t, const int*);
#define PCOPT_INV(Tc, TU, Tout)                                                                                  \
  template cudaError_t launch_tfft_inverse<Tc, TU, Tout>(Launch&, int64_t, int, const TU*, const Tc*, const Tc*, \
                                                         const Cx<Tc>::t*, Tout*, size_t, const int*,         \
                                                         FineCorrection<TU>);
PCOPT_INV(double, double2, double)
PCOPT_INV(float, float2, double)
PCOPT_INV(float, float2, float)
PCOPT_INV(float, __nv_bfloat162, double)
PCOPT_INV(float, __nv_bfloat162, float)
#undef PCOPT_INV

PCOPT_DEBUG_READER(pcopt_debug_tfft)

}  // namespace pcopt
