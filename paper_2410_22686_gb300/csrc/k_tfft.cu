// Scaled FFT along time: steps 1 and 3-4 of the four-step apply of
// P_eps^{-1} (Section 2.1), with C_{eps,n} = D^{-1} F Lambda F^* D
// (Eq. decomposition_eps), D = diag(eps^{j/n}), lambda_k = 1 - eps^{1/n} theta^{-k}.
//
// Because C_{eps,n} is real, C^T = D F conj(Lambda) F^* D^{-1}, so
//   half 1 (block C_eps^T + alpha I):  hat v1 = fft(D^{-1} v1), shifts conj(lambda_k) + alpha,
//   half 2 (block C_eps   + alpha I):  hat v2 = fft(D v2),      shifts lambda_k + alpha,
// and both are inverted by D^{+-1} ifft(.).  The two real halves are packed
// into one complex sequence z = D^{-1} v1 + i D v2 (two-for-one), and only the
// Hermitian half k = 0..n/2 is kept.  Since conj(lambda_{n-k}) = lambda_k,
// frequency n-k of half 1 has the same shifted operator as frequency k of
// half 2, so spectral plane 2k holds hat v2[k] and plane 2k+1 holds
// conj(hat v1[k]) = hat v1[n-k]: both planes of a pair share sigma_k = lambda_k + alpha.
//
// One CTA owns TS consecutive spatial points and the whole time axis: it
// reads n rows of TS values per half (coalesced along space), runs an
// in-place radix-2 FFT of length n in shared memory for all TS columns
// (threads of a warp work on consecutive columns: conflict-free), and writes
// frequency-major planes (the time<->space transpose happens in shared memory).
#include "common.cuh"

namespace pcopt {

namespace {

__device__ __forceinline__ int bitrev(int j, int logn) { return logn ? (int)(__brev((unsigned)j) >> (32 - logn)) : 0; }

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

template <typename Tc>
__global__ void __launch_bounds__(256) tfft_forward_kernel(const double* __restrict__ v, const Tc* __restrict__ dpow,
                                                           const typename Cx<Tc>::t* __restrict__ tw,
                                                           typename Cx<Tc>::t* __restrict__ spec, int64_t ms, int n,
                                                           int logn, int TS) {
  typedef typename Cx<Tc>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* z = reinterpret_cast<C*>(smem_raw);
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const double* v1 = v;
  const double* v2 = v + (int64_t)n * ms;
  for (int e = threadIdx.x; e < n * TS; e += blockDim.x) {
    const int j = e / TS;
    const int c = e - j * TS;
    const int64_t s = s0 + c;
    Tc a = Tc(0), b = Tc(0);
    if (s < ms) {
      const Tc d = dpow[j];
      a = (Tc)v1[(int64_t)j * ms + s] / d;   // D^{-1} v1
      b = (Tc)v2[(int64_t)j * ms + s] * d;   // D v2
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
    // hat v2[k] = (Z[k] - conj Z[n-k]) / (2i);  conj(hat v1[k]) = (conj Z[k] + Z[n-k]) / 2
    spec[(int64_t)(2 * k) * ms + s] = cmk<Tc>((Z.y + W.y) * hf, (W.x - Z.x) * hf);
    spec[(int64_t)(2 * k + 1) * ms + s] = cmk<Tc>((Z.x + W.x) * hf, (W.y - Z.y) * hf);
  }
}

template <typename Tc, typename TU, typename Tout>
__global__ void __launch_bounds__(256) tfft_inverse_kernel(const TU* __restrict__ spec,
                                                           const Tc* __restrict__ dpow,
                                                           const typename Cx<Tc>::t* __restrict__ tw,
                                                           Tout* __restrict__ w, int64_t ms, int n, int logn,
                                                           int TS) {
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
      sb = ldc(spec, (int64_t)(2 * k + 1) * ms + s);  // hat w1[n-k] = conj(hat w1[k])
    }
    // Y[k] = hat w1[k] + i hat w2[k] with hat w1[k] = conj(sb), hat w2[k] = sa
    z[bitrev(k, logn) * TS + c] = cmk<Tc>(sb.x - sa.y, sa.x - sb.y);
    if (k > 0 && 2 * k < n) {
      // Y[n-k] = hat w1[n-k] + i hat w2[n-k] with hat w1[n-k] = sb, hat w2[n-k] = conj(sa)
      z[bitrev(n - k, logn) * TS + c] = cmk<Tc>(sb.x + sa.y, sb.y + sa.x);
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
    const C y = z[j * TS + c];
    const Tc d = dpow[j];
    const Tc wt1 = d * (y.x * inv_n);   // D ifft(hat w1)
    const Tc wt2 = (y.y * inv_n) / d;   // D^{-1} ifft(hat w2)
    w1[(int64_t)j * ms + s] = (Tout)(wt1 - wt2);   // step 4: [[I, -I], [I, I]]
    w2[(int64_t)j * ms + s] = (Tout)(wt1 + wt2);
  }
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

template <typename Tc>
cudaError_t launch_tfft_forward(Launch& L, int64_t ms, int n, const double* v, const Tc* dpow,
                                const typename Cx<Tc>::t* tw, typename Cx<Tc>::t* spec) {
  const int TS = pick_ts<Tc>(n);
  const size_t smem = (size_t)n * TS * sizeof(typename Cx<Tc>::t);
  cudaError_t e = cudaFuncSetAttribute(tfft_forward_kernel<Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ms + TS - 1) / TS);
  const int nf = n / 2 + 1;
  const double bytes = 2.0 * n * ms * 8.0 + 2.0 * nf * ms * sizeof(typename Cx<Tc>::t);
  const double flops = (double)ms * (5.0 * n * ilog2(n) + 2.0 * n);
  L.begin(KC_TFFT_FWD);
  tfft_forward_kernel<Tc><<<blocks, 256, smem, L.stream>>>(v, dpow, tw, spec, ms, n, ilog2(n), TS);
  return L.end(KC_TFFT_FWD, bytes, flops);
}

template <typename Tc, typename TU, typename Tout>
cudaError_t launch_tfft_inverse(Launch& L, int64_t ms, int n, const TU* spec, const Tc* dpow,
                                const typename Cx<Tc>::t* tw, Tout* w) {
  const int TS = pick_ts<Tc>(n);
  const size_t smem = (size_t)n * TS * sizeof(typename Cx<Tc>::t);
  cudaError_t e =
      cudaFuncSetAttribute(tfft_inverse_kernel<Tc, TU, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ms + TS - 1) / TS);
  const int nf = n / 2 + 1;
  const double bytes = 2.0 * nf * ms * sizeof(TU) + 2.0 * n * ms * sizeof(Tout);
  const double flops = (double)ms * (5.0 * n * ilog2(n) + 4.0 * n);
  L.begin(KC_TFFT_INV);
  tfft_inverse_kernel<Tc, TU, Tout><<<blocks, 256, smem, L.stream>>>(spec, dpow, tw, w, ms, n, ilog2(n), TS);
  return L.end(KC_TFFT_INV, bytes, flops);
}

template cudaError_t launch_tfft_forward<double>(Launch&, int64_t, int, const double*, const double*, const double2*,
                                                 double2*);
template cudaError_t launch_tfft_forward<float>(Launch&, int64_t, int, const double*, const float*, const float2*,
                                                float2*);
template cudaError_t launch_tfft_inverse<double, double2, double>(Launch&, int64_t, int, const double2*,
                                                                  const double*, const double2*, double*);
template cudaError_t launch_tfft_inverse<float, float2, double>(Launch&, int64_t, int, const float2*, const float*,
                                                                const float2*, double*);
template cudaError_t launch_tfft_inverse<float, float2, float>(Launch&, int64_t, int, const float2*, const float*,
                                                               const float2*, float*);
template cudaError_t launch_tfft_inverse<float, __nv_bfloat162, double>(Launch&, int64_t, int,
                                                                        const __nv_bfloat162*, const float*,
                                                                        const float2*, double*);
template cudaError_t launch_tfft_inverse<float, __nv_bfloat162, float>(Launch&, int64_t, int, const __nv_bfloat162*,
                                                                       const float*, const float2*, float*);

}  // namespace pcopt
