// Arnoldi / GMRES building blocks, all FP64 (GMRES of Section 3, Lemma 2.1):
// multi-dot h = V^T w, Gram-Schmidt update w -= V h fused with ||w||^2,
// normalisation, Givens rotations of the Hessenberg column with the residual
// estimate, back substitution and the solution update x += Z y.
//
// Reductions are deterministic: a fixed grid writes per-block partial sums
// (warp shuffles, then shared memory), and a second kernel adds them in a
// fixed order.  The multi-dot keeps up to kChunk accumulators per thread so
// that V is read once and w once per chunk of vectors.
#include "common.cuh"

namespace pcopt {

namespace {

constexpr int kChunk = 16;
constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads) multidot_kernel(const double* __restrict__ V, size_t ldv, int i0, int cnt,
                                                            const double* __restrict__ w, size_t len,
                                                            double* __restrict__ partial, int nv) {
  double acc[kChunk];
#pragma unroll
  for (int c = 0; c < kChunk; ++c) acc[c] = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double* Vb = V + (size_t)i0 * ldv;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const double we = w[e];
#pragma unroll
    for (int c = 0; c < kChunk; ++c)
      if (c < cnt) acc[c] = fma(Vb[(size_t)c * ldv + e], we, acc[c]);
  }
  __shared__ double red[kThreads / 32][kChunk];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kChunk; ++c) {
    if (c < cnt) {
      const double v = warp_sum(acc[c]);
      if (lane == 0) red[wid][c] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q][threadIdx.x];
    partial[(size_t)blockIdx.x * nv + i0 + threadIdx.x] = s;
  }
}

// out[i] = sum_b partial[b*nv + i], one block per i, fixed order
__global__ void __launch_bounds__(kThreads) reduce_partials_kernel(const double* __restrict__ partial, int nblocks,
                                                                   int nv, double* __restrict__ out) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * nv + i];
  __shared__ double red[kThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    out[i] = t;
  }
}

__global__ void __launch_bounds__(kThreads) update_norm_kernel(const double* __restrict__ V, size_t ldv, int nv,
                                                               const double* __restrict__ h, double* __restrict__ w,
                                                               size_t len, double* __restrict__ partial) {
  extern __shared__ double hs[];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    double we = w[e];
    for (int i = 0; i < nv; ++i) we = fma(-hs[i], V[(size_t)i * ldv + e], we);
    w[e] = we;
    acc = fma(we, we, acc);
  }
  __shared__ double red[kThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) norm2_kernel(const double* __restrict__ w, size_t len,
                                                         double* __restrict__ partial) {
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) acc = fma(w[e], w[e], acc);
  __shared__ double red[kThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void scale_kernel(const double* __restrict__ w, double* __restrict__ v, size_t len,
                             const double* __restrict__ nrm2) {
  const double q = 1.0 / sqrt(nrm2[0]);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) v[e] = w[e] * q;
}

template <typename Tx>
__global__ void axpby_kernel(double a, const Tx* __restrict__ x, double b, double* __restrict__ y, size_t len) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride)
    y[e] = (b == 0.0) ? a * (double)x[e] : fma(a, (double)x[e], b * y[e]);
}

// Column j of the Hessenberg matrix: H[0..j][j] = h1 (+ h2), H[j+1][j] = sqrt(nrm2);
// apply rotations 0..j-1, build rotation j, update g, est = |g[j+1]| / ref.
__global__ void givens_kernel(int j, int ldh, double* H, double* cs, double* sn, double* g, const double* h1,
                              const double* h2, const double* nrm2, double* est, const double* ref) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + (h2 ? h2[i] : 0.0);
  col[j + 1] = sqrt(nrm2[0]);
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  double c = 1.0, s = 0.0, r = a;
  if (b != 0.0) {
    r = hypot(a, b);
    c = a / r;
    s = b / r;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = r;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  est[0] = fabs(g[j + 1]) / ref[0];
}

__global__ void backsolve_kernel(int k, int ldh, const double* H, const double* g, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(size_t)q * ldh + i] * y[q];
    y[i] = s / H[(size_t)i * ldh + i];
  }
}

template <typename Tz>
__global__ void __launch_bounds__(kThreads) xupdate_kernel(const Tz* __restrict__ Z, size_t ldz, int k,
                                                           const double* __restrict__ y, double* __restrict__ x,
                                                           size_t len) {
  extern __shared__ double ys[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    double xe = x[e];
    for (int i = 0; i < k; ++i) xe = fma(ys[i], (double)Z[(size_t)i * ldz + e], xe);
    x[e] = xe;
  }
}

__global__ void arnoldi_start_kernel(double* g, const double* nrm2, double* est, double* ref, int set_ref) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = sqrt(nrm2[0]);
  g[0] = beta;
  if (set_ref) ref[0] = beta;
  est[0] = beta / ref[0];
}

unsigned stream_blocks(size_t len) {
  size_t b = (len + kThreads - 1) / kThreads;
  const size_t cap = (size_t)num_sms() * 8;
  return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

}  // namespace

cudaError_t launch_multidot(Launch& L, const double* V, size_t ldv, int nv, const double* w, size_t len,
                            double* partial, int nblocks, double* out) {
  for (int i0 = 0; i0 < nv; i0 += kChunk) {
    const int cnt = nv - i0 < kChunk ? nv - i0 : kChunk;
    L.begin(KC_DOT);
    multidot_kernel<<<nblocks, kThreads, 0, L.stream>>>(V, ldv, i0, cnt, w, len, partial, nv);
    cudaError_t e = L.end(KC_DOT, 8.0 * len * (cnt + 1), 2.0 * len * cnt);
    if (e != cudaSuccess) return e;
  }
  L.begin(KC_REDUCE);
  reduce_partials_kernel<<<nv, kThreads, 0, L.stream>>>(partial, nblocks, nv, out);
  return L.end(KC_REDUCE, 8.0 * nblocks * nv, 1.0 * nblocks * nv);
}

cudaError_t launch_update_norm(Launch& L, const double* V, size_t ldv, int nv, const double* h, double* w, size_t len,
                               double* partial, int nblocks, double* nrm2) {
  L.begin(KC_UPDATE);
  update_norm_kernel<<<nblocks, kThreads, sizeof(double) * (nv > 0 ? nv : 1), L.stream>>>(V, ldv, nv, h, w, len,
                                                                                         partial);
  cudaError_t e = L.end(KC_UPDATE, 8.0 * len * (nv + 2), 2.0 * len * (nv + 1));
  if (e != cudaSuccess) return e;
  L.begin(KC_REDUCE);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, nblocks, 1, nrm2);
  return L.end(KC_REDUCE, 8.0 * nblocks, 1.0 * nblocks);
}

cudaError_t launch_norm2(Launch& L, const double* w, size_t len, double* partial, int nblocks, double* nrm2) {
  L.begin(KC_DOT);
  norm2_kernel<<<nblocks, kThreads, 0, L.stream>>>(w, len, partial);
  cudaError_t e = L.end(KC_DOT, 8.0 * len, 2.0 * len);
  if (e != cudaSuccess) return e;
  L.begin(KC_REDUCE);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, nblocks, 1, nrm2);
  return L.end(KC_REDUCE, 8.0 * nblocks, 1.0 * nblocks);
}

cudaError_t launch_scale_by_inv_norm(Launch& L, const double* w, double* v, size_t len, const double* nrm2) {
  L.begin(KC_SCALE);
  scale_kernel<<<stream_blocks(len), kThreads, 0, L.stream>>>(w, v, len, nrm2);
  return L.end(KC_SCALE, 16.0 * len, 1.0 * len);
}

template <typename Tx>
cudaError_t launch_axpby(Launch& L, double a, const Tx* x, double b, double* y, size_t len) {
  L.begin(KC_AXPBY);
  axpby_kernel<Tx><<<stream_blocks(len), kThreads, 0, L.stream>>>(a, x, b, y, len);
  return L.end(KC_AXPBY, (double)len * (sizeof(Tx) + (b == 0.0 ? 8.0 : 16.0)), 3.0 * len);
}
template cudaError_t launch_axpby<double>(Launch&, double, const double*, double, double*, size_t);
template cudaError_t launch_axpby<float>(Launch&, double, const float*, double, double*, size_t);

cudaError_t launch_givens(Launch& L, int j, int ldh, double* H, double* cs, double* sn, double* gvec,
                          const double* hcol, const double* nrm2, double* est, const double* ref) {
  // hcol holds two consecutive arrays of ldh entries: first and second Gram-Schmidt pass
  L.begin(KC_GIVENS);
  givens_kernel<<<1, 32, 0, L.stream>>>(j, ldh, H, cs, sn, gvec, hcol, hcol + ldh, nrm2, est, ref);
  return L.end(KC_GIVENS, 0.0, 10.0 * (j + 1));
}

cudaError_t launch_backsolve(Launch& L, int k, int ldh, const double* H, const double* gvec, double* y) {
  L.begin(KC_GIVENS);
  backsolve_kernel<<<1, 32, 0, L.stream>>>(k, ldh, H, gvec, y);
  return L.end(KC_GIVENS, 0.0, 1.0 * k * k);
}

template <typename Tz>
cudaError_t launch_xupdate(Launch& L, const Tz* Z, size_t ldz, int k, const double* y, double* x, size_t len) {
  L.begin(KC_XUPDATE);
  xupdate_kernel<Tz><<<stream_blocks(len), kThreads, sizeof(double) * (k > 0 ? k : 1), L.stream>>>(Z, ldz, k, y, x,
                                                                                                  len);
  return L.end(KC_XUPDATE, (double)len * (k * sizeof(Tz) + 16.0), 2.0 * len * k);
}
template cudaError_t launch_xupdate<double>(Launch&, const double*, size_t, int, const double*, double*, size_t);
template cudaError_t launch_xupdate<float>(Launch&, const float*, size_t, int, const double*, double*, size_t);

cudaError_t launch_arnoldi_start(Launch& L, double* gvec, const double* nrm2, double* est, double* ref_out,
                                 int set_ref) {
  L.begin(KC_GIVENS);
  arnoldi_start_kernel<<<1, 32, 0, L.stream>>>(gvec, nrm2, est, ref_out, set_ref);
  return L.end(KC_GIVENS, 0.0, 2.0);
}

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

}  // namespace pcopt
