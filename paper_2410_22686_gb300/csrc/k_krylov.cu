// Arnoldi / GMRES building blocks, all FP64 (GMRES of Section 3, Lemma 2.1).
//
// One Arnoldi step for the new vector w (stored in place of v_{j+1}):
//   pass 1  d = V^T w and ||w||^2                       (multidot, one read of V and w)
//   prep    c = sqrt(||w||^2 - ||d||^2)  (Pythagoras)    (one thread)
//   pass 2  v_{j+1} = (w - V d) / c, q = ||w - V d||^2   (update, one read of V and w, one write)
//   check   re-orthogonalise if the projection cancelled most of w or Pythagoras is
//           inaccurate: then pass 1/2 run again on v_{j+1} and it is renormalised
//           (the gated kernels return at once when the check passed)
//   givens  column j of H = d (+ c e), h_{j+1,j} = c (or c rho); rotations; |g_{j+1}|/ref
// This is classical Gram-Schmidt with selective re-orthogonalisation: two passes
// over the basis per iteration in the common case instead of four.
//
// The re-orthogonalisation pass removes what the first pass left along the basis,
// components of ~1e-6 relative size at most (the check triggers there), so its
// coefficients e = V^T v need only a few significant digits: they are formed on the
// FP32 units from 20-bit truncations of V and v (error ~1e-10 absolute for 33 M
// unknowns), and v - V e is accumulated in FP32 and subtracted from the FP64 v.  The
// Arnoldi relation stays exact to FP64 rounding (column j of H takes the same e), the
// new vector is orthogonal to ~1e-10, and the pass runs at memory speed instead of at
// the FP64 unit's rate.
//
// Reductions are deterministic: an occupancy-sized grid writes per-block partial
// sums (warp shuffles, then shared memory) and a second kernel adds them in a
// fixed order.  The multi-dot is instantiated per vector count (1..16) so that
// every FMA it issues is useful; more vectors take several chunked launches.
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace pcopt {

namespace {

constexpr int kChunk = 16;
constexpr int kThreads = 256;
constexpr int kMaxChunks = 64;   // up to 1024 basis vectors

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool gated_off(const double* gate) { return gate && gate[0] == 0.0; }

// The top 20 mantissa bits of a double as a float (sign, exponent rebiased,
// truncated), in integer operations; magnitudes below the float range become 0.
__device__ __forceinline__ float hi20(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned mag = hi & 0x7FFFFFFFu;
  const unsigned f = mag >= (897u << 20) ? (mag - (896u << 20)) << 3 : 0u;
  return __uint_as_float((hi & 0x80000000u) | f);
}

// partial[b*ld + i0 + c] = sum over block b of V_{i0+c} . w   (c < CNT)
// partial[b*ld + nv]     = sum over block b of w . w          (WITH_NORM)
// LP: FP32 products of 20-bit truncations (the re-orthogonalisation pass), no norm.
template <int CNT, bool WITH_NORM, bool LP = false>
__device__ __forceinline__ void multidot_body(const double* __restrict__ V, size_t ldv, int i0,
                                              const double* __restrict__ w, size_t len,
                                              double* __restrict__ partial, int ncol_norm, int ld) {
  double acc[CNT];
  float accf[LP ? CNT : 1];
  double ww = 0.0;
#pragma unroll
  for (int c = 0; c < CNT; ++c) acc[c] = 0.0;
#pragma unroll
  for (int c = 0; c < (LP ? CNT : 1); ++c) accf[c] = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double* Vb = V + (size_t)i0 * ldv;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const double we = w[e];
    if (LP) {
      const float wf = hi20(we);
#pragma unroll
      for (int c = 0; c < CNT; ++c) accf[LP ? c : 0] = fmaf(hi20(__ldg(Vb + (size_t)c * ldv + e)), wf, accf[LP ? c : 0]);
      continue;
    }
    if (WITH_NORM) ww = fma(we, we, ww);
#pragma unroll
    for (int c = 0; c < CNT; ++c) acc[c] = fma(__ldg(Vb + (size_t)c * ldv + e), we, acc[c]);
  }
  if (LP) {
#pragma unroll
    for (int c = 0; c < CNT; ++c) acc[c] = (double)accf[LP ? c : 0];
  }
  __shared__ double red[kThreads / 32][CNT + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    const double v = warp_sum(acc[c]);
    if (lane == 0) red[wid][c] = v;
  }
  if (WITH_NORM) {
    const double v = warp_sum(ww);
    if (lane == 0) red[wid][CNT] = v;
  }
  __syncthreads();
  if (threadIdx.x < CNT + (WITH_NORM ? 1 : 0)) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q][threadIdx.x];
    const int col = threadIdx.x < CNT ? i0 + threadIdx.x : ncol_norm;
    partial[(size_t)blockIdx.x * ld + col] = s;
  }
}

template <int CNT, bool WITH_NORM, bool LP = false>
__global__ void __launch_bounds__(kThreads) multidot_kernel(const double* __restrict__ V, size_t ldv, int i0,
                                                            const double* __restrict__ w, size_t len,
                                                            double* __restrict__ partial, int nv, int ld,
                                                            const double* __restrict__ gate) {
  if (gated_off(gate)) return;
  multidot_body<CNT, WITH_NORM, LP>(V, ldv, i0, w, len, partial, nv, ld);
}

// Device-resident Arnoldi index: nv = *jdev + 1 vectors, w = wbase + (*jdev + 1) wstride;
// the chunk [i0, i0 + 16) exits when it lies beyond nv, otherwise dispatches on its count.
// The norm column is ld - 1.
template <bool WITH_NORM, bool LP = false>
__global__ void __launch_bounds__(kThreads) multidot_dyn_kernel(const double* __restrict__ V, size_t ldv, int i0,
                                                                const double* __restrict__ wbase, size_t wstride,
                                                                const int* __restrict__ jdev, size_t len,
                                                                double* __restrict__ partial, int ld,
                                                                const double* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int nv = *jdev + 1;
  if (i0 >= nv) return;
  const double* w = wbase + (size_t)nv * wstride;
  const int cnt = nv - i0 < kChunk ? nv - i0 : kChunk;
  switch (cnt) {
#define PCOPT_DYN(k) \
  case k: multidot_body<k, WITH_NORM, LP>(V, ldv, i0, w, len, partial, ld - 1, ld); break;
    PCOPT_DYN(1) PCOPT_DYN(2) PCOPT_DYN(3) PCOPT_DYN(4) PCOPT_DYN(5) PCOPT_DYN(6) PCOPT_DYN(7) PCOPT_DYN(8)
    PCOPT_DYN(9) PCOPT_DYN(10) PCOPT_DYN(11) PCOPT_DYN(12) PCOPT_DYN(13) PCOPT_DYN(14) PCOPT_DYN(15) PCOPT_DYN(16)
#undef PCOPT_DYN
    default: break;
  }
}

// number of blocks that wrote the partial sums of each chunk of kChunk columns
struct ChunkGrids {
  unsigned nb[kMaxChunks];
};

// out[i] = sum_b partial[b*ld + i] for i < nout (column nout goes to *extra), in a
// fixed order; one block per column
// With jdev != nullptr: nout = *jdev + 1, the grid covers the largest count, blocks
// beyond nout exit, and the last block reduces the extra column ld - 1.
__global__ void __launch_bounds__(kThreads) reduce_partials_kernel(const double* __restrict__ partial, ChunkGrids cg,
                                                                   int ld, double* __restrict__ out,
                                                                   double* __restrict__ extra, int nout,
                                                                   const double* __restrict__ gate,
                                                                   const int* __restrict__ jdev) {
  if (gated_off(gate)) return;
  int i = blockIdx.x;
  if (jdev) {
    nout = *jdev + 1;
    if (extra && i == (int)gridDim.x - 1) {
      i = ld - 1;
    } else if (i >= nout) {
      return;
    }
  }
  const int nblocks = (int)cg.nb[i < nout ? i / kChunk : 0];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * ld + i];
  __shared__ double red[kThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    if (i < nout)
      out[i] = t;
    else
      extra[0] = t;
  }
}

// v = (v - sum_i coef_i V_i) * scale ;  partial[b] = sum over block b of (v - sum)^2 (before scaling)
// with jdev != nullptr: nv = *jdev + 1 and v = vbase + nv * vstride.  vf != nullptr also
// receives the FP32 rounding of the new v (the FP32 preconditioner's input).
// LP: sum_i coef_i V_i in FP32 from 20-bit truncations of V (the re-orthogonalisation
// pass, whose coefficients are tiny), subtracted from the FP64 v.
template <bool LP>
__global__ void __launch_bounds__(kThreads) update_kernel(const double* __restrict__ V, size_t ldv, int nv,
                                                          const double* __restrict__ coef, double* __restrict__ v,
                                                          size_t len, const double* __restrict__ scale,
                                                          double* __restrict__ partial,
                                                          const double* __restrict__ gate,
                                                          const int* __restrict__ jdev, size_t vstride,
                                                          float* __restrict__ vf) {
  if (gated_off(gate)) return;
  if (jdev) {
    nv = *jdev + 1;
    v += (size_t)nv * vstride;
  }
  extern __shared__ double hs[];
  float* hf = reinterpret_cast<float*>(hs);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    if (LP)
      hf[i] = (float)coef[i];
    else
      hs[i] = coef[i];
  }
  __syncthreads();
  const double sc = scale ? scale[0] : 1.0;
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    double we = v[e];
    if (LP) {
      float sf = 0.0f;
      for (int i = 0; i < nv; ++i) sf = fmaf(hf[i], hi20(__ldg(V + (size_t)i * ldv + e)), sf);
      we -= f32_to_f64(sf);
    } else {
      for (int i = 0; i < nv; ++i) we = fma(-hs[i], __ldg(V + (size_t)i * ldv + e), we);
    }
    acc = fma(we, we, acc);
    const double vn = we * sc;
    v[e] = vn;
    if (vf) vf[e] = f64_to_f32(vn);
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

// v *= 1/sqrt(nrm2[0])  (gated); vf != nullptr also receives the FP32 rounding of v
__global__ void scale_kernel(double* __restrict__ v, size_t len, const double* __restrict__ nrm2,
                             const double* __restrict__ gate, const int* __restrict__ jdev, size_t vstride,
                             float* __restrict__ vf) {
  if (gated_off(gate)) return;
  if (jdev) v += (size_t)(*jdev + 1) * vstride;
  const bool nz = nrm2[0] > 0.0;  // zero vector: nothing to normalise
  const double q = nz ? 1.0 / sqrt(nrm2[0]) : 1.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const double x = nz ? v[e] * q : v[e];
    if (nz) v[e] = x;
    if (vf) vf[e] = f64_to_f32(x);
  }
}

template <typename Tx>
__global__ void axpby_kernel(double a, const Tx* __restrict__ x, double b, double* __restrict__ y, size_t len) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride)
    y[e] = (b == 0.0) ? a * cvt<double>(x[e]) : fma(a, cvt<double>(x[e]), b * y[e]);
}

// c = sqrt(||w||^2 - ||d||^2) when that is safely positive, else 1 (and force re-orthogonalisation)
__global__ void arnoldi_prep_kernel(int nv, const double* d, ArnoldiScalars s, const int* jdev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (jdev) nv = *jdev + 1;
  double dd = 0.0;
  for (int i = 0; i < nv; ++i) dd = fma(d[i], d[i], dd);
  const double ww = s.ww[0];
  const double r = ww - dd;
  if (r > 1e-12 * ww && r > 0.0) {
    s.c[0] = sqrt(r);
    s.inv[0] = 1.0 / s.c[0];
    s.flag[0] = 0.0;
  } else {
    s.c[0] = 1.0;
    s.inv[0] = 1.0;
    s.flag[0] = 1.0;
  }
}

// re-orthogonalise when ||w - V d||^2 < 1e-10 ||w||^2 (one pass then leaves a loss
// of orthogonality of about eps ||w|| / ||w - V d|| > 1e-11) or when the Pythagorean
// norm disagrees with the computed one by more than 1e-6 (relative, squared).  With
// a strong preconditioner A P^{-1} v_j is close to v_j, so strong cancellation is the
// normal case and a tighter trigger would re-orthogonalise in many iterations.
__global__ void arnoldi_check_kernel(ArnoldiScalars s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (s.flag[0] != 0.0) return;
  const double q = s.q[0], ww = s.ww[0], c2 = s.c[0] * s.c[0];
  const bool bad = !(q >= 1e-10 * ww) || !(fabs(q - c2) <= 1e-6 * q);
  s.flag[0] = bad ? 1.0 : 0.0;
}

// Column j of H and its Givens rotation; est = |g_{j+1}| / ref.
//   no re-orthogonalisation:  w = V d + c v_{j+1}
//   re-orthogonalisation:     w = V (d + c e) + c rho v_{j+1},  rho^2 = s.rho2
__global__ void givens_kernel(int j, int ldh, double* H, double* cs, double* sn, double* g, const double* d,
                              const double* e, ArnoldiScalars s, double* est, const double* ref, const int* jdev) {
  if (blockIdx.x != 0) return;
  if (jdev) j = *jdev;
  // the warp stages the column and the rotations in shared memory; one thread then
  // applies the j sequential rotations without waiting on global memory
  __shared__ double cl[1026], sc[1024], ss[1024];
  double* col = H + (size_t)j * ldh;
  const bool re = s.flag[0] != 0.0;
  const double c = s.c[0];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    cl[i] = re ? fma(c, e[i], d[i]) : d[i];
    if (i < j) {
      sc[i] = cs[i];
      ss[i] = sn[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cl[j + 1] = re ? c * sqrt(s.rho2[0]) : c;
    for (int i = 0; i < j; ++i) {
      const double t = sc[i] * cl[i] + ss[i] * cl[i + 1];
      cl[i + 1] = -ss[i] * cl[i] + sc[i] * cl[i + 1];
      cl[i] = t;
    }
    const double a = cl[j], b = cl[j + 1];
    double cr = 1.0, sr = 0.0, r = a;
    if (b != 0.0) {
      r = hypot(a, b);
      cr = a / r;
      sr = b / r;
    }
    cs[j] = cr;
    sn[j] = sr;
    cl[j] = r;
    cl[j + 1] = 0.0;
    g[j + 1] = -sr * g[j];
    g[j] = cr * g[j];
    est[0] = fabs(g[j + 1]) / ref[0];
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = cl[i];
}

__global__ void backsolve_kernel(int k, int ldh, const double* H, const double* g, double* y, const int* kdev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (kdev) k = *kdev;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(size_t)q * ldh + i] * y[q];
    y[i] = s / H[(size_t)i * ldh + i];
  }
}

template <typename Tz>
__global__ void __launch_bounds__(kThreads) xupdate_kernel(const Tz* __restrict__ Z, size_t ldz, int k,
                                                           const double* __restrict__ y, double* __restrict__ x,
                                                           size_t len, const int* __restrict__ kdev) {
  if (kdev) k = *kdev;
  extern __shared__ double ys[];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if constexpr (std::is_same<Tz, float>::value) {
    // FP32 basis Z: sum_i y_i z_i in double-float on the FP32 units (y_i split into
    // float pairs, each product exact up to its FMA error term, the leading parts added
    // by TwoSum, every error gathered in one float; ~2^-46 of the terms), then one FP64
    // addition into x.  The FP64 unit would otherwise bound this kernel.
    float2* yf = reinterpret_cast<float2*>(ys);
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const float hi = (float)y[i];
      yf[i] = make_float2(hi, (float)(y[i] - (double)hi));
    }
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
      float sh = 0.0f, err = 0.0f;
      for (int i = 0; i < k; ++i) {
        const float2 c = yf[i];
        const float z = Z[(size_t)i * ldz + e];
        const float p = __fmul_rn(c.x, z);
        err = __fadd_rn(err, __fadd_rn(fmaf(c.x, z, -p), __fmul_rn(c.y, z)));
        const float s = __fadd_rn(sh, p);
        const float bb = __fsub_rn(s, sh);
        err = __fadd_rn(err, __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb)));
        sh = s;
      }
      x[e] += f32_to_f64(sh) + f32_to_f64(err);
    }
  } else {
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
      double xe = x[e];
      for (int i = 0; i < k; ++i) xe = fma(ys[i], cvt<double>(Z[(size_t)i * ldz + e]), xe);
      x[e] = xe;
    }
  }
}

__global__ void arnoldi_start_kernel(double* g, const double* nrm2, double* est, double* ref, int set_ref) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = sqrt(nrm2[0]);
  g[0] = beta;
  if (set_ref) ref[0] = beta;
  est[0] = beta / ref[0];
}

// Loop control of a graph-captured FGMRES iteration: k = j + 1 iterations are done;
// continue (condition 1) while the estimate is finite, above rtol and j + 1 < maxit.
__global__ void loop_control_kernel(int* jdev, int* kdev, const double* est, double rtol, int maxit,
                                    cudaGraphConditionalHandle hc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = *jdev;
  const double e = est[0];
  const bool cont = isfinite(e) && e > rtol && j + 1 < maxit;
  *kdev = j + 1;
  if (cont) *jdev = j + 1;
  cudaGraphSetConditional(hc, cont ? 1u : 0u);
}

// Before the loop: j = k = 0, and enter the loop only when the initial estimate is
// finite and above rtol.
__global__ void loop_start_kernel(int* jdev, int* kdev, const double* est, double rtol,
                                  cudaGraphConditionalHandle hc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *jdev = 0;
  *kdev = 0;
  const double e = est[0];
  cudaGraphSetConditional(hc, (isfinite(e) && e > rtol) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Double-float basis (flexible GMRES with the FP32 preconditioner).  Each basis
// vector is held as two FP32 planes, v = hi + lo to about 2^-48 relative, in a
// tiled layout: the planes of element tile t (kTile consecutive unknowns) of
// every vector are stored together, vector by vector,
//   offset(i, e, plane) = ((t nvt + i) 2 + plane) kTile + e mod kTile,  t = e / kTile,
// (nvt = vectors per tile block), so the tile of a group of vectors is one
// contiguous block: one bulk copy fills a stage.  The FP32 rounding of the newest
// vector (its hi plane) is also written contiguously for the FP32 preconditioner.
// The Arnoldi products and sums run on the FP32 units as error-free
// transformations (the product's rounding error by FMA, Knuth's TwoSum for the
// running sums), so the passes over the basis are bound by HBM instead of by
// GB300's FP64 unit.  Scalars (h_ij, norms) and the per-block reductions stay FP64.
//
// The first pass (multi-dot and update) streams the basis through shared memory
// (a producer warp issues the bulk asynchronous copies of several stages ahead on
// mbarriers); the selective second pass reads the hi planes directly.
// ---------------------------------------------------------------------------
constexpr int kTile = 512;             // elements per tile of the layout and per streamed stage (two per thread)
constexpr int kGroup = 16;             // basis vectors per stage of the update
constexpr int kBarBytes = 256;         // mbarriers (16 full, 16 empty) at the start of the dynamic shared memory
constexpr size_t kStreamSmem = 220 * 1024;  // dynamic shared-memory budget of a streaming CTA

__device__ __forceinline__ float neg_f(float x) { return -x; }

__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  hi = f64_to_f32(x);
  lo = f64_to_f32(x - f32_to_f64(hi));
}

// s + e += (ah + al)(bh + bl), the product's low-order term al*bl dropped
__device__ __forceinline__ void df_dot_acc(float ah, float al, float bh, float bl, float& s, float& e) {
  const float p = __fmul_rn(ah, bh);
  float t = fmaf(ah, bh, -p);
  t = fmaf(ah, bl, t);
  t = fmaf(al, bh, t);
  const float s2 = __fadd_rn(s, p);
  const float bb = __fsub_rn(s2, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(p, bb));
  e = __fadd_rn(e, __fadd_rn(err, t));
  s = s2;
}

// (ah, al) -= (ch + cl)(vh + vl)
__device__ __forceinline__ void df_sub_prod(float ch, float cl, float vh, float vl, float& ah, float& al) {
  const float p = __fmul_rn(ch, vh);
  float t = fmaf(ch, vh, -p);
  t = fmaf(ch, vl, t);
  t = fmaf(cl, vh, t);
  const float s = __fsub_rn(ah, p);
  const float bb = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(neg_f(p), bb));
  al = __fadd_rn(al, __fsub_rn(err, t));
  ah = s;
}

// (hi, lo) with |lo| <= ulp(hi)/2 from an unnormalised pair
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// (hi, lo) *= (sh + sl)
__device__ __forceinline__ void df_scale(float& hi, float& lo, float sh, float sl) {
  const float p = __fmul_rn(hi, sh);
  float t = fmaf(hi, sh, -p);
  t = fmaf(hi, sl, t);
  t = fmaf(lo, sh, t);
  hi = p;
  lo = t;
  df_renorm(hi, lo);
}

__device__ __forceinline__ size_t round4(size_t x) { return (x + 3) & ~(size_t)3; }

// offset of element e of plane p (0 hi, 1 lo) of basis vector i in the tiled layout
__host__ __device__ __forceinline__ size_t df_at(int nvt, int i, size_t e, int p) {
  return (((e / kTile) * (size_t)nvt + (size_t)i) * 2 + p) * kTile + e % kTile;
}

// nv basis vectors in ceil(nv / 16) chunks of nearly equal size (no small tail chunk,
// whose stages would be mostly overhead): chunk c covers [i0, i0 + cnt)
__host__ __device__ __forceinline__ void balanced_chunk(int nv, int c, int* i0, int* cnt) {
  const int nch = (nv + kChunk - 1) / kChunk;
  const int base = nv / nch, rem = nv % nch;
  *cnt = base + (c < rem ? 1 : 0);
  *i0 = c * base + (c < rem ? c : rem);
}

// Producer/consumer stream of a CTA's items through S shared-memory stages.
// The CTA has kThreads consumer threads (warps 0..7) and one producer warp (warp
// 8).  Stage q has a "full" mbarrier (one arrival with the copies' byte count,
// completed by the copy engine) and an "empty" one (one arrival per consumer
// warp once it has read the stage).  The producer's lanes issue an item's copies
// together: issue(k, stage, full, lane).  consume(k, stage) runs on every consumer
// thread.  No CTA-wide barrier inside the stream.  Every wait is bounded; one that
// runs out sets *err, ends that thread's loop, and the producer then drains the
// copies it has in flight (bounded) before the CTA leaves.
constexpr int kConsumerWarps = kThreads / 32;
constexpr int kStreamThreads = kThreads + 32;

template <typename Issue, typename Consume>
__device__ __forceinline__ void stream_items(size_t nitems, int S, size_t stage_stride, Issue issue, Consume consume,
                                             double* err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm);
  uint64_t* empty = full + 16;
  unsigned char* buf = dsm + kBarBytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kConsumerWarps);
    }
    mbar_init_fence();
  }
  __syncthreads();
  if (warp == kConsumerWarps) {  // producer
    size_t k = 0;
    bool ok = true;
    for (; k < nitems; ++k) {
      const int q = (int)(k % S);
      if (k >= (size_t)S) {
        // the consumers released this stage's previous item (use k / S - 1)
        bool got = mbar_wait_bounded(&empty[q], (uint32_t)((k / S - 1) & 1), nullptr, 0.0);
        got = __all_sync(0xffffffffu, got);
        if (!got) {
          ok = false;
          break;
        }
      }
      issue(k, buf + q * stage_stride, &full[q], lane);
    }
    if (!ok) {
      if (lane == 0) *err = kErrWaitTimeout;
      // items k - S + 1 .. k - 1 may still be in flight: wait for their copies
      const size_t lo = k >= (size_t)S ? k - S + 1 : 0;
      for (size_t m = lo; m < k; ++m) mbar_wait_bounded(&full[m % S], (uint32_t)((m / S) & 1), nullptr, 0.0);
    }
  } else {  // consumers
    for (size_t k = 0; k < nitems; ++k) {
      const int q = (int)(k % S);
      if (!mbar_wait_bounded(&full[q], (uint32_t)((k / S) & 1), err, kErrWaitTimeout)) break;
      consume(k, buf + q * stage_stride);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[q]);
    }
  }
  __syncthreads();
}

// the producer lanes' share of an item: lane 0 announces the bytes, then copy c
// (of ncopies) is issued by lane c % 32
template <typename CopyAt>
__device__ __forceinline__ void issue_copies(uint64_t* bar, uint32_t bytes, int ncopies, int lane, CopyAt copy_at) {
  if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
  __syncwarp();
  for (int c = lane; c < ncopies; c += 32) copy_at(c);
}

// First pass, multi-dot: partial[b*ld + i0 + c] = sum over CTA b of V_{i0+c} . w
// (w FP64, split on use) and, WITH_NORM, partial[b*ld + ncol_norm] = w . w.
template <int CNT, bool WITH_NORM>
__device__ __forceinline__ void multidot_df_stream(const float* __restrict__ Vf, int nvt, int i0,
                                                   const double* __restrict__ w, size_t len,
                                                   double* __restrict__ partial, int ncol_norm, int ld, int S,
                                                   size_t stage_stride, double* err) {
  float s[CNT], er[CNT];
  double ww = 0.0;
#pragma unroll
  for (int c = 0; c < CNT; ++c) s[c] = er[c] = 0.0f;
  const size_t ntiles = (len + kTile - 1) / kTile;
  const size_t mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto issue = [&](size_t k, unsigned char* st, uint64_t* bar, int lane) {
    const size_t e0 = (blockIdx.x + k * gridDim.x) * (size_t)kTile;
    const size_t n = len - e0 < (size_t)kTile ? len - e0 : (size_t)kTile;  // even: len is even
    const uint32_t vb = (uint32_t)CNT * 2 * kTile * 4, db = (uint32_t)(n * 8);
    // copy 0: the tile of vectors i0 .. i0 + CNT - 1 (contiguous); copy 1: w
    issue_copies(bar, vb + db, 2, lane, [&](int c) {
      if (c == 0)
        bulk_copy_g2s(st, Vf + df_at(nvt, i0, e0, 0), vb, bar);
      else
        bulk_copy_g2s(st + vb, w + e0, db, bar);
    });
  };
  // thread t takes elements 2t and 2t + 1 of a tile (8-byte and 16-byte shared loads;
  // both lie inside or both beyond len, which is even)
  auto consume = [&](size_t k, const unsigned char* st) {
    const size_t e0 = (blockIdx.x + k * gridDim.x) * (size_t)kTile;
    if (e0 + 2 * threadIdx.x >= len) return;
    const float2* sv = reinterpret_cast<const float2*>(st);
    const double2 w2 = reinterpret_cast<const double2*>(st + (size_t)2 * CNT * kTile * 4)[threadIdx.x];
    float wh0, wl0, wh1, wl1;
    split_f64(w2.x, wh0, wl0);
    split_f64(w2.y, wh1, wl1);
    if (WITH_NORM) ww = fma(w2.y, w2.y, fma(w2.x, w2.x, ww));
#pragma unroll
    for (int c = 0; c < CNT; ++c) {
      const float2 h = sv[(2 * c) * (kTile / 2) + threadIdx.x], l = sv[(2 * c + 1) * (kTile / 2) + threadIdx.x];
      df_dot_acc(h.x, l.x, wh0, wl0, s[c], er[c]);
      df_dot_acc(h.y, l.y, wh1, wl1, s[c], er[c]);
    }
  };
  stream_items(mine, S, stage_stride, issue, consume, err);
  __shared__ double red[kStreamThreads / 32][CNT + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    const double v = warp_sum(f32_to_f64(s[c]) + f32_to_f64(er[c]));
    if (lane == 0) red[wid][c] = v;
  }
  if (WITH_NORM) {
    const double v = warp_sum(ww);
    if (lane == 0) red[wid][CNT] = v;
  }
  __syncthreads();
  if (threadIdx.x < CNT + (WITH_NORM ? 1 : 0)) {
    double t = 0.0;
    for (int q = 0; q < kStreamThreads / 32; ++q) t += red[q][threadIdx.x];
    const int col = threadIdx.x < CNT ? i0 + threadIdx.x : ncol_norm;
    partial[(size_t)blockIdx.x * ld + col] = t;
  }
}

template <int CNT, bool WITH_NORM>
__global__ void __launch_bounds__(kStreamThreads, 1) multidot_df_kernel(const float* __restrict__ Vf, int nvt, int i0,
                                                                        const double* __restrict__ w, size_t len,
                                                                        double* __restrict__ partial, int nv, int ld,
                                                                        int S, size_t stage_stride, double* err) {
  multidot_df_stream<CNT, WITH_NORM>(Vf, nvt, i0, w, len, partial, nv, ld, S, stage_stride, err);
}

// device-resident index: nv = *jdev + 1 vectors; launch `chunk` of the balanced split
// (exits when nv needs fewer chunks)
template <bool WITH_NORM>
__global__ void __launch_bounds__(kStreamThreads, 1) multidot_df_dyn_kernel(const float* __restrict__ Vf, int nvt,
                                                                            int chunk, const double* __restrict__ w,
                                                                            const int* __restrict__ jdev, size_t len,
                                                                            double* __restrict__ partial, int ld,
                                                                            int S, size_t stage_stride, double* err) {
  const int nv = *jdev + 1;
  if (chunk >= (nv + kChunk - 1) / kChunk) return;
  if (!PC_DOK(nv < nvt && (len & 1) == 0, 201)) return;  // vector nv and the tiles exist
  int i0, cnt;
  balanced_chunk(nv, chunk, &i0, &cnt);
  switch (cnt) {
#define PCOPT_DYN(k) \
  case k: multidot_df_stream<k, WITH_NORM>(Vf, nvt, i0, w, len, partial, ld - 1, ld, S, stage_stride, err); break;
    PCOPT_DYN(1) PCOPT_DYN(2) PCOPT_DYN(3) PCOPT_DYN(4) PCOPT_DYN(5) PCOPT_DYN(6) PCOPT_DYN(7) PCOPT_DYN(8)
    PCOPT_DYN(9) PCOPT_DYN(10) PCOPT_DYN(11) PCOPT_DYN(12) PCOPT_DYN(13) PCOPT_DYN(14) PCOPT_DYN(15) PCOPT_DYN(16)
#undef PCOPT_DYN
    default: break;
  }
}

// First pass, update: vector nv = (w - sum_{i < nv} coef_i V_i) * scale (double-float),
// vf = its hi plane (contiguous), partial[b] = CTA sum of |w - sum|^2 (FP64, before
// scaling).  The stream walks (tile, group of 16 vectors) items; w is copied with a
// tile's first group.  With jdev: nv = *jdev + 1.
__global__ void __launch_bounds__(kStreamThreads, 1) update_df_kernel(float* Vf, int nvt, int nv,
                                                                      const double* __restrict__ coef,
                                                                      const double* __restrict__ w, float* vf,
                                                                      size_t len, const double* __restrict__ scale,
                                                                      double* __restrict__ partial,
                                                                      const int* __restrict__ jdev, int S,
                                                                      size_t stage_stride, double* err) {
  if (jdev) nv = *jdev + 1;
  if (!PC_DOK(nv >= 1 && nv < nvt && nv <= 1024 && (len & 1) == 0, 202)) return;
  __shared__ float2 cf[1024];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    float hi, lo;
    split_f64(coef[i], hi, lo);
    cf[i] = make_float2(hi, lo);
  }
  float sh = 1.0f, sl = 0.0f;
  if (scale) split_f64(scale[0], sh, sl);
  const int G = (nv + kGroup - 1) / kGroup;  // groups of 16 (the last one holds the rest)
  const size_t ntiles = (len + kTile - 1) / kTile;
  const size_t mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  float ah[2], al[2], bh[2], bl[2];  // two elements x (even, odd) double-float partial sums
  double acc = 0.0;
  auto issue = [&](size_t k, unsigned char* st, uint64_t* bar, int lane) {
    const size_t e0 = (blockIdx.x + (k / G) * gridDim.x) * (size_t)kTile;
    const int g = (int)(k % G);
    const int i0 = g * kGroup, cnt = nv - i0 < kGroup ? nv - i0 : kGroup;
    const size_t n = len - e0 < (size_t)kTile ? len - e0 : (size_t)kTile;
    const uint32_t vb = (uint32_t)cnt * 2 * kTile * 4, db = (uint32_t)(n * 8);
    // copy 0: the tile of vectors i0 .. i0 + cnt - 1 (contiguous); copy 1 (first group): w
    issue_copies(bar, vb + (g == 0 ? db : 0u), g == 0 ? 2 : 1, lane, [&](int c) {
      if (c == 0)
        bulk_copy_g2s(st, Vf + df_at(nvt, i0, e0, 0), vb, bar);
      else
        bulk_copy_g2s(st + (size_t)2 * kGroup * kTile * 4, w + e0, db, bar);
    });
  };
  // thread t takes elements 2t and 2t + 1 of a tile; each element's sum runs in two
  // double-float accumulators (even and odd vectors) for four independent chains
  auto consume = [&](size_t k, const unsigned char* st) {
    const size_t e0 = (blockIdx.x + (k / G) * gridDim.x) * (size_t)kTile;
    if (e0 + 2 * threadIdx.x >= len) return;
    const int g = (int)(k % G);
    const int i0 = g * kGroup, cnt = nv - i0 < kGroup ? nv - i0 : kGroup;
    const float2* sv = reinterpret_cast<const float2*>(st);
    if (g == 0) {
      const double2 w2 = reinterpret_cast<const double2*>(st + (size_t)2 * kGroup * kTile * 4)[threadIdx.x];
      split_f64(w2.x, ah[0], al[0]);
      split_f64(w2.y, ah[1], al[1]);
      bh[0] = bl[0] = bh[1] = bl[1] = 0.0f;
    }
    int c = 0;
    auto pair = [&](int cc) {
      const float2 c0 = cf[i0 + cc], c1 = cf[i0 + cc + 1];
      const float2 h0 = sv[(2 * cc) * (kTile / 2) + threadIdx.x], l0 = sv[(2 * cc + 1) * (kTile / 2) + threadIdx.x];
      const float2 h1 = sv[(2 * cc + 2) * (kTile / 2) + threadIdx.x], l1 = sv[(2 * cc + 3) * (kTile / 2) + threadIdx.x];
      df_sub_prod(c0.x, c0.y, h0.x, l0.x, ah[0], al[0]);
      df_sub_prod(c0.x, c0.y, h0.y, l0.y, ah[1], al[1]);
      df_sub_prod(c1.x, c1.y, h1.x, l1.x, bh[0], bl[0]);
      df_sub_prod(c1.x, c1.y, h1.y, l1.y, bh[1], bl[1]);
    };
    if (cnt == kGroup) {  // a full group: unrolled, so the shared loads run ahead of the sums
#pragma unroll
      for (int cc = 0; cc < kGroup; cc += 2) pair(cc);
      c = kGroup;
    } else {
      for (; c + 1 < cnt; c += 2) pair(c);
    }
    if (c < cnt) {
      const float2 c0 = cf[i0 + c];
      const float2 h0 = sv[(2 * c) * (kTile / 2) + threadIdx.x], l0 = sv[(2 * c + 1) * (kTile / 2) + threadIdx.x];
      df_sub_prod(c0.x, c0.y, h0.x, l0.x, ah[0], al[0]);
      df_sub_prod(c0.x, c0.y, h0.y, l0.y, ah[1], al[1]);
    }
    if (g == G - 1) {
      float hv[2], lv[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        // (ah, al) + (bh, bl) in double-float, then normalised
        float hi = __fadd_rn(ah[q], bh[q]);
        const float bb = __fsub_rn(hi, ah[q]);
        float lo = __fadd_rn(__fsub_rn(ah[q], __fsub_rn(hi, bb)), __fsub_rn(bh[q], bb));
        lo = __fadd_rn(lo, __fadd_rn(al[q], bl[q]));
        df_renorm(hi, lo);
        const double x = f32_to_f64(hi) + f32_to_f64(lo);
        acc = fma(x, x, acc);
        if (scale) df_scale(hi, lo, sh, sl);
        hv[q] = hi;
        lv[q] = lo;
      }
      float* o = Vf + df_at(nvt, nv, e0, 0);
      reinterpret_cast<float2*>(o)[threadIdx.x] = make_float2(hv[0], hv[1]);
      reinterpret_cast<float2*>(o + kTile)[threadIdx.x] = make_float2(lv[0], lv[1]);
      reinterpret_cast<float2*>(vf + e0)[threadIdx.x] = make_float2(hv[0], hv[1]);
    }
  };
  __syncthreads();  // coefficients staged
  stream_items(mine * (size_t)G, S, stage_stride, issue, consume, err);
  __shared__ double red[kStreamThreads / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kStreamThreads / 32; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

// Second pass (re-orthogonalisation, gated): e_c = hi_{i0+c} . x with x the hi plane of
// the new vector nv (FP32 products of hi planes: the coefficients removed here are ~1e-6).
template <int CNT>
__device__ __forceinline__ void multidot_lp_body(const float* __restrict__ Vf, int nvt, int i0, int nv, size_t len,
                                                 double* __restrict__ partial, int ld) {
  float s[CNT];
#pragma unroll
  for (int c = 0; c < CNT; ++c) s[c] = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const float x = Vf[df_at(nvt, nv, e, 0)];
    const float* vb = Vf + df_at(nvt, i0, e, 0);  // vector i0 + c at vb + 2 c kTile
#pragma unroll
    for (int c = 0; c < CNT; ++c) s[c] = fmaf(__ldg(vb + (size_t)2 * c * kTile), x, s[c]);
  }
  __shared__ double red[kThreads / 32][CNT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    const double v = warp_sum(f32_to_f64(s[c]));
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < CNT) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q][threadIdx.x];
    partial[(size_t)blockIdx.x * ld + i0 + threadIdx.x] = t;
  }
}

template <int CNT>
__global__ void __launch_bounds__(kThreads) multidot_lp_kernel(const float* __restrict__ Vf, int nvt, int i0, int nv,
                                                               size_t len, double* __restrict__ partial, int ld,
                                                               const double* __restrict__ gate) {
  if (gated_off(gate)) return;
  multidot_lp_body<CNT>(Vf, nvt, i0, nv, len, partial, ld);
}

__global__ void __launch_bounds__(kThreads) multidot_lp_dyn_kernel(const float* __restrict__ Vf, int nvt, int i0,
                                                                   const int* __restrict__ jdev, size_t len,
                                                                   double* __restrict__ partial, int ld,
                                                                   const double* __restrict__ gate) {
  if (gated_off(gate)) return;
  const int nv = *jdev + 1;
  if (i0 >= nv) return;
  if (!PC_DOK(nv < nvt, 205)) return;
  const int cnt = nv - i0 < kChunk ? nv - i0 : kChunk;
  switch (cnt) {
#define PCOPT_DYN(k) \
  case k: multidot_lp_body<k>(Vf, nvt, i0, nv, len, partial, ld); break;
    PCOPT_DYN(1) PCOPT_DYN(2) PCOPT_DYN(3) PCOPT_DYN(4) PCOPT_DYN(5) PCOPT_DYN(6) PCOPT_DYN(7) PCOPT_DYN(8)
    PCOPT_DYN(9) PCOPT_DYN(10) PCOPT_DYN(11) PCOPT_DYN(12) PCOPT_DYN(13) PCOPT_DYN(14) PCOPT_DYN(15) PCOPT_DYN(16)
#undef PCOPT_DYN
    default: break;
  }
}

// Second pass update (gated): vector nv -= sum_i e_i hi_i (FP32 sum of hi planes) in
// place; partial[b] = block sum of |v|^2.  With jdev: nv = *jdev + 1.
__global__ void __launch_bounds__(kThreads) update_lp_kernel(float* Vf, int nvt, int nv,
                                                             const double* __restrict__ coef, size_t len,
                                                             double* __restrict__ partial,
                                                             const double* __restrict__ gate,
                                                             const int* __restrict__ jdev) {
  if (gated_off(gate)) return;
  if (jdev) nv = *jdev + 1;
  if (!PC_DOK(nv >= 1 && nv < nvt && nv <= 1024, 203)) return;
  __shared__ float cf[1024];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cf[i] = (float)coef[i];
  __syncthreads();
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    float* o = Vf + df_at(nvt, nv, e, 0);
    float ah = o[0], al = o[kTile];
    const float* vb = Vf + df_at(nvt, 0, e, 0);  // vector i at vb + 2 i kTile
    float sf = 0.0f;
    for (int i = 0; i < nv; ++i) sf = fmaf(cf[i], __ldg(vb + (size_t)2 * i * kTile), sf);
    const float s2 = __fsub_rn(ah, sf);
    const float bb = __fsub_rn(s2, ah);
    al = __fadd_rn(al, __fadd_rn(__fsub_rn(ah, __fsub_rn(s2, bb)), __fsub_rn(neg_f(sf), bb)));
    ah = s2;
    df_renorm(ah, al);
    const double x = f32_to_f64(ah) + f32_to_f64(al);
    acc = fma(x, x, acc);
    o[0] = ah;
    o[kTile] = al;
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

// vector 0 = src / sqrt(nrm2[0]) in double-float (a zero norm copies src unscaled), vf = hi
__global__ void split_scale_kernel(const double* __restrict__ src, float* __restrict__ Vf, int nvt, float* vf,
                                   size_t len, const double* __restrict__ nrm2) {
  const bool nz = nrm2[0] > 0.0;
  const double q = nz ? 1.0 / sqrt(nrm2[0]) : 1.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    float hi, lo;
    split_f64(src[e] * q, hi, lo);
    float* o = Vf + df_at(nvt, 0, e, 0);
    o[0] = hi;
    o[kTile] = lo;
    vf[e] = hi;
  }
}

// vector nv *= 1/sqrt(nrm2[0]) in double-float, vf = its hi plane (gated; with jdev
// nv = *jdev + 1)
__global__ void scale_df_kernel(float* Vf, int nvt, int nv, float* vf, size_t len, const double* __restrict__ nrm2,
                                const double* __restrict__ gate, const int* __restrict__ jdev) {
  if (gated_off(gate)) return;
  if (jdev) nv = *jdev + 1;
  if (!PC_DOK(nv >= 0 && nv < nvt, 204)) return;
  if (!(nrm2[0] > 0.0)) return;
  float sh, sl;
  split_f64(1.0 / sqrt(nrm2[0]), sh, sl);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    float* o = Vf + df_at(nvt, nv, e, 0);
    float hi = o[0], lo = o[kTile];
    df_scale(hi, lo, sh, sl);
    o[0] = hi;
    o[kTile] = lo;
    vf[e] = hi;
  }
}

// blocks that fit the device at once for kernel `fn` (one wave), capped by the work size
template <typename K>
unsigned wave_blocks(K fn, size_t smem, size_t len) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  if (per_sm > kMaxBlocksPerSM) per_sm = kMaxBlocksPerSM;
  size_t b = (size_t)num_sms() * per_sm;
  const size_t need = (len + kThreads - 1) / kThreads;
  if (need < b) b = need ? need : 1;
  return (unsigned)b;
}

unsigned stream_blocks(size_t len) {
  size_t b = (len + kThreads - 1) / kThreads;
  const size_t cap = (size_t)num_sms() * 8;
  return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

ChunkGrids one_grid(unsigned nb) {
  ChunkGrids g;
  for (int c = 0; c < kMaxChunks; ++c) g.nb[c] = nb;
  return g;
}

template <int CNT, bool N>
cudaError_t multidot_chunk(Launch& L, const double* V, size_t ldv, int i0, const double* w, size_t len,
                           double* partial, int nv, int ld, const double* gate, unsigned* blocks_out, bool lp) {
  // gated launches are the re-orthogonalisation pass: FP32 products (see the file header)
  // unless lp is false (FP64 products throughout)
  auto kern = (gate && lp) ? multidot_kernel<CNT, N, true> : multidot_kernel<CNT, N, false>;
  const unsigned nb = wave_blocks(kern, 0, len);
  *blocks_out = nb;
  const int kc = gate ? KC_REORTH : KC_DOT;
  L.begin(kc);
  kern<<<nb, kThreads, 0, L.stream>>>(V, ldv, i0, w, len, partial, nv, ld, gate);
  return gate ? L.end(kc, 0.0, 0.0) : L.end(kc, 8.0 * len * (CNT + 1), 2.0 * len * (CNT + (N ? 1 : 0)));
}

template <bool N>
cudaError_t multidot_dispatch(int cnt, Launch& L, const double* V, size_t ldv, int i0, const double* w, size_t len,
                              double* partial, int nv, int ld, const double* gate, unsigned* nb, bool lp) {
  switch (cnt) {
#define PCOPT_CASE(k) \
  case k: return multidot_chunk<k, N>(L, V, ldv, i0, w, len, partial, nv, ld, gate, nb, lp);
    PCOPT_CASE(1) PCOPT_CASE(2) PCOPT_CASE(3) PCOPT_CASE(4) PCOPT_CASE(5) PCOPT_CASE(6) PCOPT_CASE(7)
    PCOPT_CASE(8) PCOPT_CASE(9) PCOPT_CASE(10) PCOPT_CASE(11) PCOPT_CASE(12) PCOPT_CASE(13) PCOPT_CASE(14)
    PCOPT_CASE(15) PCOPT_CASE(16)
#undef PCOPT_CASE
    default: return cudaErrorInvalidValue;
  }
}

size_t round128(size_t x) { return (x + 127) & ~(size_t)127; }

// stages of `stride` bytes that fit the streaming CTA's shared-memory budget
int stream_stages_for(size_t stride) {
  const size_t s = (kStreamSmem - kBarBytes) / stride;
  return (int)(s < 2 ? 2 : (s > 12 ? 12 : s));
}

// one streaming CTA per SM (the stages fill its shared memory), at most one per tile
unsigned stream_grid(size_t len) {
  const size_t ntiles = (len + kTile - 1) / kTile;
  const size_t sms = (size_t)num_sms();
  return (unsigned)(ntiles < sms ? (ntiles ? ntiles : 1) : sms);
}

template <typename K>
cudaError_t allow_smem(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int CNT, bool N>
cudaError_t multidot_df_chunk(Launch& L, const float* Vf, int nvt, int i0, const double* w, size_t len,
                              double* partial, int nv, int ld, double* err, unsigned* blocks_out) {
  const size_t stride = round128((size_t)2 * CNT * kTile * 4 + (size_t)kTile * 8);
  const int S = stream_stages_for(stride);
  const size_t smem = kBarBytes + S * stride;
  auto kern = multidot_df_kernel<CNT, N>;
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned nb = stream_grid(len);
  *blocks_out = nb;
  L.begin(KC_DOT);
  kern<<<nb, kStreamThreads, smem, L.stream>>>(Vf, nvt, i0, w, len, partial, nv, ld, S, stride, err);
  return L.end(KC_DOT, 8.0 * len * (CNT + 1), 2.0 * len * (CNT + (N ? 1 : 0)));
}

template <bool N>
cudaError_t multidot_df_dispatch(int cnt, Launch& L, const float* Vf, int nvt, int i0, const double* w,
                                 size_t len, double* partial, int nv, int ld, double* err, unsigned* nb) {
  switch (cnt) {
#define PCOPT_CASE(k) \
  case k: return multidot_df_chunk<k, N>(L, Vf, nvt, i0, w, len, partial, nv, ld, err, nb);
    PCOPT_CASE(1) PCOPT_CASE(2) PCOPT_CASE(3) PCOPT_CASE(4) PCOPT_CASE(5) PCOPT_CASE(6) PCOPT_CASE(7)
    PCOPT_CASE(8) PCOPT_CASE(9) PCOPT_CASE(10) PCOPT_CASE(11) PCOPT_CASE(12) PCOPT_CASE(13) PCOPT_CASE(14)
    PCOPT_CASE(15) PCOPT_CASE(16)
#undef PCOPT_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int CNT>
cudaError_t multidot_lp_chunk(Launch& L, const float* Vf, int nvt, int i0, int nv, size_t len, double* partial, int ld,
                              const double* gate, unsigned* blocks_out) {
  auto kern = multidot_lp_kernel<CNT>;
  const unsigned nb = wave_blocks(kern, 0, len);
  *blocks_out = nb;
  L.begin(KC_REORTH);
  kern<<<nb, kThreads, 0, L.stream>>>(Vf, nvt, i0, nv, len, partial, ld, gate);
  return L.end(KC_REORTH, 0.0, 0.0);
}

cudaError_t multidot_lp_dispatch(int cnt, Launch& L, const float* Vf, int nvt, int i0, int nv, size_t len,
                                 double* partial, int ld, const double* gate, unsigned* nb) {
  switch (cnt) {
#define PCOPT_CASE(k) \
  case k: return multidot_lp_chunk<k>(L, Vf, nvt, i0, nv, len, partial, ld, gate, nb);
    PCOPT_CASE(1) PCOPT_CASE(2) PCOPT_CASE(3) PCOPT_CASE(4) PCOPT_CASE(5) PCOPT_CASE(6) PCOPT_CASE(7)
    PCOPT_CASE(8) PCOPT_CASE(9) PCOPT_CASE(10) PCOPT_CASE(11) PCOPT_CASE(12) PCOPT_CASE(13) PCOPT_CASE(14)
    PCOPT_CASE(15) PCOPT_CASE(16)
#undef PCOPT_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_multidot(Launch& L, const double* V, size_t ldv, int nv, const double* w, size_t len,
                            double* partial, double* out, double* ww, const double* gate, bool lp_reorth) {
  if (nv < 1 || nv > kChunk * kMaxChunks) return cudaErrorInvalidValue;
  const int ld = nv + 1;
  ChunkGrids cg = one_grid(1);
  double nb_sum = 0;
  for (int i0 = 0, c = 0; i0 < nv; i0 += kChunk, ++c) {
    const int cnt = nv - i0 < kChunk ? nv - i0 : kChunk;
    unsigned nb = 0;
    cudaError_t e =
        (i0 == 0 && ww) ? multidot_dispatch<true>(cnt, L, V, ldv, i0, w, len, partial, nv, ld, gate, &nb, lp_reorth)
                        : multidot_dispatch<false>(cnt, L, V, ldv, i0, w, len, partial, nv, ld, gate, &nb, lp_reorth);
    if (e != cudaSuccess) return e;
    cg.nb[c] = nb;
    nb_sum += nb * (double)cnt;
  }
  const int ncols = nv + (ww ? 1 : 0);
  const int kc = gate ? KC_REORTH : KC_REDUCE;
  L.begin(kc);
  reduce_partials_kernel<<<ncols, kThreads, 0, L.stream>>>(partial, cg, ld, out, ww, nv, gate, nullptr);
  return gate ? L.end(kc, 0.0, 0.0) : L.end(kc, 8.0 * nb_sum, nb_sum);
}

cudaError_t launch_update(Launch& L, const double* V, size_t ldv, int nv, const double* coef, double* v, size_t len,
                          const double* scale, double* partial, double* q, const double* gate, float* vf,
                          bool lp_reorth) {
  const size_t smem = sizeof(double) * (nv > 0 ? nv : 1);
  auto kern = (gate && lp_reorth) ? update_kernel<true> : update_kernel<false>;  // gated: re-orthogonalisation
  const unsigned nb = wave_blocks(kern, smem, len);
  const int kc = gate ? KC_REORTH : KC_UPDATE;
  L.begin(kc);
  kern<<<nb, kThreads, smem, L.stream>>>(V, ldv, nv, coef, v, len, scale, partial, gate, nullptr, 0, vf);
  cudaError_t e = gate ? L.end(kc, 0.0, 0.0)
                       : L.end(kc, 8.0 * len * (nv + 2) + (vf ? 4.0 * len : 0.0), 2.0 * len * (nv + 1));
  if (e != cudaSuccess) return e;
  const int kr = gate ? KC_REORTH : KC_REDUCE;
  L.begin(kr);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, one_grid(nb), 1, q, q, 1, gate, nullptr);
  return gate ? L.end(kr, 0.0, 0.0) : L.end(kr, 8.0 * nb, 1.0 * nb);
}

cudaError_t launch_norm2(Launch& L, const double* w, size_t len, double* partial, double* nrm2) {
  const unsigned nb = wave_blocks(norm2_kernel, 0, len);
  L.begin(KC_DOT);
  norm2_kernel<<<nb, kThreads, 0, L.stream>>>(w, len, partial);
  cudaError_t e = L.end(KC_DOT, 8.0 * len, 2.0 * len);
  if (e != cudaSuccess) return e;
  L.begin(KC_REDUCE);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, one_grid(nb), 1, nrm2, nrm2, 1, nullptr,
                                                       nullptr);
  return L.end(KC_REDUCE, 8.0 * nb, 1.0 * nb);
}

cudaError_t launch_scale_by_inv_norm(Launch& L, double* v, size_t len, const double* nrm2, const double* gate,
                                     float* vf) {
  const int kc = gate ? KC_REORTH : KC_SCALE;
  L.begin(kc);
  scale_kernel<<<stream_blocks(len), kThreads, 0, L.stream>>>(v, len, nrm2, gate, nullptr, 0, vf);
  return gate ? L.end(kc, 0.0, 0.0) : L.end(kc, 16.0 * len + (vf ? 4.0 * len : 0.0), 1.0 * len);
}

template <typename Tx>
cudaError_t launch_axpby(Launch& L, double a, const Tx* x, double b, double* y, size_t len) {
  L.begin(KC_AXPBY);
  axpby_kernel<Tx><<<stream_blocks(len), kThreads, 0, L.stream>>>(a, x, b, y, len);
  return L.end(KC_AXPBY, (double)len * (sizeof(Tx) + (b == 0.0 ? 8.0 : 16.0)), 3.0 * len);
}
template cudaError_t launch_axpby<double>(Launch&, double, const double*, double, double*, size_t);
template cudaError_t launch_axpby<float>(Launch&, double, const float*, double, double*, size_t);

cudaError_t launch_arnoldi_prep(Launch& L, int nv, const double* d, ArnoldiScalars s) {
  L.begin(KC_GIVENS);
  arnoldi_prep_kernel<<<1, 32, 0, L.stream>>>(nv, d, s, nullptr);
  return L.end(KC_GIVENS, 0.0, 2.0 * nv);
}

cudaError_t launch_arnoldi_check(Launch& L, ArnoldiScalars s) {
  L.begin(KC_GIVENS);
  arnoldi_check_kernel<<<1, 32, 0, L.stream>>>(s);
  return L.end(KC_GIVENS, 0.0, 4.0);
}

cudaError_t launch_givens(Launch& L, int j, int ldh, double* H, double* cs, double* sn, double* gvec, const double* d,
                          const double* e, ArnoldiScalars s, double* est, const double* ref) {
  L.begin(KC_GIVENS);
  givens_kernel<<<1, 32, 0, L.stream>>>(j, ldh, H, cs, sn, gvec, d, e, s, est, ref, nullptr);
  return L.end(KC_GIVENS, 0.0, 10.0 * (j + 1));
}

cudaError_t launch_backsolve(Launch& L, int k, int ldh, const double* H, const double* gvec, double* y) {
  L.begin(KC_GIVENS);
  backsolve_kernel<<<1, 32, 0, L.stream>>>(k, ldh, H, gvec, y, nullptr);
  return L.end(KC_GIVENS, 0.0, 1.0 * k * k);
}

template <typename Tz>
cudaError_t launch_xupdate(Launch& L, const Tz* Z, size_t ldz, int k, const double* y, double* x, size_t len) {
  const size_t smem = sizeof(double) * (k > 0 ? k : 1);
  L.begin(KC_XUPDATE);
  xupdate_kernel<Tz><<<wave_blocks(xupdate_kernel<Tz>, smem, len), kThreads, smem, L.stream>>>(Z, ldz, k, y, x, len,
                                                                                               nullptr);
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

// ---------------------------------------------------------------------------
// double-float basis in the tiled layout (df_at); vector nv is the new one
cudaError_t launch_multidot_df(Launch& L, const float* Vf, int nvt, int nv, const double* w, size_t len,
                               double* partial, double* out, double* ww, const double* gate, double* err) {
  if (nv < 1 || nv >= nvt || nv > kChunk * kMaxChunks) return cudaErrorInvalidValue;
  if (len & 1) return cudaErrorInvalidValue;  // the streamed tiles need an even length
  const bool lp = gate != nullptr;  // gated launches are the re-orthogonalisation pass
  const int ld = nv + 1;
  ChunkGrids cg = one_grid(1);
  double nb_sum = 0;
  if (lp) {  // fixed chunks of 16 (their grids differ with the chunk's register use)
    for (int i0 = 0, c = 0; i0 < nv; i0 += kChunk, ++c) {
      const int cnt = nv - i0 < kChunk ? nv - i0 : kChunk;
      unsigned nb = 0;
      cudaError_t e = multidot_lp_dispatch(cnt, L, Vf, nvt, i0, nv, len, partial, ld, gate, &nb);
      if (e != cudaSuccess) return e;
      cg.nb[c] = nb;
      nb_sum += nb * (double)cnt;
    }
  } else {  // balanced chunks, every one on the same streaming grid
    const int nch = (nv + kChunk - 1) / kChunk;
    unsigned nb = 0;
    for (int c = 0; c < nch; ++c) {
      int i0, cnt;
      balanced_chunk(nv, c, &i0, &cnt);
      cudaError_t e = (i0 == 0 && ww) ? multidot_df_dispatch<true>(cnt, L, Vf, nvt, i0, w, len, partial, nv, ld, err, &nb)
                                      : multidot_df_dispatch<false>(cnt, L, Vf, nvt, i0, w, len, partial, nv, ld, err, &nb);
      if (e != cudaSuccess) return e;
      nb_sum += nb * (double)cnt;
    }
    cg = one_grid(nb);
  }
  const int ncols = nv + (ww && !lp ? 1 : 0);
  const int kc = lp ? KC_REORTH : KC_REDUCE;
  L.begin(kc);
  reduce_partials_kernel<<<ncols, kThreads, 0, L.stream>>>(partial, cg, ld, out, lp ? nullptr : ww, nv, gate,
                                                          nullptr);
  return lp ? L.end(kc, 0.0, 0.0) : L.end(kc, 8.0 * nb_sum, nb_sum);
}

cudaError_t launch_update_df(Launch& L, float* Vf, int nvt, int nv, const double* coef, const double* w, float* vf,
                             size_t len, const double* scale, double* partial, double* q, const double* gate,
                             double* err) {
  if (nv < 1 || nv >= nvt || nv > 1024) return cudaErrorInvalidValue;
  if (len & 1) return cudaErrorInvalidValue;
  const bool lp = gate != nullptr;
  unsigned nb;
  cudaError_t e;
  if (lp) {
    nb = wave_blocks(update_lp_kernel, 0, len);
    L.begin(KC_REORTH);
    update_lp_kernel<<<nb, kThreads, 0, L.stream>>>(Vf, nvt, nv, coef, len, partial, gate, nullptr);
    e = L.end(KC_REORTH, 0.0, 0.0);
  } else {
    const size_t stride = round128((size_t)2 * kGroup * kTile * 4 + (size_t)kTile * 8);
    const int S = stream_stages_for(stride);
    const size_t smem = kBarBytes + S * stride;
    if ((e = allow_smem(update_df_kernel, smem)) != cudaSuccess) return e;
    nb = stream_grid(len);
    L.begin(KC_UPDATE);
    update_df_kernel<<<nb, kStreamThreads, smem, L.stream>>>(Vf, nvt, nv, coef, w, vf, len, scale, partial, nullptr, S,
                                                            stride, err);
    e = L.end(KC_UPDATE, 8.0 * len * (nv + 2) + 4.0 * len, 2.0 * len * (nv + 1));
  }
  if (e != cudaSuccess) return e;
  const int kr = lp ? KC_REORTH : KC_REDUCE;
  L.begin(kr);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, one_grid(nb), 1, q, q, 1, gate, nullptr);
  return lp ? L.end(kr, 0.0, 0.0) : L.end(kr, 8.0 * nb, 1.0 * nb);
}

cudaError_t launch_split_scale(Launch& L, const double* src, float* Vf, int nvt, float* vf, size_t len,
                               const double* nrm2) {
  L.begin(KC_SCALE);
  split_scale_kernel<<<stream_blocks(len), kThreads, 0, L.stream>>>(src, Vf, nvt, vf, len, nrm2);
  return L.end(KC_SCALE, 20.0 * len, 2.0 * len);
}

cudaError_t launch_scale_df(Launch& L, float* Vf, int nvt, int nv, float* vf, size_t len, const double* nrm2,
                            const double* gate) {
  const int kc = gate ? KC_REORTH : KC_SCALE;
  L.begin(kc);
  scale_df_kernel<<<stream_blocks(len), kThreads, 0, L.stream>>>(Vf, nvt, nv, vf, len, nrm2, gate, nullptr);
  return gate ? L.end(kc, 0.0, 0.0) : L.end(kc, 20.0 * len, 1.0 * len);
}

cudaError_t launch_multidot_df_dev(Launch& L, const float* Vf, int nvt, int nv_max, const int* jdev, const double* w,
                                   size_t len, double* partial, double* out, double* ww, const double* gate,
                                   double* err) {
  if (nv_max < 1 || nv_max >= nvt || nv_max > kChunk * kMaxChunks) return cudaErrorInvalidValue;
  if (len & 1) return cudaErrorInvalidValue;
  const bool lp = gate != nullptr;
  const int ld = nv_max + 1;
  const int kc = lp ? KC_REORTH : KC_DOT;
  ChunkGrids cg;
  if (lp) {
    const unsigned nb = wave_blocks(multidot_lp_dyn_kernel, 0, len);
    cg = one_grid(nb);
    for (int i0 = 0; i0 < nv_max; i0 += kChunk) {
      L.begin(kc);
      multidot_lp_dyn_kernel<<<nb, kThreads, 0, L.stream>>>(Vf, nvt, i0, jdev, len, partial, ld, gate);
      cudaError_t e = L.end(kc, 0.0, 0.0);
      if (e != cudaSuccess) return e;
    }
  } else {
    const size_t stride = round128((size_t)2 * kChunk * kTile * 4 + (size_t)kTile * 8);
    const int S = stream_stages_for(stride);
    const size_t smem = kBarBytes + S * stride;
    cudaError_t e = allow_smem(multidot_df_dyn_kernel<true>, smem);
    if (e == cudaSuccess) e = allow_smem(multidot_df_dyn_kernel<false>, smem);
    if (e != cudaSuccess) return e;
    const unsigned nb = stream_grid(len);
    cg = one_grid(nb);
    for (int c = 0; c < (nv_max + kChunk - 1) / kChunk; ++c) {
      L.begin(kc);
      if (c == 0 && ww)
        multidot_df_dyn_kernel<true><<<nb, kStreamThreads, smem, L.stream>>>(Vf, nvt, c, w, jdev, len, partial, ld,
                                                                            S, stride, err);
      else
        multidot_df_dyn_kernel<false><<<nb, kStreamThreads, smem, L.stream>>>(Vf, nvt, c, w, jdev, len, partial, ld,
                                                                             S, stride, err);
      e = L.end(kc, 0.0, 0.0);
      if (e != cudaSuccess) return e;
    }
  }
  L.begin(kc);
  reduce_partials_kernel<<<nv_max + (ww && !lp ? 1 : 0), kThreads, 0, L.stream>>>(partial, cg, ld, out,
                                                                                 lp ? nullptr : ww, nv_max, gate,
                                                                                 jdev);
  return L.end(kc, 0.0, 0.0);
}

cudaError_t launch_update_df_dev(Launch& L, float* Vf, int nvt, int nv_max, const int* jdev, const double* coef,
                                 const double* w, float* vf, size_t len, const double* scale, double* partial,
                                 double* q, const double* gate, double* err) {
  if (nv_max < 1 || nv_max >= nvt || nv_max > 1024) return cudaErrorInvalidValue;
  if (len & 1) return cudaErrorInvalidValue;
  const bool lp = gate != nullptr;
  const int kc = lp ? KC_REORTH : KC_UPDATE;
  unsigned nb;
  cudaError_t e;
  L.begin(kc);
  if (lp) {
    nb = wave_blocks(update_lp_kernel, 0, len);
    update_lp_kernel<<<nb, kThreads, 0, L.stream>>>(Vf, nvt, nv_max, coef, len, partial, gate, jdev);
  } else {
    const size_t stride = round128((size_t)2 * kGroup * kTile * 4 + (size_t)kTile * 8);
    const int S = stream_stages_for(stride);
    const size_t smem = kBarBytes + S * stride;
    if ((e = allow_smem(update_df_kernel, smem)) != cudaSuccess) return e;
    nb = stream_grid(len);
    update_df_kernel<<<nb, kStreamThreads, smem, L.stream>>>(Vf, nvt, nv_max, coef, w, vf, len, scale, partial, jdev,
                                                            S, stride, err);
  }
  e = L.end(kc, 0.0, 0.0);
  if (e != cudaSuccess) return e;
  L.begin(kc);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, one_grid(nb), 1, q, q, 1, gate, nullptr);
  return L.end(kc, 0.0, 0.0);
}

cudaError_t launch_scale_df_dev(Launch& L, float* Vf, int nvt, const int* jdev, float* vf, size_t len,
                                const double* nrm2, const double* gate) {
  L.begin(KC_REORTH);
  scale_df_kernel<<<stream_blocks(len), kThreads, 0, L.stream>>>(Vf, nvt, 0, vf, len, nrm2, gate, jdev);
  return L.end(KC_REORTH, 0.0, 0.0);
}

// ---------------------------------------------------------------------------
// device-index launchers: every launch below is independent of the iteration
// index, which the kernels read from `jdev`, so one captured iteration serves all
cudaError_t launch_multidot_dev(Launch& L, const double* V, size_t ldv, int nv_max, const int* jdev,
                                const double* wbase, size_t wstride, size_t len, double* partial, double* out,
                                double* ww, const double* gate, bool lp_reorth) {
  if (nv_max < 1 || nv_max > kChunk * kMaxChunks) return cudaErrorInvalidValue;
  const int ld = nv_max + 1;
  // gated launches are the re-orthogonalisation pass: FP32 products (see the file header)
  auto plain = (gate && lp_reorth) ? multidot_dyn_kernel<false, true> : multidot_dyn_kernel<false, false>;
  const unsigned nb_norm = wave_blocks(multidot_dyn_kernel<true>, 0, len);
  const unsigned nb_plain = wave_blocks(plain, 0, len);
  ChunkGrids cg = one_grid(nb_plain);
  const int kc = gate ? KC_REORTH : KC_DOT;
  for (int i0 = 0, c = 0; i0 < nv_max; i0 += kChunk, ++c) {
    L.begin(kc);
    if (i0 == 0 && ww) {
      cg.nb[0] = nb_norm;
      multidot_dyn_kernel<true><<<nb_norm, kThreads, 0, L.stream>>>(V, ldv, i0, wbase, wstride, jdev, len, partial,
                                                                   ld, gate);
    } else {
      plain<<<nb_plain, kThreads, 0, L.stream>>>(V, ldv, i0, wbase, wstride, jdev, len, partial, ld, gate);
    }
    cudaError_t e = L.end(kc, 0.0, 0.0);
    if (e != cudaSuccess) return e;
  }
  L.begin(kc);
  reduce_partials_kernel<<<nv_max + (ww ? 1 : 0), kThreads, 0, L.stream>>>(partial, cg, ld, out, ww, nv_max, gate,
                                                                          jdev);
  return L.end(kc, 0.0, 0.0);
}

cudaError_t launch_update_dev(Launch& L, const double* V, size_t ldv, int nv_max, const int* jdev, const double* coef,
                              double* vbase, size_t vstride, size_t len, const double* scale, double* partial,
                              double* q, const double* gate, float* vf, bool lp_reorth) {
  const size_t smem = sizeof(double) * nv_max;
  auto kern = (gate && lp_reorth) ? update_kernel<true> : update_kernel<false>;  // gated: re-orthogonalisation
  const unsigned nb = wave_blocks(kern, smem, len);
  const int kc = gate ? KC_REORTH : KC_UPDATE;
  L.begin(kc);
  kern<<<nb, kThreads, smem, L.stream>>>(V, ldv, nv_max, coef, vbase, len, scale, partial, gate, jdev,
                                                  vstride, vf);
  cudaError_t e = L.end(kc, 0.0, 0.0);
  if (e != cudaSuccess) return e;
  L.begin(kc);
  reduce_partials_kernel<<<1, kThreads, 0, L.stream>>>(partial, one_grid(nb), 1, q, q, 1, gate, nullptr);
  return L.end(kc, 0.0, 0.0);
}

cudaError_t launch_scale_dev(Launch& L, double* vbase, size_t vstride, const int* jdev, size_t len,
                             const double* nrm2, const double* gate, float* vf) {
  L.begin(KC_REORTH);
  scale_kernel<<<stream_blocks(len), kThreads, 0, L.stream>>>(vbase, len, nrm2, gate, jdev, vstride, vf);
  return L.end(KC_REORTH, 0.0, 0.0);
}

cudaError_t launch_arnoldi_prep_dev(Launch& L, const int* jdev, const double* d, ArnoldiScalars s) {
  L.begin(KC_GIVENS);
  arnoldi_prep_kernel<<<1, 32, 0, L.stream>>>(0, d, s, jdev);
  return L.end(KC_GIVENS, 0.0, 0.0);
}

cudaError_t launch_givens_dev(Launch& L, const int* jdev, int ldh, double* H, double* cs, double* sn, double* gvec,
                              const double* d, const double* e, ArnoldiScalars s, double* est, const double* ref) {
  L.begin(KC_GIVENS);
  givens_kernel<<<1, 32, 0, L.stream>>>(0, ldh, H, cs, sn, gvec, d, e, s, est, ref, jdev);
  return L.end(KC_GIVENS, 0.0, 0.0);
}

cudaError_t launch_loop_control(Launch& L, int* jdev, int* kdev, const double* est, double rtol, int maxit,
                                cudaGraphConditionalHandle hc) {
  L.begin(KC_GIVENS);
  loop_control_kernel<<<1, 32, 0, L.stream>>>(jdev, kdev, est, rtol, maxit, hc);
  return L.end(KC_GIVENS, 0.0, 0.0);
}

cudaError_t launch_loop_start(Launch& L, int* jdev, int* kdev, const double* est, double rtol,
                              cudaGraphConditionalHandle hc) {
  L.begin(KC_GIVENS);
  loop_start_kernel<<<1, 32, 0, L.stream>>>(jdev, kdev, est, rtol, hc);
  return L.end(KC_GIVENS, 0.0, 0.0);
}

cudaError_t launch_backsolve_dev(Launch& L, const int* kdev, int ldh, const double* H, const double* gvec, double* y) {
  L.begin(KC_GIVENS);
  backsolve_kernel<<<1, 32, 0, L.stream>>>(0, ldh, H, gvec, y, kdev);
  return L.end(KC_GIVENS, 0.0, 0.0);
}

template <typename Tz>
cudaError_t launch_xupdate_dev(Launch& L, const Tz* Z, size_t ldz, int kmax, const int* kdev, const double* y,
                               double* x, size_t len) {
  const size_t smem = sizeof(double) * (kmax > 0 ? kmax : 1);
  L.begin(KC_XUPDATE);
  xupdate_kernel<Tz><<<wave_blocks(xupdate_kernel<Tz>, smem, len), kThreads, smem, L.stream>>>(Z, ldz, kmax, y, x,
                                                                                               len, kdev);
  return L.end(KC_XUPDATE, 0.0, 0.0);
}
template cudaError_t launch_xupdate_dev<double>(Launch&, const double*, size_t, int, const int*, const double*,
                                                double*, size_t);
template cudaError_t launch_xupdate_dev<float>(Launch&, const float*, size_t, int, const int*, const double*, double*,
                                               size_t);

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

PCOPT_DEBUG_READER(pcopt_debug_krylov)

}  // namespace pcopt
