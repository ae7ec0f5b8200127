// Lower part of the 2D V(1,0) cycle (Section 2.1, step 2 of the apply of
// P_eps^{-1}, variable a) in one launch: from the first level with at most 63^2
// points down to the one-point level and back, for FP32 iterates (FP64 handles keep
// the coarse-cycle kernel from 31^2: with FP64 values a plane needs one 133 KB CTA,
// which made the two-plane steps of the ideal preconditioner slower).
//
// One CTA owns one spectral plane and keeps ONE array per level in shared memory,
// updated in place:
//   down, level q (array a = r_q on entry):
//     red   (i1 + i2 even):  a = r / (sigma + d)                      -> u_red
//     black (i1 + i2 odd):   a = (r + sum_k w_k u_red(nb_k)) / (sigma + d)
//     restriction by full weighting into level q+1; the sweep starts from zero,
//     so the residual of the black points is zero and that of a red point is
//     sum_k w_k u_black(nb_k) (no r needed any more):
//       rc(I, J) = 1/4 res(2I+1, 2J+1) + 1/16 sum res(2I+1 +- 1, 2J+1 +- 1)
//     (the edge points of the 3 x 3 stencil are black);
//   one-point level: a = r / (sigma + d);
//   up: a_q += P a_{q+1} (bilinear interpolation), finest tail level stored.
// This is the arithmetic of the level-by-level kernels (same sweep, residual,
// restriction and prolongation), with one array instead of three per level, so
// that the 63^2 level fits beside the coarser ones: in FP32 two CTAs (planes) of
// 512 threads share an SM and all planes of a 255^2 x 256 apply run in one wave.
// The plane's right-hand side and the face weights and diagonals of the levels
// below the first one are staged in shared memory by cp.async, all in flight at
// once; the first level's coefficients are staged too when they fit, else they
// are read through L2 (shared by all planes).  For odd m the parity of
// s = i1 + m i2 is that of i1 + i2, so red points are the even s.
#include <algorithm>

#include "common.cuh"
#include "regfft.cuh"

namespace pcopt {

namespace {

template <typename Tc>
__host__ __device__ constexpr int tail_threads() {
  return 512;
}

// 1 / (sigma + d); FP32 with the hardware-approximate divide (2 ulp, far inside
// what a smoother needs)
__device__ __forceinline__ float2 tail_inv(float2 sig, float d) {
  const float a = sig.x + d;
  const float q = __fdividef(1.0f, fmaf(a, a, sig.y * sig.y));
  return make_float2(a * q, -sig.y * q);
}

template <typename C, typename T>
__device__ __forceinline__ void tail_fma(C& acc, T w, C v) {
  acc.x = fma(w, v.x, acc.x);
  acc.y = fma(w, v.y, acc.y);
}

// row of linear index s on an m x m level: (s + 1/2) / m is at least 1/(2m) away
// from an integer, far more than the FP32 rounding of the product for m <= 1023
__device__ __forceinline__ int row_of(int s, float rm) { return (int)(((float)s + 0.5f) * rm); }

// residual at red point (i1, i2) = linear index s: sum_k w_k u_black(nb_k)
template <typename Tc>
__device__ __forceinline__ typename Cx<Tc>::t red_residual(const typename Cx<Tc>::t* a, const Tc* w, int np, int m,
                                                           int s, int i1, int i2) {
  typedef typename Cx<Tc>::t C;
  C acc = czero<Tc>();
  if (i1 > 0) tail_fma(acc, w[s], a[s - 1]);
  if (i1 < m - 1) tail_fma(acc, w[np + s], a[s + 1]);
  if (i2 > 0) tail_fma(acc, w[2 * np + s], a[s - m]);
  if (i2 < m - 1) tail_fma(acc, w[3 * np + s], a[s + m]);
  return acc;
}

// Points per thread handled as one batch: every load of a batch is issued before
// its first store (the arrays are reached through generic pointers, so a store
// would otherwise keep the next point's loads behind it)
constexpr int kTailBatch = 4;

template <typename Tc>
__global__ void __launch_bounds__(tail_threads<Tc>(), sizeof(Tc) == 4 ? 2 : 1) mg_tail2_kernel(const CoarseLevels<Tc> lv,
                                                                      const typename Cx<Tc>::t* __restrict__ r0,
                                                                      typename Cx<Tc>::t* __restrict__ u0,
                                                                      const typename Cx<Tc>::t* __restrict__ sigma,
                                                                      int stage0) {
  typedef typename Cx<Tc>::t C;
  constexpr int NT = tail_threads<Tc>();
  constexpr int K = kTailBatch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x;
  const int tid = threadIdx.x;
  const C sig = sigma[p];
  const int nl = lv.count;
  const int np0 = (int)lv.np[0];
  C* A[kMaxCoarseLevels];
  const Tc* W[kMaxCoarseLevels];  // four face-weight planes (-x, +x, -y, +y), then the diagonal
  {
    // the plane's right-hand side and the staged coefficients, all in flight at once
    unsigned char* q = smem_raw;
    for (int l = 0; l < nl; ++l) {
      A[l] = reinterpret_cast<C*>(q);
      q += (((size_t)lv.np[l] * sizeof(C) + 15) / 16) * 16;
    }
    const C* src = r0 + (int64_t)p * np0;
    for (int s = tid; s < np0; s += NT) cp_async<sizeof(C)>(A[0] + s, src + s, true);
    for (int l = 0; l < nl; ++l) {
      const int np = (int)lv.np[l];
      if (l == 0 && !stage0) {
        W[0] = lv.w[0];
        continue;
      }
      Tc* w = reinterpret_cast<Tc*>(q);
      q += ((5 * (size_t)np * sizeof(Tc) + 15) / 16) * 16;
      const Tc* wl = lv.w[l];
      const Tc* dl = lv.diag[l];
      for (int e = tid; e < 4 * np; e += NT) cp_async<sizeof(Tc)>(w + e, wl + e, true);
      for (int e = tid; e < np; e += NT) cp_async<sizeof(Tc)>(w + 4 * np + e, dl + e, true);
      W[l] = w;
    }
    cp_async_commit();
    cp_async_wait<0>();
  }
  __syncthreads();
  // ---- down
  for (int l = 0; l < nl; ++l) {
    const int m = lv.m[l];
    const int np = (int)lv.np[l];
    C* a = A[l];
    const Tc* w = W[l];
    const Tc* dg = (l == 0 && !stage0) ? lv.diag[0] : w + 4 * np;
    // red: u = r / (sigma + d)
    for (int s0 = 2 * tid; s0 < np; s0 += 2 * NT * K) {
      C av[K];
      Tc dv[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int s = s0 + 2 * NT * i;
        av[i] = czero<Tc>();
        dv[i] = Tc(1);
        if (s < np) {
          av[i] = a[s];
          dv[i] = dg[s];
        }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int s = s0 + 2 * NT * i;
        if (s < np) a[s] = cmul(av[i], tail_inv(sig, dv[i]));
      }
    }
    if (l + 1 == nl) break;  // the one-point level is solved exactly by its red step
    __syncthreads();
    const float rm = 1.0f / (float)m;
    // black: u = (r + sum_k w_k u_red(nb_k)) / (sigma + d)
    for (int s0 = 1 + 2 * tid; s0 < np; s0 += 2 * NT * K) {
      C acc[K];
      Tc dv[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int s = s0 + 2 * NT * i;
        acc[i] = czero<Tc>();
        dv[i] = Tc(1);
        if (s < np) {
          const int i2 = row_of(s, rm);
          const int i1 = s - i2 * m;
          acc[i] = a[s];
          if (i1 > 0) tail_fma(acc[i], w[s], a[s - 1]);
          if (i1 < m - 1) tail_fma(acc[i], w[np + s], a[s + 1]);
          if (i2 > 0) tail_fma(acc[i], w[2 * np + s], a[s - m]);
          if (i2 < m - 1) tail_fma(acc[i], w[3 * np + s], a[s + m]);
          dv[i] = dg[s];
        }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int s = s0 + 2 * NT * i;
        if (s < np) a[s] = cmul(acc[i], tail_inv(sig, dv[i]));
      }
    }
    __syncthreads();
    // full weighting of the red residuals into level l + 1
    const int mc = lv.m[l + 1];
    const int npc = (int)lv.np[l + 1];
    const float rmc = 1.0f / (float)mc;
    C* ac = A[l + 1];
    for (int c0 = tid; c0 < npc; c0 += NT * K) {
      C v[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int sc = c0 + NT * i;
        v[i] = czero<Tc>();
        if (sc < npc) {
          const int J = row_of(sc, rmc);
          const int I = sc - J * mc;
          const int f1 = 2 * I + 1, f2 = 2 * J + 1;
          const int fs = f2 * m + f1;
          const C ctr = red_residual<Tc>(a, w, np, m, fs, f1, f2);
          C cor = red_residual<Tc>(a, w, np, m, fs - m - 1, f1 - 1, f2 - 1);
          cor = cor + red_residual<Tc>(a, w, np, m, fs - m + 1, f1 + 1, f2 - 1);
          cor = cor + red_residual<Tc>(a, w, np, m, fs + m - 1, f1 - 1, f2 + 1);
          cor = cor + red_residual<Tc>(a, w, np, m, fs + m + 1, f1 + 1, f2 + 1);
          v[i].x = fma(Tc(0.25), ctr.x, Tc(0.0625) * cor.x);
          v[i].y = fma(Tc(0.25), ctr.y, Tc(0.0625) * cor.y);
        }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int sc = c0 + NT * i;
        if (sc < npc) ac[sc] = v[i];
      }
    }
    __syncthreads();
  }
  __syncthreads();
  // ---- up: a_l += P a_{l+1}; odd fine index f sits on coarse (f - 1) / 2, even f
  // halfway between f/2 - 1 and f/2 (a parent outside the level is the zero boundary)
  for (int l = nl - 2; l >= 0; --l) {
    const int m = lv.m[l], mc = lv.m[l + 1];
    const int np = (int)lv.np[l];
    const float rm = 1.0f / (float)m;
    C* a = A[l];
    const C* ac = A[l + 1];
    for (int s0 = tid; s0 < np; s0 += NT * K) {
      C v[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int s = s0 + NT * i;
        v[i] = czero<Tc>();
        if (s < np) {
          const int i2 = row_of(s, rm);
          const int i1 = s - i2 * m;
          int c1[2], c2[2];
          Tc w1[2], w2[2];
          if (i1 & 1) {
            c1[0] = c1[1] = (i1 - 1) >> 1;
            w1[0] = Tc(1);
            w1[1] = Tc(0);
          } else {
            c1[0] = (i1 >> 1) - 1;
            c1[1] = i1 >> 1;
            w1[0] = c1[0] >= 0 ? Tc(0.5) : Tc(0);
            w1[1] = c1[1] < mc ? Tc(0.5) : Tc(0);
            c1[0] = max(c1[0], 0);
            c1[1] = min(c1[1], mc - 1);
          }
          if (i2 & 1) {
            c2[0] = c2[1] = (i2 - 1) >> 1;
            w2[0] = Tc(1);
            w2[1] = Tc(0);
          } else {
            c2[0] = (i2 >> 1) - 1;
            c2[1] = i2 >> 1;
            w2[0] = c2[0] >= 0 ? Tc(0.5) : Tc(0);
            w2[1] = c2[1] < mc ? Tc(0.5) : Tc(0);
            c2[0] = max(c2[0], 0);
            c2[1] = min(c2[1], mc - 1);
          }
          v[i] = a[s];
#pragma unroll
          for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const Tc wt = w2[b] * w1[q];
              if (wt != Tc(0)) tail_fma(v[i], wt, ac[c2[b] * mc + c1[q]]);
            }
        }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int s = s0 + NT * i;
        if (s < np) a[s] = v[i];
      }
    }
    __syncthreads();
  }
  C* dst = u0 + (int64_t)p * np0;
#pragma unroll 4
  for (int s = tid; s < np0; s += NT) dst[s] = A[0][s];
}

template <typename Tc>
size_t tail_arrays_smem(const CoarseLevels<Tc>& lv) {
  size_t b = 0;
  for (int l = 0; l < lv.count; ++l) b += (((size_t)lv.np[l] * sizeof(typename Cx<Tc>::t) + 15) / 16) * 16;
  return b;
}

template <typename Tc>
size_t tail_coef_smem(const CoarseLevels<Tc>& lv, int from) {
  size_t b = 0;
  for (int l = from; l < lv.count; ++l) b += ((5 * (size_t)lv.np[l] * sizeof(Tc) + 15) / 16) * 16;
  return b;
}

}  // namespace

// levels it takes: 2D, odd m halving down to one point, first level at most 63^2
bool mg_tail2_supported(const CoarseLevels<float>& lv) {
  if (lv.count < 1 || lv.count > kMaxCoarseLevels || lv.m[0] > kMgTailMaxM) return false;
  for (int l = 0; l < lv.count; ++l) {
    if (lv.m[l] < 1 || (lv.m[l] & 1) == 0 || lv.np[l] != (int64_t)lv.m[l] * lv.m[l]) return false;
    if (l + 1 < lv.count && lv.m[l + 1] != (lv.m[l] - 1) / 2) return false;
  }
  return lv.m[lv.count - 1] == 1;
}

cudaError_t launch_mg_tail2(Launch& L, int planes, const CoarseLevels<float>& lv, const float2* sigma, const float2* r0,
                            float2* u0) {
  typedef float Tc;
  if (!mg_tail2_supported(lv) || planes < 1) return cudaErrorInvalidValue;
  // stage the first level's coefficients too when two CTAs still fit on an SM
  const size_t base = tail_arrays_smem<Tc>(lv) + tail_coef_smem<Tc>(lv, 1);
  const size_t all = base + tail_coef_smem<Tc>(lv, 0) - tail_coef_smem<Tc>(lv, 1);
  const int stage0 = all <= 100 * 1024 ? 1 : 0;
  const size_t smem = stage0 ? all : base;
  cudaError_t e = cudaFuncSetAttribute(mg_tail2_kernel<Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  double pts = 0;
  for (int l = 0; l < lv.count; ++l) pts += (double)lv.np[l];
  const double cs = sizeof(float2);
  L.begin(KC_MG_COARSE);
  mg_tail2_kernel<Tc><<<planes, tail_threads<Tc>(), smem, L.stream>>>(lv, r0, u0, sigma, stage0);
  return L.end(KC_MG_COARSE, (double)planes * lv.np[0] * 2.0 * cs, (double)planes * pts * 60.0);
}

}  // namespace pcopt
