// Fast sine transform (DST-I) along one axis of the spectral planes: the exact
// spatial solves of the constant-coefficient case (step 2 of the four-step
// apply, Section 2.1), O(m log m) per grid line instead of the dense O(m^2)
// product with the DST matrix.
//
// With N = m + 1 a power of two, the orthonormal DST-I of a line x_1..x_m,
//   X_k = sqrt(2/N) sum_j x_j sin(pi j k / N),
// is read off the length-L = 2N FFT of the odd extension y (y_0 = y_N = 0,
// y_j = x_j, y_{L-j} = -x_j): Y_k = -2i sum_j x_j sin(pi j k / N), so
// X_k = sqrt(2/N) (i/2) Y_k.  The transform is its own inverse.
//
// One CTA of 256 threads owns COLS = 256/N1 grid lines along the axis:
//  * the tile (m values of each line) is copied into shared memory with the
//    line index fastest, so a warp reads whole 32-byte sectors for every axis
//    (along x1 four consecutive values of each of eight lines, along x2/x3
//    consecutive lines) and the shared-memory accesses are conflict-free;
//  * the L-point FFT is the four-step split L = N1 N2 of the time FFT: an
//    N2-point register FFT per thread row, a twiddle, one shared-memory
//    exchange, an N1-point register FFT;
//  * the results go back through shared memory and out with the same pattern.
// The last axis of a solve runs fused: forward transform, the spectral divide
// by (sigma_p M + tau K) eigenvalues, inverse transform, one read and one write.
#include <cmath>

#include "common.cuh"
#include "regfft.cuh"

namespace pcopt {

namespace {

// Exchange layout of the four-step FFT: row k2 (N1 entries of COLS lines) padded by
// COLS entries, so that the rows a warp reads in step (C) fall on different banks.
template <int N1, int COLS>
__device__ __forceinline__ int xidx(int k2, int j1, int c) {
  return (k2 * (N1 + 1) + j1) * COLS + c;
}

// One DST-I of every line of the tile in `src` ([j][c], j < m, line index c
// fastest); the result lands in `sm` with the same layout (src may be sm).  Ends
// with a barrier.  `sm` holds at least N2 (N1 + 1) COLS entries.  after_read() runs
// once every thread has read `src` (behind two barriers), between the first
// exchange and the second register FFT: the persistent kernel refills `src` with
// the next tile there.
template <typename Tc, int N1, int N2, typename AfterRead>
__device__ __forceinline__ void dst_tile(typename Cx<Tc>::t* sm, const typename Cx<Tc>::t* src,
                                         const typename Cx<Tc>::t* __restrict__ tw, int m, Tc half_scale, int r,
                                         int c, AfterRead&& after_read) {
  typedef typename Cx<Tc>::t C;
  constexpr int L = N1 * N2;
  constexpr int N = L / 2;
  constexpr int COLS = 256 / N1;
  // (A) rows j = r + N1 j2 of the odd extension, N2-point DFT over j2
  C x[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    const int j = r + N1 * j2;
    C v = czero<Tc>();
    if (j > 0 && j < N) {
      v = src[(j - 1) * COLS + c];
    } else if (j > N) {
      const C t = src[(L - j - 1) * COLS + c];
      v = cmk<Tc>(-t.x, -t.y);
    }
    x[j2] = v;
  }
  __syncthreads();  // every read of the tile is done before the exchange overwrites it
  reg_fft<N2, false>(x, tw, N1);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const C y = (k2 == 0 || r == 0) ? x[k2] : cmul(tw[r * k2], x[k2]);
    sm[xidx<N1, COLS>(k2, r, c)] = y;
  }
  __syncthreads();
  after_read();  // here no transform values are held in registers
  // (C) N1-point DFT over j1 for each k2, Y[k2 + N2 k1]; written as X_k = sqrt(2/N) (i/2) Y_k
  auto put = [&](int k, C y) {
    if (k >= 1 && k <= m) sm[(k - 1) * COLS + c] = cmk<Tc>(-y.y * half_scale, y.x * half_scale);
  };
  if constexpr (N1 == 2 * N2 && sizeof(Tc) == 4) {
    // every thread row works: row r < N2 transforms the even j1 of k2 = r, row r + N2 the
    // odd ones (N2-point DFTs), and the two halves meet in one radix-2 step.  (FP32 only:
    // it halves the registers for four CTAs per SM; the FP64 kernel is bound by its
    // arithmetic, where the extra exchange costs more than the occupancy gains.)
    constexpr int H = N1 / 2;
    const int k2 = r < N2 ? r : r - N2;
    const int b = r < N2 ? 0 : 1;
    C y[H];
#pragma unroll
    for (int a = 0; a < H; ++a) y[a] = sm[xidx<N1, COLS>(k2, 2 * a + b, c)];
    __syncthreads();
    reg_fft<H, false>(y, tw, 2 * N2);
#pragma unroll
    for (int q = 0; q < H; ++q) {
      C v = y[q];
      if (b == 1 && q != 0) v = cmul(tw[q * N2], v);  // w_{N1}^{q} = exp(-2 pi i q / N1)
      sm[xidx<N1, COLS>(k2, b * H + q, c)] = v;
    }
    __syncthreads();
    C e[H], o[H];
#pragma unroll
    for (int q = 0; q < H; ++q) {
      e[q] = sm[xidx<N1, COLS>(k2, q, c)];
      o[q] = sm[xidx<N1, COLS>(k2, H + q, c)];
    }
    __syncthreads();
    // row b = 0 writes k1 = q (even + odd), row b = 1 writes k1 = q + H (even - odd)
#pragma unroll
    for (int q = 0; q < H; ++q) put(k2 + N2 * (q + b * H), b == 0 ? e[q] + o[q] : e[q] - o[q]);
  } else {
    C y[N1];
    if (r < N2) {
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) y[j1] = sm[xidx<N1, COLS>(r, j1, c)];
    }
    __syncthreads();
    if (r < N2) {
      reg_fft<N1, false>(y, tw, N2);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) put(r + N2 * k1, y[k1]);
    }
  }
  __syncthreads();
}

// DIVIDE: forward DST, sm *= rmass / (sigma_p + lamK), inverse DST (the last axis).
// in may equal out: a CTA reads its whole tile before it writes it back.
// Lines: plane p = line / (np / m); inside the plane, a line along `axis` starts at
// outer * m * lstride + inner with lstride = m^axis, inner < lstride.
template <typename Tc, int N1, int N2, bool DIVIDE>
__global__ void __launch_bounds__(256, sizeof(Tc) == 4 ? (N1 * N2 <= 512 ? 4 : 2) : 1) fst4_kernel(const typename Cx<Tc>::t* in, typename Cx<Tc>::t* out,
                                                   const typename Cx<Tc>::t* __restrict__ tw, int m, int64_t np,
                                                   int64_t lstride, int64_t nlines, Tc half_scale,
                                                   const Tc* __restrict__ lamK, const Tc* __restrict__ rmass,
                                                   const typename Cx<Tc>::t* __restrict__ sigma) {
  typedef typename Cx<Tc>::t C;
  constexpr int COLS = 256 / N1;
  extern __shared__ __align__(16) unsigned char fst_smem[];
  C* sm = reinterpret_cast<C*>(fst_smem);
  __shared__ int64_t lbase[COLS];  // offset of each line's first value (plane included)
  __shared__ int lplane[COLS];
  const int tid = threadIdx.x;
  const int64_t line0 = (int64_t)blockIdx.x * COLS;
  if (tid < COLS) {
    const int64_t l = line0 + tid;
    const int64_t lpp = np / m;  // lines per plane
    int64_t b = 0;
    int p = 0;
    if (l < nlines) {
      p = (int)(l / lpp);
      b = l - (int64_t)p * lpp;
    }
    const int64_t outer = b / lstride, inner = b - outer * lstride;
    lbase[tid] = (int64_t)p * np + outer * lstride * m + inner;
    lplane[tid] = l < nlines ? p : -1;
  }
  __syncthreads();
  const int tot = COLS * m;
  for (int e = tid; e < tot; e += 256) {
    const int j = e / COLS, c = e - j * COLS;
    sm[e] = lplane[c] >= 0 ? in[lbase[c] + (int64_t)j * lstride] : czero<Tc>();
  }
  __syncthreads();
  const int r = tid / COLS, c = tid - (tid / COLS) * COLS;
  dst_tile<Tc, N1, N2>(sm, sm, tw, m, half_scale, r, c, [] {});
  if (DIVIDE) {
    for (int e = tid; e < tot; e += 256) {
      const int j = e / COLS, cc = e - j * COLS;
      const int p = lplane[cc];
      if (p < 0) continue;
      const int64_t s = lbase[cc] - (int64_t)p * np + (int64_t)j * lstride;  // spectral index in the plane
      C v = sm[e];
      if (rmass) v = cscale(v, rmass[s]);
      sm[e] = cmul(v, inv_diag<Tc>(sigma[p], lamK[s]));
    }
    __syncthreads();
    dst_tile<Tc, N1, N2>(sm, sm, tw, m, half_scale, r, c, [] {});
  }
  for (int e = tid; e < tot; e += 256) {
    const int j = e / COLS, cc = e - j * COLS;
    if (lplane[cc] >= 0) out[lbase[cc] + (int64_t)j * lstride] = sm[e];
  }
}

// Persistent streaming variant of fst4_kernel: each CTA walks tiles blockIdx.x,
// + gridDim.x, ...; the next tile is copied into the stage with cp.async as soon as
// the current one has been read into registers, so its load overlaps the transform,
// the spectral divide and the stores of the current tile.  Shared memory: the
// exchange area (N2 (N1 + 1) COLS entries) followed by the stage (m COLS entries).
// in may equal out: tiles are disjoint sets of lines, and a tile is read whole
// before any of it is written.
template <typename Tc, int N1, int N2, bool DIVIDE>
__global__ void __launch_bounds__(256, sizeof(Tc) == 4 ? (N1 * N2 <= 256 ? 4 : N1 * N2 <= 512 ? 3 : 2) : 1) fst4s_kernel(const typename Cx<Tc>::t* in, typename Cx<Tc>::t* out,
                                                   const typename Cx<Tc>::t* __restrict__ tw, int m, int64_t np,
                                                   int64_t lstride, int64_t nlines, int ntiles, Tc half_scale,
                                                   const Tc* __restrict__ lamK, const Tc* __restrict__ rmass,
                                                   const typename Cx<Tc>::t* __restrict__ sigma) {
  typedef typename Cx<Tc>::t C;
  constexpr int COLS = 256 / N1;
  extern __shared__ __align__(16) unsigned char fst_smem[];
  C* sm = reinterpret_cast<C*>(fst_smem);
  C* stage = sm + N2 * (N1 + 1) * COLS;
  __shared__ int64_t lbase[2][COLS];
  __shared__ int lplane[2][COLS];
  const int tid = threadIdx.x;
  const int tot = COLS * m;
  const int r = tid / COLS, c = tid - (tid / COLS) * COLS;
  auto bases = [&](int tile, int slot) {  // threads < COLS: where the tile's lines start
    if (tid < COLS) {
      const int64_t l = (int64_t)tile * COLS + tid;
      const int64_t lpp = np / m;
      int64_t b = 0;
      int p = 0;
      if (l < nlines) {
        p = (int)(l / lpp);
        b = l - (int64_t)p * lpp;
      }
      const int64_t outer = b / lstride, inner = b - outer * lstride;
      lbase[slot][tid] = (int64_t)p * np + outer * lstride * m + inner;
      lplane[slot][tid] = l < nlines ? p : -1;
    }
  };
  auto issue = [&](int slot) {  // the tile whose bases are in `slot` -> stage
    for (int e = tid; e < tot; e += 256) {
      const int j = e / COLS, cc = e - j * COLS;
      const bool ok = lplane[slot][cc] >= 0;
      cp_async<sizeof(C)>(stage + e, in + (ok ? lbase[slot][cc] + (int64_t)j * lstride : 0), ok);
    }
    cp_async_commit();
  };
  int tile = blockIdx.x, slot = 0;
  if (tile < ntiles) bases(tile, 0);
  __syncthreads();
  if (tile < ntiles) issue(0);
  for (; tile < ntiles; tile += gridDim.x, slot ^= 1) {
    const int next = tile + (int)gridDim.x;
    cp_async_wait<0>();
    __syncthreads();  // the stage holds this tile; the previous tile's stores are done
    if (next < ntiles) bases(next, slot ^ 1);
    dst_tile<Tc, N1, N2>(sm, stage, tw, m, half_scale, r, c, [&] {
      if (next < ntiles) issue(slot ^ 1);
    });
    if (DIVIDE) {
      for (int e = tid; e < tot; e += 256) {
        const int j = e / COLS, cc = e - j * COLS;
        const int p = lplane[slot][cc];
        if (p < 0) continue;
        const int64_t s = lbase[slot][cc] - (int64_t)p * np + (int64_t)j * lstride;
        C v = sm[e];
        if (rmass) v = cscale(v, rmass[s]);
        sm[e] = cmul(v, inv_diag<Tc>(sigma[p], lamK[s]));
      }
      __syncthreads();
      dst_tile<Tc, N1, N2>(sm, sm, tw, m, half_scale, r, c, [] {});
    }
    for (int e = tid; e < tot; e += 256) {
      const int j = e / COLS, cc = e - j * COLS;
      if (lplane[slot][cc] >= 0) out[lbase[slot][cc] + (int64_t)j * lstride] = sm[e];
    }
  }
  cp_async_wait<0>();
}

template <typename Tc, int N1, int N2, bool DIVIDE>
cudaError_t fst4s(Launch& L, const Grid& g, int64_t lstride, int64_t nlines, Tc hs, const typename Cx<Tc>::t* tw,
                  const Tc* lamK, const Tc* rmass, const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* in,
                  typename Cx<Tc>::t* out) {
  constexpr int COLS = 256 / N1;
  const size_t smem = ((size_t)(N1 + 1) * N2 * COLS + (size_t)g.m * COLS) * sizeof(typename Cx<Tc>::t);
  auto kern = fst4s_kernel<Tc, N1, N2, DIVIDE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem)) != cudaSuccess) return e;
  const int ntiles = (int)((nlines + COLS - 1) / COLS);
  const int sms = L.tiles && L.tiles->sms > 0 ? L.tiles->sms : 152;
  const int grid = std::min(ntiles, std::max(1, per_sm) * sms);
  kern<<<grid, 256, smem, L.stream>>>(in, out, tw, g.m, g.np, lstride, nlines, ntiles, hs, lamK, rmass, sigma);
  return cudaGetLastError();
}

template <typename Tc, int N1, int N2>
cudaError_t fst4(Launch& L, const Grid& g, int planes, int axis, bool divide, const typename Cx<Tc>::t* tw,
                 const Tc* lamK, const Tc* rmass, const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* in,
                 typename Cx<Tc>::t* out, bool stream) {
  constexpr int COLS = 256 / N1;
  const size_t smem = (size_t)(N1 + 1) * N2 * COLS * sizeof(typename Cx<Tc>::t);
  int64_t lstride = 1;
  for (int a = 0; a < axis; ++a) lstride *= g.m;
  const int64_t nlines = (int64_t)planes * (g.np / g.m);
  const unsigned blocks = (unsigned)((nlines + COLS - 1) / COLS);
  const Tc hs = (Tc)(0.5 * std::sqrt(2.0 / (g.m + 1)));
  if constexpr (sizeof(Tc) == 4 || N1 * N2 <= 256) {  // FP64 at L = 512 has no registers to spare
    if (stream)
      return divide ? fst4s<Tc, N1, N2, true>(L, g, lstride, nlines, hs, tw, lamK, rmass, sigma, in, out)
                    : fst4s<Tc, N1, N2, false>(L, g, lstride, nlines, hs, tw, nullptr, nullptr, nullptr, in, out);
  }
  cudaError_t e;
  if (divide) {
    e = cudaFuncSetAttribute(fst4_kernel<Tc, N1, N2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fst4_kernel<Tc, N1, N2, true><<<blocks, 256, smem, L.stream>>>(in, out, tw, g.m, g.np, lstride, nlines, hs, lamK,
                                                                   rmass, sigma);
  } else {
    e = cudaFuncSetAttribute(fst4_kernel<Tc, N1, N2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fst4_kernel<Tc, N1, N2, false><<<blocks, 256, smem, L.stream>>>(in, out, tw, g.m, g.np, lstride, nlines, hs,
                                                                    nullptr, nullptr, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace

template <typename Tc>
bool fst_fast_supported(int m) {
  const int L = 2 * (m + 1);
  return (L & (L - 1)) == 0 && L >= 4 && L <= (sizeof(Tc) == 4 ? 1024 : 512);
}

template <typename Tc>
cudaError_t launch_fst_fast(Launch& L, const Grid& g, int planes, int axis, bool divide,
                            const typename Cx<Tc>::t* tw, const Tc* lamK, const Tc* rmass,
                            const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* in,
                            typename Cx<Tc>::t* out) {
  const int Lfft = 2 * (g.m + 1);
  const double tot = (double)planes * (double)g.np;
  const double cs = sizeof(typename Cx<Tc>::t);
  const int kc = divide ? KC_FST_DIVIDE : KC_FST_AXIS;
  // fst_stream bit 0: the axis passes stream tiles, bit 1: the fused last-axis pass does
  const bool stream = L.tiles && (L.tiles->fst_stream & (divide ? 2 : 1));
  const double lg = std::log2((double)Lfft);
  // per line: (divide ? 2 : 1) complex FFTs of length 2(m+1)
  const double flops = (divide ? 2.0 : 1.0) * (tot / g.m) * 5.0 * Lfft * lg;
  L.begin(kc);
  cudaError_t e;
  switch (Lfft) {
#define PCOPT_FST_CASE(LL, A, B) \
  case LL: e = fst4<Tc, A, B>(L, g, planes, axis, divide, tw, lamK, rmass, sigma, in, out, stream); break;
    PCOPT_FST_CASE(4, 2, 2)
    PCOPT_FST_CASE(8, 4, 2)
    PCOPT_FST_CASE(16, 4, 4)
    PCOPT_FST_CASE(32, 8, 4)
    PCOPT_FST_CASE(64, 8, 8)
    PCOPT_FST_CASE(128, 16, 8)
    PCOPT_FST_CASE(256, 16, 16)
    PCOPT_FST_CASE(512, 32, 16)
#undef PCOPT_FST_CASE
    case 1024:
      if constexpr (sizeof(Tc) == 4) {
        e = fst4<Tc, 32, 32>(L, g, planes, axis, divide, tw, lamK, rmass, sigma, in, out, stream);
        break;
      } else {
        return cudaErrorNotSupported;
      }
    default:
      return cudaErrorNotSupported;
  }
  if (e != cudaSuccess) return e;
  return L.end(kc, 2.0 * tot * cs, flops);
}

template bool fst_fast_supported<float>(int);
template bool fst_fast_supported<double>(int);
template cudaError_t launch_fst_fast<float>(Launch&, const Grid&, int, int, bool, const float2*, const float*,
                                            const float*, const float2*, const float2*, float2*);
template cudaError_t launch_fst_fast<double>(Launch&, const Grid&, int, int, bool, const double2*, const double*,
                                             const double*, const double2*, const double2*, double2*);

}  // namespace pcopt
