// Fast sine transform (DST-I) along one axis of the spectral planes: the exact
// spatial solves of the constant-coefficient case (step 2 of the four-step
// apply, Section 2.1), O(m log m) per grid line instead of the dense O(m^2)
// product with the DST matrix.
//
// With N = m + 1 a power of two, the orthonormal DST-I of a line x_1..x_m,
//   X_k = sqrt(2/N) sum_j x_j sin(pi j k / N),
// is its own inverse.  Two ways to get it from an FFT:
//  * half length (N >= 8, used in practice): with x_0 = x_N = 0 form
//      y_j = sin(pi j / N) (x_j + x_{N-j}) + (x_j - x_{N-j}) / 2,  j = 0..N-1,
//    and its N-point FFT Y.  Splitting y into the part symmetric under j -> N-j
//    and the antisymmetric part gives, for real x, X_{2q} = -Im Y_q and
//    X_{2q+1} - X_{2q-1} = Re Y_q; written with Y_{N-q} instead of conjugates,
//      X_{2q} = (i/2) (Y_q - Y_{N-q}),   X_{2q+1} = Y_0 / 2 + sum_{p=1..q} (Y_p + Y_{N-p}) / 2,
//    which is linear in x and so holds for complex lines too.  The odd outputs
//    are a prefix sum, taken in chunks per thread plus one pass over the chunk
//    totals (error growth ~ (chunk + threads per line) u, not N u);
//  * odd extension (N < 8): the length-L = 2N FFT of y (y_0 = y_N = 0, y_j = x_j,
//    y_{L-j} = -x_j) is Y_k = -2i sum_j x_j sin(pi j k / N), so
//    X_k = sqrt(2/N) (i/2) Y_k: twice the FFT length of the first way.
//
// One CTA of 256 threads owns COLS = 256/N1 grid lines along the axis:
//  * the tile (m values of each line) is copied into shared memory with the
//    line index fastest, so a warp reads whole 32-byte sectors for every axis
//    (along x1 four consecutive values of each of eight lines, along x2/x3
//    consecutive lines) and the shared-memory accesses are conflict-free;
//  * the FFT (N or L points) is the four-step split N1 N2 of the time FFT: an
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

// The half-length DST-I (file header) of every line of the tile in `src` into `sm`,
// N = N1 N2 = m + 1 >= 8, with the twiddle table of length 2N: the N-point FFT uses
// tw[2q] and sin(pi j / N) = -Im tw[j].  `scale` = sqrt(2/N).  Same contract as
// dst_tile: ends with a barrier; after_read() runs behind two barriers after every
// read of `src`, when no transform values are held in registers.
template <typename Tc, int N1, int N2, typename AfterRead>
__device__ __forceinline__ void dsth_tile(typename Cx<Tc>::t* sm, const typename Cx<Tc>::t* src,
                                          const typename Cx<Tc>::t* __restrict__ tw, int m, Tc scale, int r, int c,
                                          AfterRead&& after_read) {
  typedef typename Cx<Tc>::t C;
  constexpr int N = N1 * N2;
  constexpr int COLS = 256 / N1;
  constexpr int Q = N / 2 / N1;  // odd outputs per thread row
  static_assert(Q >= 1, "N must be at least 2 N1");
  __shared__ C tot[N1 * COLS];  // chunk totals of the prefix sum
  // (A) rows j = r + N1 j2 of y, N2-point DFT over j2
  C x[N2];
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    const int j = r + N1 * j2;
    const C a = (j >= 1) ? src[(j - 1) * COLS + c] : czero<Tc>();       // x_j (j <= N - 1 = m)
    const C b = (j >= 1) ? src[(N - j - 1) * COLS + c] : czero<Tc>();   // x_{N-j}; x_N = 0 when j = 0
    const Tc sj = -tw[j].y;
    const Tc h = Tc(0.5);
    x[j2] = cmk<Tc>(sj * (a.x + b.x) + h * (a.x - b.x), sj * (a.y + b.y) + h * (a.y - b.y));
  }
  __syncthreads();  // every read of the tile is done before the exchange overwrites it
  reg_fft<N2, false>(x, tw, 2 * N1);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const C y = (k2 == 0 || r == 0) ? x[k2] : cmul(tw[2 * r * k2], x[k2]);
    sm[xidx<N1, COLS>(k2, r, c)] = y;
  }
  __syncthreads();
  after_read();  // here no transform values are held in registers
  // (C) row k2 = r (< N2): N1-point DFT over j1 -> Y[k2 + N2 k1], stored as [k][c]
  {
    C y[N1];
    if (r < N2) {
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) y[j1] = sm[xidx<N1, COLS>(r, j1, c)];
    }
    __syncthreads();
    if (r < N2) {
      reg_fft<N1, false>(y, tw, 2 * N2);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) sm[(r + N2 * k1) * COLS + c] = y[k1];
    }
  }
  __syncthreads();
  // outputs: thread row r owns q = r Q .. r Q + Q - 1 (odd outputs 2q + 1, even 2q)
  C ev[Q], od[Q];
  C run = czero<Tc>();
  const Tc hs = Tc(0.5) * scale;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int q = r * Q + i;
    const C yq = sm[q * COLS + c];
    const C ym = sm[((N - q) & (N - 1)) * COLS + c];
    ev[i] = cmk<Tc>(-(yq.y - ym.y) * hs, (yq.x - ym.x) * hs);  // (i/2)(Y_q - Y_{N-q}) scale
    const Tc w = q == 0 ? Tc(0.25) * scale : hs;
    run = cmk<Tc>(run.x + (yq.x + ym.x) * w, run.y + (yq.y + ym.y) * w);
    od[i] = run;
  }
  tot[r * COLS + c] = run;
  __syncthreads();  // every Y read and every chunk total are in
  C off = czero<Tc>();
  for (int rr = 0; rr < r; ++rr) off = off + tot[rr * COLS + c];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int q = r * Q + i;
    sm[(2 * q) * COLS + c] = off + od[i];                // X_{2q+1} at index 2q
    if (q >= 1) sm[(2 * q - 1) * COLS + c] = ev[i];      // X_{2q} at index 2q - 1
  }
  __syncthreads();
}

// DIVIDE: forward DST, sm *= rmass / (sigma_p + lamK), inverse DST (the last axis).
// in may equal out: a CTA reads its whole tile before it writes it back.
// Lines: plane p = line / (np / m); inside the plane, a line along `axis` starts at
// outer * m * lstride + inner with lstride = m^axis, inner < lstride.
// one line-tile DST of the kind HALF selects (dsth_tile or dst_tile)
template <typename Tc, int N1, int N2, bool HALF, typename AfterRead>
__device__ __forceinline__ void dst_any(typename Cx<Tc>::t* sm, const typename Cx<Tc>::t* src,
                                        const typename Cx<Tc>::t* __restrict__ tw, int m, Tc scale, int r, int c,
                                        AfterRead&& after_read) {
  if constexpr (HALF)
    dsth_tile<Tc, N1, N2>(sm, src, tw, m, scale, r, c, after_read);
  else
    dst_tile<Tc, N1, N2>(sm, src, tw, m, scale, r, c, after_read);
}

// CTAs per SM the kernels are compiled for (registers per thread = 65536 / (256 x it))
template <typename Tc, int NP, bool STREAM>
constexpr int fst_min_blocks() {
  if constexpr (sizeof(Tc) == 4) return NP <= 256 ? (STREAM ? 3 : 4) : 2;
  return (NP <= 256 && !STREAM) ? 2 : 1;
}

template <typename Tc, int N1, int N2, bool DIVIDE, bool HALF>
__global__ void __launch_bounds__(256, fst_min_blocks<Tc, N1 * N2, false>()) fst4_kernel(const typename Cx<Tc>::t* in, typename Cx<Tc>::t* out,
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
  dst_any<Tc, N1, N2, HALF>(sm, sm, tw, m, half_scale, r, c, [] {});
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
    dst_any<Tc, N1, N2, HALF>(sm, sm, tw, m, half_scale, r, c, [] {});
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
template <typename Tc, int N1, int N2, bool DIVIDE, bool HALF>
__global__ void __launch_bounds__(256, fst_min_blocks<Tc, N1 * N2, true>()) fst4s_kernel(const typename Cx<Tc>::t* in, typename Cx<Tc>::t* out,
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
    dst_any<Tc, N1, N2, HALF>(sm, stage, tw, m, half_scale, r, c, [&] {
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
      dst_any<Tc, N1, N2, HALF>(sm, sm, tw, m, half_scale, r, c, [] {});
    }
    for (int e = tid; e < tot; e += 256) {
      const int j = e / COLS, cc = e - j * COLS;
      if (lplane[slot][cc] >= 0) out[lbase[slot][cc] + (int64_t)j * lstride] = sm[e];
    }
  }
  cp_async_wait<0>();
}

template <typename Tc, int N1, int N2, bool DIVIDE, bool HALF>
cudaError_t fst4s(Launch& L, const Grid& g, int64_t lstride, int64_t nlines, Tc hs, const typename Cx<Tc>::t* tw,
                  const Tc* lamK, const Tc* rmass, const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* in,
                  typename Cx<Tc>::t* out) {
  constexpr int COLS = 256 / N1;
  const size_t smem = ((size_t)(N1 + 1) * N2 * COLS + (size_t)g.m * COLS) * sizeof(typename Cx<Tc>::t);
  auto kern = fst4s_kernel<Tc, N1, N2, DIVIDE, HALF>;
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

// HALF: N1 N2 = m + 1 (half-length DST); otherwise N1 N2 = 2(m + 1) (odd extension)
template <typename Tc, int N1, int N2, bool HALF>
cudaError_t fst4(Launch& L, const Grid& g, int planes, int axis, bool divide, const typename Cx<Tc>::t* tw,
                 const Tc* lamK, const Tc* rmass, const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* in,
                 typename Cx<Tc>::t* out, bool stream) {
  constexpr int COLS = 256 / N1;
  const size_t smem = (size_t)(N1 + 1) * N2 * COLS * sizeof(typename Cx<Tc>::t);
  int64_t lstride = 1;
  for (int a = 0; a < axis; ++a) lstride *= g.m;
  const int64_t nlines = (int64_t)planes * (g.np / g.m);
  const unsigned blocks = (unsigned)((nlines + COLS - 1) / COLS);
  const double s2n = std::sqrt(2.0 / (g.m + 1));
  const Tc hs = (Tc)(HALF ? s2n : 0.5 * s2n);
  if constexpr (sizeof(Tc) == 4 || N1 * N2 <= 256) {  // FP64 at 512 points has no registers to spare
    if (stream)
      return divide ? fst4s<Tc, N1, N2, true, HALF>(L, g, lstride, nlines, hs, tw, lamK, rmass, sigma, in, out)
                    : fst4s<Tc, N1, N2, false, HALF>(L, g, lstride, nlines, hs, tw, nullptr, nullptr, nullptr, in,
                                                     out);
  }
  cudaError_t e;
  if (divide) {
    auto kern = fst4_kernel<Tc, N1, N2, true, HALF>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, 256, smem, L.stream>>>(in, out, tw, g.m, g.np, lstride, nlines, hs, lamK, rmass, sigma);
  } else {
    auto kern = fst4_kernel<Tc, N1, N2, false, HALF>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, 256, smem, L.stream>>>(in, out, tw, g.m, g.np, lstride, nlines, hs, nullptr, nullptr, nullptr);
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
  const int N = g.m + 1;
  // half-length transforms (N points) from N = 8 on, the odd extension (2N points) below
  const int Lfft_used = N >= 8 ? N : Lfft;
  const double lg = std::log2((double)Lfft_used);
  // per line: (divide ? 2 : 1) complex FFTs of the length used
  const double flops = (divide ? 2.0 : 1.0) * (tot / g.m) * 5.0 * Lfft_used * lg;
  L.begin(kc);
  cudaError_t e;
  switch (N) {
#define PCOPT_FST_CASE(NN, A, B, HALF) \
  case NN: e = fst4<Tc, A, B, HALF>(L, g, planes, axis, divide, tw, lamK, rmass, sigma, in, out, stream); break;
    PCOPT_FST_CASE(2, 2, 2, false)    // odd extension, 4 points
    PCOPT_FST_CASE(4, 4, 2, false)    // odd extension, 8 points
    PCOPT_FST_CASE(8, 4, 2, true)
    PCOPT_FST_CASE(16, 4, 4, true)
    PCOPT_FST_CASE(32, 8, 4, true)
    PCOPT_FST_CASE(64, 8, 8, true)
    PCOPT_FST_CASE(128, 16, 8, true)
    PCOPT_FST_CASE(256, 16, 16, true)
#undef PCOPT_FST_CASE
    case 512:
      if constexpr (sizeof(Tc) == 4) {
        e = fst4<Tc, 32, 16, true>(L, g, planes, axis, divide, tw, lamK, rmass, sigma, in, out, stream);
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
