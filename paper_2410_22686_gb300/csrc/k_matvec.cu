// All-at-once matrix-vector product y = A x (Eq. matrix_A, Section 2.1):
//
//   y1_j = alpha x1_j + (T^T x2)_j,   (T^T v)_j = v_j - v_{j+1} + tau K v_j,
//   y2_j = -(T x1)_j + alpha x2_j,     (T v)_j  = v_j - v_{j-1} + tau K v_j,
//
// and the transpose A^T = [[alpha I, -T^T], [T, alpha I]].
//
// One thread owns one spatial point and marches over a chunk of time blocks:
// its 2*dim face weights and the diagonal of tau K are loaded once, the time
// neighbour x1_{j-1} / x2_{j+1} is carried in registers, and the spatial
// neighbours come through L1/L2 (the rows above/below belong to blocks that
// run concurrently on the same time chunk).  DRAM traffic is the minimum:
// read x once, write y once.
#include "common.cuh"

namespace pcopt {

namespace {

template <typename Tin, int DIM, bool TRANSPOSE>
__global__ void __launch_bounds__(256) matvec_kernel(const Tin* __restrict__ x, double* __restrict__ y,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ diag, int m, int64_t ms,
                                                     int n, int tj, double alpha, size_t xstride, size_t ystride,
                                                     const int* __restrict__ jdev) {
  if (jdev) {  // device-resident Arnoldi index: x = Z_j, y = V_{j+1}
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ms) return;
  const int j0 = blockIdx.y * tj;
  const int j1 = min(n, j0 + tj);
  if (j0 >= n) return;

  const int i1 = (int)(s % m);
  const int64_t r = s / m;
  const int i2 = (int)(DIM == 2 ? r : r % m);
  const int i3 = (int)(DIM == 3 ? r / m : 0);

  // neighbour offsets (0 when the neighbour is a boundary node -> value 0)
  int64_t off[2 * DIM];
  bool ex[2 * DIM];
  double wv[2 * DIM];
  const int64_t mm = (int64_t)m * m;
  off[0] = -1;
  ex[0] = i1 > 0;
  off[1] = 1;
  ex[1] = i1 < m - 1;
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
  for (int k = 0; k < 2 * DIM; ++k) wv[k] = w[(int64_t)k * ms + s];
  const double dg = diag[s];

  const Tin* x1 = x;
  const Tin* x2 = x + (int64_t)n * ms;
  double* y1 = y;
  double* y2 = y + (int64_t)n * ms;

  auto tauK = [&](const Tin* base, double centre) -> double {
    double acc = dg * centre;
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k) {
      double nb = ex[k] ? cvt<double>(__ldg(base + off[k])) : 0.0;
      acc = fma(-wv[k], nb, acc);
    }
    return acc;
  };

  double x1prev = (j0 > 0) ? cvt<double>(x1[(int64_t)(j0 - 1) * ms + s]) : 0.0;
  double x2c = cvt<double>(x2[(int64_t)j0 * ms + s]);
#pragma unroll 2
  for (int j = j0; j < j1; ++j) {
    const int64_t idx = (int64_t)j * ms + s;
    const double x1c = cvt<double>(x1[idx]);
    const double x2n = (j + 1 < n) ? cvt<double>(x2[idx + ms]) : 0.0;
    const double k1 = tauK(x1 + idx, x1c);
    const double k2 = tauK(x2 + idx, x2c);
    const double tT_x2 = x2c - x2n + k2;     // (T^T x2)_j
    const double t_x1 = x1c - x1prev + k1;   // (T x1)_j
    if (!TRANSPOSE) {
      y1[idx] = fma(alpha, x1c, tT_x2);
      y2[idx] = fma(alpha, x2c, -t_x1);
    } else {
      y1[idx] = fma(alpha, x1c, -tT_x2);
      y2[idx] = fma(alpha, x2c, t_x1);
    }
    x1prev = x1c;
    x2c = x2n;
  }
}

}  // namespace

// time blocks per thread: the tuned value, else 32 (a thread carries its time
// neighbour in registers, so longer chunks re-read fewer x values)
static int time_chunk(const Launch& L, int n) {
  int tj = L.tiles && L.tiles->mv_tj > 0 ? L.tiles->mv_tj : 32;
  return tj < n ? tj : n;
}

template <typename Tin>
cudaError_t launch_matvec(Launch& L, const Grid& g, int n, const Stencil<double>& st, double alpha,
                          const Tin* x, double* y, bool transpose, size_t xstride, size_t ystride,
                          const int* jdev) {
  const int threads = 256;
  const int tj = time_chunk(L, n);
  dim3 grid((unsigned)((g.np + threads - 1) / threads), (unsigned)((n + tj - 1) / tj));
  const double U = 2.0 * (double)n * (double)g.np;
  const double bytes = U * (sizeof(Tin) + sizeof(double)) + (2.0 * g.dim + 1) * g.np * 8.0;
  const double flops = U * (4.0 * g.dim + 5.0);
  L.begin(KC_MATVEC);
  if (g.dim == 2) {
    if (transpose)
      matvec_kernel<Tin, 2, true><<<grid, threads, 0, L.stream>>>(x, y, st.w, st.diag, g.m, g.np, n, tj, alpha, xstride, ystride, jdev);
    else
      matvec_kernel<Tin, 2, false><<<grid, threads, 0, L.stream>>>(x, y, st.w, st.diag, g.m, g.np, n, tj, alpha, xstride, ystride, jdev);
  } else {
    if (transpose)
      matvec_kernel<Tin, 3, true><<<grid, threads, 0, L.stream>>>(x, y, st.w, st.diag, g.m, g.np, n, tj, alpha, xstride, ystride, jdev);
    else
      matvec_kernel<Tin, 3, false><<<grid, threads, 0, L.stream>>>(x, y, st.w, st.diag, g.m, g.np, n, tj, alpha, xstride, ystride, jdev);
  }
  return L.end(KC_MATVEC, bytes, flops);
}

template cudaError_t launch_matvec<double>(Launch&, const Grid&, int, const Stencil<double>&, double,
                                           const double*, double*, bool, size_t, size_t, const int*);
template cudaError_t launch_matvec<float>(Launch&, const Grid&, int, const Stencil<double>&, double,
                                          const float*, double*, bool, size_t, size_t, const int*);

}  // namespace pcopt

// ---------------------------------------------------------------------------
// The same product for an FP32 input z (the flexible-GMRES basis Z), evaluated in
// double-float arithmetic on the FP32 units: every FP64 coefficient c is held as
// c_hi + c_lo (two floats), c*z is formed exactly up to c_lo*z by an FMA error
// term (p = c_hi z, e = fma(c_hi, z, -p)), the leading parts are added by a
// pairwise tree of Knuth's TwoSum (depth log2 of the term count, so the chains stay
// short), and only the final hi + lo becomes an FP64 value (one FP64 addition).
// The relative error is of order 2^-46 of the largest term, far below what the
// Arnoldi relation needs, while GB300's FP64 unit (1/57 of the FP32 rate) would
// otherwise bound this kernel.
namespace pcopt {
namespace {

// a + b exactly as hi + err (Knuth).  The _rn intrinsics keep every operation a
// separately rounded IEEE operation: with FMA contraction the compiler could fuse a
// rounded product feeding `a + b` into an FMA, which breaks the exactness.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int DIM>
__global__ void __launch_bounds__(256) matvec_df_kernel(const float* __restrict__ x, double* __restrict__ y,
                                                        const float2* __restrict__ w, const float2* __restrict__ dg,
                                                        float2 alpha, int m, int64_t ms, int n, int tj,
                                                        size_t xstride, size_t ystride, const int* __restrict__ jdev) {
  if (jdev) {
    x += (size_t)(*jdev) * xstride;
    y += (size_t)(*jdev + 1) * ystride;
  }
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ms) return;
  const int j0 = blockIdx.y * tj;
  const int j1 = min(n, j0 + tj);
  if (j0 >= n) return;
  const int i1 = (int)(s % m);
  const int64_t r = s / m;
  const int i2 = (int)(DIM == 2 ? r : r % m);
  const int i3 = (int)(DIM == 3 ? r / m : 0);
  int64_t off[2 * DIM];
  bool ex[2 * DIM];
  float2 wv[2 * DIM];
  const int64_t mm = (int64_t)m * m;
  off[0] = -1;
  ex[0] = i1 > 0;
  off[1] = 1;
  ex[1] = i1 < m - 1;
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
  for (int k = 0; k < 2 * DIM; ++k) {
    if (!PC_DOK(!ex[k] || (s + off[k] >= 0 && s + off[k] < ms), 101)) return;  // neighbour inside the grid
    const float2 c = w[(int64_t)k * ms + s];
    wv[k] = make_float2(-c.x, -c.y);  // off-diagonal entries of tau K are -w
  }
  if (!PC_DOK(j1 <= n && j0 >= 0, 102)) return;
  const float2 d = dg[s];
  const float* x1 = x;
  const float* x2 = x + (int64_t)n * ms;
  double* y1 = y;
  double* y2 = y + (int64_t)n * ms;
  float x1prev = (j0 > 0) ? x1[(int64_t)(j0 - 1) * ms + s] : 0.0f;
  float x2c = x2[(int64_t)j0 * ms + s];
  constexpr int NT = 2 * DIM + 4;  // terms per output
#pragma unroll 2
  for (int j = j0; j < j1; ++j) {
    const int64_t idx = (int64_t)j * ms + s;
    const float x1c = x1[idx];
    const float x2n = (j + 1 < n) ? x2[idx + ms] : 0.0f;
    // y1 = alpha x1 + x2_j - x2_{j+1} + tau K x2_j ; y2 = alpha x2 - (x1_j - x1_{j-1} + tau K x1_j).
    // Leading parts of all terms are summed by a pairwise TwoSum tree; every rounding
    // error (products and sums) is gathered in a separate float.
    float ta[NT], tb[NT];
    float ea = 0.0f, eb = 0.0f;
    auto prod = [&](float2 c, float x, float& t, float& e) {
      t = __fmul_rn(c.x, x);  // rounded product, never fused downstream
      e += fmaf(c.x, x, -t) + c.y * x;
    };
    prod(d, x2c, ta[0], ea);
    prod(make_float2(-d.x, -d.y), x1c, tb[0], eb);
#pragma unroll
    for (int k = 0; k < 2 * DIM; ++k) {
      const float n2 = ex[k] ? __ldg(x2 + idx + off[k]) : 0.0f;
      const float n1 = ex[k] ? __ldg(x1 + idx + off[k]) : 0.0f;
      prod(wv[k], n2, ta[1 + k], ea);
      prod(make_float2(-wv[k].x, -wv[k].y), n1, tb[1 + k], eb);
    }
    ta[2 * DIM + 1] = x2c;
    ta[2 * DIM + 2] = -x2n;
    prod(alpha, x1c, ta[2 * DIM + 3], ea);
    tb[2 * DIM + 1] = -x1c;
    tb[2 * DIM + 2] = x1prev;
    prod(alpha, x2c, tb[2 * DIM + 3], eb);
#pragma unroll
    for (int step = 1; step < NT; step <<= 1) {
#pragma unroll
      for (int i = 0; i + step < NT; i += 2 * step) {
        float s1, r1, s2, r2;
        two_sum(ta[i], ta[i + step], s1, r1);
        two_sum(tb[i], tb[i + step], s2, r2);
        ta[i] = s1;
        ea += r1;
        tb[i] = s2;
        eb += r2;
      }
    }
    y1[idx] = f32_to_f64(ta[0]) + f32_to_f64(ea);
    y2[idx] = f32_to_f64(tb[0]) + f32_to_f64(eb);
    x1prev = x1c;
    x2c = x2n;
  }
}

}  // namespace

cudaError_t launch_matvec_df(Launch& L, const Grid& g, int n, const float2* w, const float2* diag, float2 alpha,
                             const float* x, double* y, size_t xstride, size_t ystride, const int* jdev) {
  const int threads = 256;
  const int tj = time_chunk(L, n);
  dim3 grid((unsigned)((g.np + threads - 1) / threads), (unsigned)((n + tj - 1) / tj));
  const double U = 2.0 * (double)n * (double)g.np;
  const double bytes = U * (sizeof(float) + sizeof(double)) + (2.0 * g.dim + 1) * g.np * 8.0;
  L.begin(KC_MATVEC);
  if (g.dim == 2)
    matvec_df_kernel<2><<<grid, threads, 0, L.stream>>>(x, y, w, diag, alpha, g.m, g.np, n, tj, xstride, ystride, jdev);
  else
    matvec_df_kernel<3><<<grid, threads, 0, L.stream>>>(x, y, w, diag, alpha, g.m, g.np, n, tj, xstride, ystride, jdev);
  return L.end(KC_MATVEC, jdev ? 0.0 : bytes, jdev ? 0.0 : U * (4.0 * g.dim + 5.0));
}

PCOPT_DEBUG_READER(pcopt_debug_matvec)

}  // namespace pcopt
