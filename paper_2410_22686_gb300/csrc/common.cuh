// Internal declarations shared by the translation units of libpcopt.
// Nothing here is part of the public C ABI (include/pcopt.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace pcopt {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };

template <typename T>
__host__ __device__ __forceinline__ typename Cx<T>::t cmk(T re, T im) {
  typename Cx<T>::t r;
  r.x = re;
  r.y = im;
  return r;
}
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// 1/z = conj(z)/|z|^2
__host__ __device__ __forceinline__ float2 cinv(float2 z) {
  float q = 1.0f / (z.x * z.x + z.y * z.y);
  return make_float2(z.x * q, -z.y * q);
}
__host__ __device__ __forceinline__ double2 cinv(double2 z) {
  double q = 1.0 / (z.x * z.x + z.y * z.y);
  return make_double2(z.x * q, -z.y * q);
}
template <typename T>
__host__ __device__ __forceinline__ typename Cx<T>::t czero() { return cmk<T>(T(0), T(0)); }
// 1 / (sigma + d) for a complex shift sigma and a real diagonal d
template <typename Tc>
__device__ __forceinline__ typename Cx<Tc>::t inv_diag(typename Cx<Tc>::t sig, Tc dg) {
  return cinv(cmk<Tc>(sig.x + dg, sig.y));
}

// FP64 <-> FP32 conversions on the integer pipes.  GB300 executes F2F
// conversions on its FP64 unit, whose rate is 1/64 of FP32, which made plain
// casts the bottleneck of the FP32 kernels that read FP64 vectors.  Both follow
// the IEEE-754 binary64/binary32 layouts.  FP64 -> FP32 rounds half up on the
// magnitude (ties away from zero; differs from round-to-nearest-even only on
// exact ties), flushes results below the FP32 normal range to a signed zero and
// saturates larger magnitudes, infinities and NaNs to infinity: it feeds FP32
// preconditioner inputs only.  FP32 -> FP64 is exact; FP32 subnormals flush to
// zero, infinities and NaNs are kept.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned mag = hi & 0x7FFFFFFFu;  // exponent (11 bits) and top 20 mantissa bits
  // rebias 1023 -> 127, keep 23 mantissa bits, round half up on the magnitude (a carry
  // moves into the exponent); magnitudes below the FP32 normal range flush to zero,
  // above it (and infinities, NaNs) saturate to infinity
  unsigned f = ((mag - (896u << 20)) << 3) | (lo >> 29);
  f += (lo >> 28) & 1u;
  f = mag < (897u << 20) ? 0u : f;
  f = mag >= (1151u << 20) ? 0x7F800000u : f;
  return __uint_as_float(sign | f);
}
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned hi, lo;
  if (e == 0) {
    hi = sign;
    lo = 0u;
  } else if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
    lo = m << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}
// generic casts used by templated kernels
template <typename To, typename From>
__device__ __forceinline__ To cvt(From x) { return (To)x; }
template <>
__device__ __forceinline__ float cvt<float, double>(double x) { return f64_to_f32(x); }
template <>
__device__ __forceinline__ double cvt<double, float>(float x) { return f32_to_f64(x); }

// storage of complex multigrid iterates: the compute type itself, or a BF16 pair
// (FP32 arithmetic, BF16 storage) for the BF16-storage smoother variant
__device__ __forceinline__ float2 ldc(const float2* p, int64_t i) { return p[i]; }
__device__ __forceinline__ double2 ldc(const double2* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float2 ldc(const __nv_bfloat162* p, int64_t i) { return __bfloat1622float2(p[i]); }
__device__ __forceinline__ void stc(float2* p, int64_t i, float2 v) { p[i] = v; }
__device__ __forceinline__ void stc(double2* p, int64_t i, double2 v) { p[i] = v; }
__device__ __forceinline__ void stc(__nv_bfloat162* p, int64_t i, float2 v) { p[i] = __float22bfloat162_rn(v); }

// ---------------------------------------------------------------------------
// Debug build (-DPCOPT_DEBUG): explicit checks of index arithmetic that record the
// first failing check's code in a device word of the translation unit and let the
// caller skip the access, instead of trapping.  In the release build PC_DOK(c, code)
// is `true` and costs nothing.  Codes: 1xx matvec, 2xx Krylov, 3xx time FFT.
// ---------------------------------------------------------------------------
#ifdef PCOPT_DEBUG
static __device__ int pcopt_dbg_err = 0;
__device__ __forceinline__ bool pcopt_dok(bool ok, int code) {
  if (!ok) atomicCAS(&pcopt_dbg_err, 0, code);
  return ok;
}
#define PC_DOK(cond, code) (pcopt_dok((cond), (code)))
#define PCOPT_DEBUG_READER(fn)                                                    \
  int fn(int reset) {                                                             \
    int v = 0;                                                                    \
    if (cudaMemcpyFromSymbol(&v, pcopt_dbg_err, sizeof(int)) != cudaSuccess) v = -1; \
    if (reset) {                                                                  \
      const int z = 0;                                                            \
      cudaMemcpyToSymbol(pcopt_dbg_err, &z, sizeof(int));                         \
    }                                                                             \
    return v;                                                                     \
  }
#else
#define PC_DOK(cond, code) (true)
#define PCOPT_DEBUG_READER(fn) \
  int fn(int) { return 0; }
#endif
// per translation unit: the recorded code (0 none, -1 unreadable); reset clears it
int pcopt_debug_matvec(int reset);
int pcopt_debug_krylov(int reset);
int pcopt_debug_tfft(int reset);

// ---------------------------------------------------------------------------
// kernel classes (instrumentation buckets)
// ---------------------------------------------------------------------------
enum KernelClass {
  KC_MATVEC = 0,
  KC_TFFT_FWD,
  KC_TFFT_INV,
  KC_FST_AXIS,
  KC_FST_DIVIDE,
  KC_MG_SMOOTH,
  KC_MG_RESID_RESTRICT,
  KC_MG_PROLONG,
  KC_MG_COARSEST,
  KC_DOT,
  KC_UPDATE,
  KC_REDUCE,
  KC_SCALE,
  KC_GIVENS,
  KC_XUPDATE,
  KC_AXPBY,
  KC_RHS,
  KC_GRAD,
  KC_REORTH,  // gated re-orthogonalisation passes (bytes booked only when they ran)
  KC_MG_COARSE,
  KC_MG_DOWN,  // fused smooth + residual + restriction of one level
  KC_FE_APPLY, // finite-element mass / stiffness product of single fields
  KC_IDEAL_STEP,  // ideal RBD preconditioner: per-time-step right-hand sides and the final rotation
  KC_COUNT
};
const char* kernel_class_name(int kc);

// ---------------------------------------------------------------------------
// launch context: stream + launch counting + optional event timing
// ---------------------------------------------------------------------------
struct Prof {
  bool on = false;
  uint64_t mask = ~0ull;  // kernel classes timed while on (bit kc)
  int64_t launches[KC_COUNT] = {0};
  double bytes[KC_COUNT] = {0};
  double flops[KC_COUNT] = {0};
  double ms[KC_COUNT] = {0};
  struct Pending {
    int kc;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  int64_t total = 0;
  cudaError_t flush();  // resolve pending event pairs into ms[]
  void reset();
  ~Prof();
};

// Tile shapes of the tunable kernels, 0 = the built-in default.  Chosen per
// problem by pc_autotune (timed candidates) or set from a stored table.
struct Tiles {
  int mg_cx = 0;    // fused 2D down leg: coarse points per tile axis (8 or 16)
  int mg_ctas = 0;  // fused 2D down leg: CTAs per SM its grid is sized for (sets planes per CTA per level)
  int mv_tj = 0;    // matvec kernels: time blocks per thread
  int pro_pch = 0;  // prolongation and per-level (3D) multigrid kernels: planes per CTA
  int fft_stream = 0;  // time FFTs: 0 one CTA per column tile, 1 persistent CTAs streaming tiles (cp.async)
  int mg_march = 0;    // fused 2D down leg with FP32 iterates: 0 shared-memory tiles, 1 register-marching warps
  int mg_seg = 0;      // register-marching down leg: coarse rows per warp segment (default 16)
  int fst_stream = 0;  // sine transforms, persistent CTAs streaming tiles (cp.async) in: bit 0 the axis
                       // passes, bit 1 the fused last-axis pass; one CTA per line tile otherwise
  int sms = 0;      // SMs of the device (set at setup)
};

struct Launch {
  cudaStream_t stream;
  Prof* prof;
  const Tiles* tiles = nullptr;
  // record around one kernel launch; `bytes`/`flops` are algorithmic figures
  cudaEvent_t ev_a = nullptr;
  void begin(int kc);
  cudaError_t end(int kc, double bytes, double flops);
};

// ---------------------------------------------------------------------------
// device-side problem description used by the kernels
// ---------------------------------------------------------------------------
struct Grid {
  int dim;     // 2 or 3
  int m;       // points per dimension on this level
  int64_t np;  // m^dim
};

// stencil of one level: per-point face weights tau*a_f/h^2 towards
// (-x1, +x1, -x2, +x2[, -x3, +x3]) and their sum (the diagonal of tau K)
template <typename T>
struct Stencil {
  const T* w;     // [2*dim][np]
  const T* diag;  // [np]
};

// ---------------------------------------------------------------------------
// launchers (defined in the k_*.cu files)
// ---------------------------------------------------------------------------
// y = A x (transpose=false) or A^T x; x in Tin (double or float), y double.
// With jdev != nullptr: x += (*jdev) * xstride and y += (*jdev + 1) * ystride.
template <typename Tin>
cudaError_t launch_matvec(Launch& L, const Grid& g, int n, const Stencil<double>& st, double alpha,
                          const Tin* x, double* y, bool transpose, size_t xstride = 0, size_t ystride = 0,
                          const int* jdev = nullptr);

// y = A x for an FP32 x in double-float arithmetic (FP64 output): the inner matvec
// of flexible GMRES.  w/diag hold tau a_f / h^2 and its sum as (hi, lo) float pairs.
cudaError_t launch_matvec_df(Launch& L, const Grid& g, int n, const float2* w, const float2* diag, float2 alpha,
                             const float* x, double* y, size_t xstride = 0, size_t ystride = 0,
                             const int* jdev = nullptr);

// Finite elements in space (bilinear / trilinear, constant coefficient c): the
// mass and stiffness matrices are wM and wK times fixed integer stencils.
struct FeScale {
  double wM = 0.0;  // (h/6)^dim
  double wK = 0.0;  // c (h/6)^(dim-1) / h
};
FeScale fe_scale(int dim, int m1, double c);
// y = A x or A^T x with A = [[alpha I(x)M, T^T], [-T, alpha I(x)M]], T = B_n(x)M + tau I(x)K;
// x in Tin, FP64 arithmetic and output; strides / jdev as launch_matvec
template <typename Tin>
cudaError_t launch_matvec_fe(Launch& L, const Grid& g, int n, double alpha, FeScale fs, double tau, const Tin* x,
                             double* y, bool transpose, size_t xstride = 0, size_t ystride = 0,
                             const int* jdev = nullptr);
// out_p = cM (M/wM) in_p + cK (K/wK) in_p + beta out_p for `planes` fields of g.np values
cudaError_t launch_fe_apply(Launch& L, const Grid& g, int planes, double cM, double cK, const double* in, double beta,
                            double* out);

// 2D bilinear elements with a nodal coefficient (k_fevar.cu): E holds one value per
// element ((m+1)^2, the mean of its corner values), h2 = h^2 of the level
cudaError_t launch_fevar_apply(Launch& L, int m, int planes, double h2, const double* E, double cM, double cK,
                               const double* in, double beta, double* out);
// (strides / jdev as launch_matvec)
template <typename Tin>
cudaError_t launch_matvec_fevar(Launch& L, int m, int n, double h2, double alpha, double tau, const double* E,
                                const Tin* x, double* y, bool transpose, size_t xstride = 0, size_t ystride = 0,
                                const int* jdev = nullptr);
template <typename Tc>
cudaError_t launch_fevar_smooth(Launch& L, int m, int planes, Tc h2, Tc tau, const Tc* E,
                                const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, typename Cx<Tc>::t* u);
template <typename Tc>
cudaError_t launch_fevar_resid_restrict(Launch& L, int m, int planes, Tc h2, Tc tau, const Tc* E,
                                        const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r,
                                        const typename Cx<Tc>::t* u, typename Cx<Tc>::t* res,
                                        typename Cx<Tc>::t* rc);
cudaError_t launch_fevar_level_elements(Launch& L, const double* a_nodes, int M0, int stride, int m, double* e64,
                                        float* e32);
cudaError_t launch_fevar_grad(Launch& L, int m, int n, double tau, const double* a_int, const double* x,
                              const double* lam, double* part, int max_chunks, double* grad);
cudaError_t launch_fevar_objective(Launch& L, int m, int n, double h2, double tau, double gamma, const double* x,
                                   const double* g, double* partial, int max_partial, double* J);
cudaError_t launch_fevar_objective_grad(Launch& L, int m, int n, double h2, double tau, double gamma,
                                        const double* x, const double* g, const double* gJ, double* gx, double* gg);

// 3D trilinear elements with a nodal coefficient (k_fevar3.cu): E holds one value per
// element ((m+1)^3, the mean of its eight corner values), h = the level's mesh width
cudaError_t launch_fevar3_apply(Launch& L, int m, int planes, double h, const double* E, double cM, double cK,
                                const double* in, double beta, double* out);
template <typename Tin>
cudaError_t launch_matvec_fevar3(Launch& L, int m, int n, double h, double alpha, double tau, const double* E,
                                 const Tin* x, double* y, bool transpose, size_t xstride = 0, size_t ystride = 0,
                                 const int* jdev = nullptr);
template <typename Tc>
cudaError_t launch_fevar3_smooth(Launch& L, int m, int planes, Tc h, Tc tau, const Tc* E,
                                 const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, typename Cx<Tc>::t* u);
template <typename Tc>
cudaError_t launch_fevar3_resid_restrict(Launch& L, int m, int planes, Tc h, Tc tau, const Tc* E,
                                         const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r,
                                         const typename Cx<Tc>::t* u, typename Cx<Tc>::t* res,
                                         typename Cx<Tc>::t* rc);
cudaError_t launch_fevar3_level_elements(Launch& L, const double* a_nodes, int M0, int stride, int m, double* e64,
                                         float* e32);
cudaError_t launch_fevar3_grad(Launch& L, int m, int n, double h, double tau, const double* a_int, const double* x,
                               const double* lam, double* part, int max_chunks, double* grad);
cudaError_t launch_fevar3_objective(Launch& L, int m, int n, double h, double tau, double gamma, const double* x,
                                    const double* g, double* partial, int max_partial, double* J);
cudaError_t launch_fevar3_objective_grad(Launch& L, int m, int n, double h, double tau, double gamma,
                                         const double* x, const double* g, const double* gJ, double* gx,
                                         double* gg);

// forward scaled time FFT: v (FP64 [2][n][ms]) -> spectral planes [2*nfreq][ms]
// dpow[j] = eps^{j/n}, dinv[j] = eps^{-j/n}, tw[k] = exp(-2 pi i k/n) for k = 0..n-1
// With jdev != nullptr the input is v + (*jdev) * vstride (device-resident Arnoldi index).
// input v: FP64 basis vectors, or (Tc = float) their FP32 rounding
template <typename Tc, typename Tin = double>
cudaError_t launch_tfft_forward(Launch& L, int64_t ms, int n, const Tin* v, const Tc* dpow, const Tc* dinv,
                                const typename Cx<Tc>::t* tw, typename Cx<Tc>::t* spec, size_t vstride = 0,
                                const int* jdev = nullptr);
// inverse scaled time FFT + butterfly: spectral planes (stored as TU) -> w (Tout [2][n][ms])
// With jdev != nullptr the output is w + (*jdev) * wstride.
// Last step of the multigrid up leg, done while the inverse time transform loads
// the finest level: u_f + P e_c, P the (bi/tri)linear prolongation from the next
// coarser level (mc = (mf - 1) / 2 points per axis, zero outside).  ec == nullptr:
// the planes are used as they are.
template <typename TU>
struct FineCorrection {
  const TU* ec = nullptr;
  int dim = 0, mf = 0, mc = 0;
  int64_t npc = 0;
};

template <typename Tc, typename TU, typename Tout>
cudaError_t launch_tfft_inverse(Launch& L, int64_t ms, int n, const TU* spec, const Tc* dpow, const Tc* dinv,
                                const typename Cx<Tc>::t* tw, Tout* w, size_t wstride = 0,
                                const int* jdev = nullptr, FineCorrection<TU> fc = FineCorrection<TU>());

// FST: one DST-I along `axis` of every plane (out = S in), and the spectral divide
// buf *= rmass / (sigma + lamK) (rmass == nullptr: 1)
template <typename Tc>
cudaError_t launch_fst_axis(Launch& L, const Grid& g, int planes, int axis, const Tc* S,
                            const typename Cx<Tc>::t* in, typename Cx<Tc>::t* out);
template <typename Tc>
cudaError_t launch_fst_divide(Launch& L, const Grid& g, int planes, const Tc* lamK, const Tc* rmass,
                              const typename Cx<Tc>::t* sigma, typename Cx<Tc>::t* buf);
// Fast sine transforms (k_fst.cu) for m + 1 a power of two, 2(m+1) <= 1024 (FP32) /
// 512 (FP64): out = S in along `axis` (S the orthonormal DST-I), or with `divide`
// out = S diag(rmass / (sigma_p + lamK)) S in along the last axis.  tw: the
// 2(m+1)-point twiddle circle exp(-2 pi i q / (2(m+1))).  in may equal out.
template <typename Tc>
bool fst_fast_supported(int m);
template <typename Tc>
cudaError_t launch_fst_fast(Launch& L, const Grid& g, int planes, int axis, bool divide,
                            const typename Cx<Tc>::t* tw, const Tc* lamK, const Tc* rmass,
                            const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* in,
                            typename Cx<Tc>::t* out);

// multigrid pieces (planes = 2*nfreq, sigma per plane); iterates u stored as TU
template <typename Tc, typename TU>
cudaError_t launch_mg_smooth(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                             const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u);
// residual of the sweep's result and its full weighting onto the next level; rb_sweep:
// u is a red-black sweep from zero, whose residual follows from the sweep's identity
template <typename Tc, typename TU>
cudaError_t launch_mg_resid_restrict(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                                     const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, const TU* u,
                                     typename Cx<Tc>::t* res, typename Cx<Tc>::t* rc, bool rb_sweep = true);
// Gauss-Seidel sweep from zero in the natural order (one CTA per plane, diagonal by diagonal)
template <typename Tc, typename TU>
cudaError_t launch_mg_smooth_lex(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                                 const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u);
template <typename Tc, typename TU>
cudaError_t launch_mg_down(Launch& L, const Grid& g, int planes, const Stencil<Tc>& st,
                           const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r, TU* u,
                           typename Cx<Tc>::t* rc, int cx = 0, int pch = 0, const float4* w4 = nullptr);
int mg_down_default_cx(int tc_bytes);
int mg_down_default_pch(int m, int planes, int cx, int ctas_per_sm, int sms);
template <typename Tc, typename TU>
cudaError_t launch_mg_prolong(Launch& L, const Grid& gf, int planes, const TU* ec, TU* uf);
template <typename Tc, typename TU>
cudaError_t launch_mg_coarsest(Launch& L, int planes, const Tc* diag, const typename Cx<Tc>::t* sigma,
                               const typename Cx<Tc>::t* r, TU* u);

// Coarse part of the multigrid cycle run by one kernel (levels l0..last):
// sizes and per-level stencils, passed by value.
constexpr int kMaxCoarseLevels = 8;
template <typename T>
struct CoarseLevels {
  int count;
  int m[kMaxCoarseLevels];
  int64_t np[kMaxCoarseLevels];
  const T* w[kMaxCoarseLevels];
  const T* diag[kMaxCoarseLevels];
};
// 2D FP32 iterates: the lower part of the cycle from the first level with
// m <= kMgTailMaxM, one array per level updated in place (k_mgtail.cu)
constexpr int kMgTailMaxM = 63;
bool mg_tail2_supported(const CoarseLevels<float>& lv);
cudaError_t launch_mg_tail2(Launch& L, int planes, const CoarseLevels<float>& lv, const float2* sigma, const float2* r0,
                            float2* u0);
template <typename Tc, typename TU>
size_t mg_coarse_cycle_smem(const CoarseLevels<Tc>& lv);
template <typename Tc, typename TU>
cudaError_t launch_mg_coarse_cycle(Launch& L, int dim, int planes, const CoarseLevels<Tc>& lv,
                                   const typename Cx<Tc>::t* sigma, const typename Cx<Tc>::t* r0, TU* u0);

// Krylov (FP64).  Device scalars of one Arnoldi step.
struct ArnoldiScalars {
  double* ww;    // ||w||^2 of the new vector (pass 1)
  double* c;     // normalisation used in pass 2 (Pythagorean norm, or 1)
  double* inv;   // 1/c
  double* q;     // computed ||w - V d||^2
  double* rho2;  // squared norm after re-orthogonalisation
  double* flag;  // 1.0 when the step re-orthogonalised
};
constexpr int kMaxBlocksPerSM = 8;  // 256-thread blocks: partial-sum buffers hold SMs*8 rows
// out = V^T w for nv vectors (stride ldv); optionally *ww = ||w||^2; skipped when gate && *gate == 0
// (gated launches are booked under KC_REORTH with zero bytes; the caller adds them if they ran)
// lp_reorth: gated (re-orthogonalisation) launches take FP32 products of 20-bit truncations;
// false keeps FP64 products there too
cudaError_t launch_multidot(Launch& L, const double* V, size_t ldv, int nv, const double* w, size_t len,
                            double* partial, double* out, double* ww, const double* gate, bool lp_reorth = true);
// v = (v - sum_i coef_i V_i) * (*scale or 1); *q = ||v - sum_i coef_i V_i||^2 (before scaling); gated
cudaError_t launch_update(Launch& L, const double* V, size_t ldv, int nv, const double* coef, double* v, size_t len,
                          const double* scale, double* partial, double* q, const double* gate, float* vf = nullptr,
                          bool lp_reorth = true);
cudaError_t launch_norm2(Launch& L, const double* w, size_t len, double* partial, double* nrm2);
// v *= 1/sqrt(*nrm2); gated
cudaError_t launch_scale_by_inv_norm(Launch& L, double* v, size_t len, const double* nrm2, const double* gate,
                                     float* vf = nullptr);
// y = a*x + b*y (x may be float)
template <typename Tx>
cudaError_t launch_axpby(Launch& L, double a, const Tx* x, double b, double* y, size_t len);
cudaError_t launch_arnoldi_prep(Launch& L, int nv, const double* d, ArnoldiScalars s);
cudaError_t launch_arnoldi_check(Launch& L, ArnoldiScalars s);
// column j of H from d (and e after re-orthogonalisation), Givens update, residual estimate
cudaError_t launch_givens(Launch& L, int j, int ldh, double* H, double* cs, double* sn, double* gvec, const double* d,
                          const double* e, ArnoldiScalars s, double* est, const double* ref);
cudaError_t launch_backsolve(Launch& L, int k, int ldh, const double* H, const double* gvec, double* y);
template <typename Tz>
cudaError_t launch_xupdate(Launch& L, const Tz* Z, size_t ldz, int k, const double* y, double* x, size_t len);
// Device-index variants for graph-captured iterations: the Arnoldi index j is read
// from jdev (nv = j + 1 basis vectors, the new vector is base + (j + 1) * stride),
// launch shapes are sized for nv_max, and their traffic is not booked (no events
// can be recorded inside a conditional graph body).
cudaError_t launch_multidot_dev(Launch& L, const double* V, size_t ldv, int nv_max, const int* jdev,
                                const double* wbase, size_t wstride, size_t len, double* partial, double* out,
                                double* ww, const double* gate, bool lp_reorth = true);
cudaError_t launch_update_dev(Launch& L, const double* V, size_t ldv, int nv_max, const int* jdev, const double* coef,
                              double* vbase, size_t vstride, size_t len, const double* scale, double* partial,
                              double* q, const double* gate, float* vf = nullptr, bool lp_reorth = true);
cudaError_t launch_scale_dev(Launch& L, double* vbase, size_t vstride, const int* jdev, size_t len,
                             const double* nrm2, const double* gate, float* vf = nullptr);
cudaError_t launch_arnoldi_prep_dev(Launch& L, const int* jdev, const double* d, ArnoldiScalars s);
cudaError_t launch_givens_dev(Launch& L, const int* jdev, int ldh, double* H, double* cs, double* sn, double* gvec,
                              const double* d, const double* e, ArnoldiScalars s, double* est, const double* ref);
// loop control of the captured iteration (sets the WHILE condition; k = iterations done)
cudaError_t launch_loop_control(Launch& L, int* jdev, int* kdev, const double* est, double rtol, int maxit,
                                cudaGraphConditionalHandle hc);
cudaError_t launch_loop_start(Launch& L, int* jdev, int* kdev, const double* est, double rtol,
                              cudaGraphConditionalHandle hc);
cudaError_t launch_backsolve_dev(Launch& L, const int* kdev, int ldh, const double* H, const double* gvec, double* y);
template <typename Tz>
cudaError_t launch_xupdate_dev(Launch& L, const Tz* Z, size_t ldz, int kmax, const int* kdev, const double* y,
                               double* x, size_t len);

// start vector: v0 = r / ||r||, gvec[0] = ||r||, ref := ||r0|| or given
cudaError_t launch_arnoldi_start(Launch& L, double* gvec, const double* nrm2, double* est, double* ref_out,
                                 int set_ref);

// RHS assembly and gradient
// double-float basis: each vector two FP32 planes (hi, lo) in a layout tiled by 512
// unknowns, nvt vectors per tile block (vector nv is the new one; len even; the
// allocation holds ceil(len/512) * nvt * 1024 floats).  The first pass streams the
// basis through shared memory with bulk copies; a wait that runs out of its budget
// writes a nonzero value into *err (device) and the kernel returns early.
// gate != nullptr selects the (gated) second pass on the hi planes.  vf receives the
// contiguous hi plane (FP32 rounding) of the vector a kernel finishes.
cudaError_t launch_multidot_df(Launch& L, const float* Vf, int nvt, int nv, const double* w, size_t len,
                               double* partial, double* out, double* ww, const double* gate, double* err);
cudaError_t launch_update_df(Launch& L, float* Vf, int nvt, int nv, const double* coef, const double* w, float* vf,
                             size_t len, const double* scale, double* partial, double* q, const double* gate,
                             double* err);
cudaError_t launch_split_scale(Launch& L, const double* src, float* Vf, int nvt, float* vf, size_t len,
                               const double* nrm2);
cudaError_t launch_scale_df(Launch& L, float* Vf, int nvt, int nv, float* vf, size_t len, const double* nrm2,
                            const double* gate);
cudaError_t launch_multidot_df_dev(Launch& L, const float* Vf, int nvt, int nv_max, const int* jdev, const double* w,
                                   size_t len, double* partial, double* out, double* ww, const double* gate,
                                   double* err);
cudaError_t launch_update_df_dev(Launch& L, float* Vf, int nvt, int nv_max, const int* jdev, const double* coef,
                                 const double* w, float* vf, size_t len, const double* scale, double* partial,
                                 double* q, const double* gate, double* err);
cudaError_t launch_scale_df_dev(Launch& L, float* Vf, int nvt, const int* jdev, float* vf, size_t len,
                                const double* nrm2, const double* gate);
cudaError_t launch_build_rhs(Launch& L, int64_t ms, int n, double tau, double sqrt_gamma, const double* f,
                             const double* g, const double* y0, double* b);

// end-point solves of the time discretisation (k_misc.cu)
cudaError_t launch_endpoint_rhs(Launch& L, const double* x, int64_t ms, int n, double tau, double gamma,
                                const double* fT, const double* g0, const double* y0, const double* pN, double* rhs_y,
                                double* rhs_p);
cudaError_t launch_apply_E(Launch& L, const Grid& g, const Stencil<double>& st, const double* u, double* out);
template <typename Tc>
cudaError_t launch_real_to_plane(Launch& L, const double* v, typename Cx<Tc>::t* plane, int64_t ms);
template <typename TU>
cudaError_t launch_plane_to_real(Launch& L, const TU* plane, double* v, int64_t ms);
// grad_P = scale * a_P * sum_j sum_faces [(l1_P-l1_Q)(x2_P-x2_Q) - (l2_P-l2_Q)(x1_P-x1_Q)]
// a(x) at the interior nodes = exp(log_a) into the nodal array and the interior copy
cudaError_t launch_set_log_coefficient(Launch& L, int dim, int m1, const double* log_a, double* a_nodes,
                                       double* a_int);
// face weights of one level from the fine nodal coefficient (level node I = fine node stride*I)
cudaError_t launch_level_stencil(Launch& L, int dim, int M0, int stride, int m, double tau, double* w64,
                                 double* d64, float* w32, float* d32, float4* w4, float2* wdf, float2* ddf,
                                 const double* a_nodes);
cudaError_t launch_grad_g(Launch& L, const double* lam, int64_t len, double tau, double* out);
cudaError_t launch_objective(Launch& L, const double* x, const double* g, int64_t half, double gamma, double c,
                             double* partial, int max_partial, double* J);
cudaError_t launch_objective_grad(Launch& L, const double* x, const double* g, int64_t half, double gamma, double c,
                                  const double* gJ, double* gx, double* gg);
// ideal RBD preconditioner (Eq. matrix_P): step j of the two block substitutions in time
template <typename Tc, typename TU, typename Tin, typename Tout>
cudaError_t launch_ideal_step(Launch& L, const Tin* v, const TU* u, typename Cx<Tc>::t* r, Tout* w, int64_t ms, int n,
                              int j);
template <typename T>
cudaError_t launch_rbd_butterfly(Launch& L, T* w, int64_t half);
cudaError_t launch_grad_chunked(Launch& L, const Grid& g, int n, double scale, const double* a_int, const double* x,
                                const double* lam, double* partial, int tj, double* grad);

int num_sms();

// record `msg` as the calling thread's last error (pc_last_error) and return `status`
int set_error(int status, const std::string& msg);

}  // namespace pcopt
