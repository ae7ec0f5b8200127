// C ABI of libpcopt (include/pcopt.h): handle set-up, the four-step
// preconditioner apply (Section 2.1), the all-at-once matvec (Eq. matrix_A),
// the GMRES driver (Section 3, Lemma 2.1), the adjoint solve and gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pcopt.h"
#include "common.cuh"

using namespace pcopt;

// ---------------------------------------------------------------------------
// error state
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error = "no error";

static int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}
static int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return PC_ERR_CUDA;
}
namespace pcopt {
int set_error(int status, const std::string& msg) { return fail(status, msg); }
}  // namespace pcopt

#define PC_CUDA(call)                                  \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
namespace pcopt {
const char* kernel_class_name(int kc) {
  static const char* names[KC_COUNT] = {"matvec",        "tfft_forward", "tfft_inverse_butterfly",
                                        "fst_axis",      "fst_divide",   "mg_smooth_rb",
                                        "mg_resid_restrict", "mg_prolong_correct", "mg_coarsest",
                                        "arnoldi_dot",   "arnoldi_update_norm", "reduce_partials",
                                        "normalize",     "givens",       "x_update",
                                        "axpby",         "build_rhs",    "grad_stencil",
                                        "arnoldi_reorth", "mg_coarse_cycle", "mg_down",
                                        "fe_apply",      "ideal_rbd_step"};
  return (kc >= 0 && kc < KC_COUNT) ? names[kc] : "?";
}

void Launch::begin(int kc) {
  ev_a = nullptr;
  if (prof && prof->on && (prof->mask >> kc & 1ull)) {
    if (prof->pool.empty()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) == cudaSuccess) prof->pool.push_back(e);
    }
    if (!prof->pool.empty()) {
      ev_a = prof->pool.back();
      prof->pool.pop_back();
      cudaEventRecord(ev_a, stream);
    }
  }
}

cudaError_t Launch::end(int kc, double bytes, double flops) {
  cudaError_t e = cudaGetLastError();
  if (prof) {
    if (kc != KC_REORTH) prof->launches[kc]++;  // re-orthogonalisations are counted when they ran
    prof->total++;
    prof->bytes[kc] += bytes;
    prof->flops[kc] += flops;
    if (prof->on && ev_a) {
      cudaEvent_t b = nullptr;
      if (prof->pool.empty()) {
        cudaEvent_t t;
        if (cudaEventCreate(&t) == cudaSuccess) prof->pool.push_back(t);
      }
      if (!prof->pool.empty()) {
        b = prof->pool.back();
        prof->pool.pop_back();
        cudaEventRecord(b, stream);
        prof->pending.push_back({kc, ev_a, b});
      } else {
        prof->pool.push_back(ev_a);
      }
    }
  }
  ev_a = nullptr;
  return e;
}

cudaError_t Prof::flush() {
  for (auto& p : pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e != cudaSuccess) return e;
    float t = 0.f;
    e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e != cudaSuccess) return e;
    ms[p.kc] += t;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  return cudaSuccess;
}

void Prof::reset() {
  for (int k = 0; k < KC_COUNT; ++k) {
    launches[k] = 0;
    bytes[k] = 0;
    flops[k] = 0;
    ms[k] = 0;
  }
  total = 0;
}

Prof::~Prof() {
  for (auto& p : pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}
}  // namespace pcopt

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
// time chunks of the element stiffness-derivative partial sums
constexpr int kFeGradChunks = 16;

struct LevelBuf {
  int m = 0;
  int64_t np = 0;
  double* w64 = nullptr;   // [2*dim][np]  tau*a_f/h^2
  double* d64 = nullptr;   // [np]
  float* w32 = nullptr;
  float* d32 = nullptr;
  float4* w4 = nullptr;    // 2D FP32 handles: the four face weights of each point packed (np)
  void* r = nullptr;       // complex spectral planes (Tc)
  void* u = nullptr;
  void* res = nullptr;
  double* e64 = nullptr;   // 2D elements with a nodal coefficient: one value per element ((m+1)^2)
  float* e32 = nullptr;
};

struct pc_handle {
  pc_params prm;
  // caller-provided device memory holding V and Z (pc_setup_shared), else null
  const unsigned char* kws = nullptr;
  size_t kws_bytes = 0;
  int dim = 2, m1 = 0, n = 0, nf = 0, planes = 0, logn = 0;
  int64_t ms = 0;
  size_t U = 0;
  double tau = 0, alpha = 0, sqrtg = 0, h = 0;
  int spatial = PC_SPATIAL_MG;
  bool fp32 = false;
  bool bf16s = false;  // multigrid iterates stored as BF16 pairs (FP32 arithmetic)
  int cap = 0;
  double a_const = 1.0;
  bool fe = false;  // finite elements in space (mass matrix M)
  bool fevar = false;  // elements solved by the element multigrid (any nodal coefficient)
  double* fe_gpart = nullptr;  // elements: per-element partial sums of the stiffness derivative
  bool lex = false;  // multigrid smoother in the natural order (per-level kernels on every level)
  FeScale fes;

  std::vector<LevelBuf> lv;
  int coarse_l0 = 0;                 // first level run by the fused coarse-cycle kernel
  bool tail2 = false;                // 2D FP32 iterates: that kernel is mg_tail2 (from 63^2)
  Tiles tiles;                       // tile shapes of the tunable kernels (0 = default)
  float2* wdf = nullptr;             // level-0 face weights and diagonal as (hi, lo) float pairs
  float2* ddf = nullptr;
  float2 alpha_df{0.f, 0.f};
  CoarseLevels<float> coarse32{};
  CoarseLevels<double> coarse64{};
  // time FFT tables
  double* dpow64 = nullptr;  // eps^{j/n}
  float* dpow32 = nullptr;
  double* dinv64 = nullptr;  // eps^{-j/n}
  float* dinv32 = nullptr;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  double2* sig64 = nullptr;
  double2* sig1_64 = nullptr;  // the shift 1 (end-point solves)
  float2* sig1_32 = nullptr;
  float2* sig32 = nullptr;
  // ideal RBD preconditioner (Eq. matrix_P): the real shift 1 + alpha of both planes
  int precond_kind = PC_PRECOND_EPS_CIRCULANT;
  int arnoldi = PC_ARNOLDI_AUTO;  // pc_arnoldi: basis storage and product precision of flexible GMRES
  double2* sigP64 = nullptr;
  float2* sigP32 = nullptr;
  // FST tables
  double* S64 = nullptr;
  float* S32 = nullptr;
  double* lamK64 = nullptr;
  float* lamK32 = nullptr;
  double* rmass64 = nullptr;  // finite elements: 1 / (eigenvalue of M) per sine mode
  float* rmass32 = nullptr;
  double2* fst_tw64 = nullptr;  // fast sine transforms: exp(-2 pi i q / (2(m+1))), q < 2(m+1)
  float2* fst_tw32 = nullptr;
  void* fst_tmp = nullptr;
  // gradient
  double* a_int = nullptr;
  double* a_nodes_dev = nullptr;  // nodal coefficient incl. the boundary, (m1+2)^dim (device)
  double* grad_partial = nullptr;
  int grad_tj = 16;
  // Krylov workspace
  double* V = nullptr;     // (cap+1) x U
  void* Z = nullptr;       // cap x U (double or float)
  float* vf32 = nullptr;   // U: FP32 rounding of the newest basis vector (mixed handles)
  double* wbuf = nullptr;  // U
  double* tbuf = nullptr;  // U
  double* adjbuf = nullptr;  // U: S c of the adjoint solve
  double* H = nullptr;     // (cap+1) x cap, column-major, ldh = cap+1
  double* cs = nullptr;
  double* sn = nullptr;
  double* gvec = nullptr;
  double* hcol = nullptr;  // 2 x (cap+1)
  double* ycoef = nullptr;
  double* scal = nullptr;  // [0] nrm2, [1] est, [2] ref, [3] tmp, [4..9] Arnoldi step scalars
  double* partial = nullptr;
  int nblocks = 0;         // rows of `partial`: SMs x blocks per SM
  double* host = nullptr;  // pinned, mapped: [0] est, [1] ref, [2] nrm2, ... (16 doubles) + 4 ints
  int last_k = -1;          // iterations of the last solve (-1: none yet)
  double last_res0 = 0.0;   // its initial relative residual (history entry 0)
  double* host_dev = nullptr;  // device view of `host`
  std::vector<void*> allocs;
  Prof prof;
  // graph-captured solve
  int* idx = nullptr;                 // device: [0] Arnoldi index j, [1] iterations done k
  cudaStream_t cap_stream = nullptr;  // capture streams (a batch captures each problem on its own)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t scal_ev = nullptr;      // marks the copy of the per-iteration scalars
  cudaGraphExec_t gexec = nullptr;    // single-problem solve graph and what it was built for
  const double* g_b = nullptr;
  double* g_x = nullptr;
  double g_rtol = 0.0;
  int g_maxit = 0;
};

static int dev_alloc(pc_handle* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  return PC_OK;
}
template <typename T>
static int dev_alloc_t(pc_handle* h, T** p, size_t count) {
  return dev_alloc(h, (void**)p, count * sizeof(T));
}

static void release(pc_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  if (h->scal_ev) cudaEventDestroy(h->scal_ev);
  h->scal_ev = nullptr;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
  h->cap_stream = h->aux_stream = nullptr;
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->host) cudaFreeHost(h->host);
  h->host = nullptr;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static void drop_graphs(pc_handle* h);

// a must be finite, > 0 at interior nodes and >= 0 at boundary nodes (faces to the
// boundary then carry a_f = (a_P + a_Q)/2 > 0, so K stays symmetric positive definite)
static int check_coefficient(const double* a, int m1, int dim) {
  const int M = m1 + 2;
  const size_t nodes = dim == 2 ? (size_t)M * M : (size_t)M * M * M;
  for (size_t i = 0; i < nodes; ++i) {
    const int i1 = (int)(i % M);
    const size_t r = i / M;
    const int i2 = (int)(dim == 2 ? r : r % M);
    const int i3 = dim == 3 ? (int)(r / M) : 1;
    const bool interior = i1 > 0 && i1 < M - 1 && i2 > 0 && i2 < M - 1 && i3 > 0 && i3 < M - 1;
    const double v = a[i];
    if (!std::isfinite(v) || !(interior ? v > 0 : v >= 0))
      return fail(PC_ERR_ARG, "a(x) must be finite, > 0 at interior nodes and >= 0 on the boundary");
  }
  return PC_OK;
}

// per-point face weights tau*a_f/h^2 and their sum for one level (host)
static void level_stencil(const std::vector<double>& a, int m, int dim, double tau, std::vector<double>& w,
                          std::vector<double>& d) {
  const int M = m + 2;
  const int64_t np = dim == 2 ? (int64_t)m * m : (int64_t)m * m * m;
  const double h = 1.0 / (m + 1);
  const double sc = tau / (h * h);
  w.assign((size_t)2 * dim * np, 0.0);
  d.assign((size_t)np, 0.0);
  auto node = [&](int i1, int i2, int i3) -> double {
    return dim == 2 ? a[(size_t)i2 * M + i1] : a[((size_t)i3 * M + i2) * M + i1];
  };
  for (int64_t s = 0; s < np; ++s) {
    const int i1 = (int)(s % m) + 1;
    const int64_t r = s / m;
    const int i2 = (int)(dim == 2 ? r : r % m) + 1;
    const int i3 = dim == 3 ? (int)(r / m) + 1 : 0;
    const double aP = node(i1, i2, i3);
    double nb[6];
    nb[0] = node(i1 - 1, i2, i3);
    nb[1] = node(i1 + 1, i2, i3);
    nb[2] = node(i1, i2 - 1, i3);
    nb[3] = node(i1, i2 + 1, i3);
    if (dim == 3) {
      nb[4] = node(i1, i2, i3 - 1);
      nb[5] = node(i1, i2, i3 + 1);
    }
    double sum = 0.0;
    for (int k = 0; k < 2 * dim; ++k) {
      const double wf = sc * 0.5 * (aP + nb[k]);
      w[(size_t)k * np + s] = wf;
      sum += wf;
    }
    d[(size_t)s] = sum;
  }
}

// stencils of every level: level 0 from `a`, coarser levels (multigrid) from the
// nodal coefficient injected level by level, a_c[I] = a[2I] (boundary nodes included)
static void all_level_stencils(const std::vector<double>& a, int m1, int dim, double tau, bool multigrid,
                               std::vector<std::vector<double>>& ws, std::vector<std::vector<double>>& ds,
                               std::vector<int>& ms) {
  std::vector<double> acur = a;
  int m = m1;
  ws.clear();
  ds.clear();
  ms.clear();
  while (true) {
    std::vector<double> w, d;
    level_stencil(acur, m, dim, tau, w, d);
    ws.push_back(std::move(w));
    ds.push_back(std::move(d));
    ms.push_back(m);
    if (!multigrid || m <= 1) break;
    const int mc = (m - 1) / 2, Mc = mc + 2, Mf = m + 2;
    std::vector<double> ac(dim == 2 ? (size_t)Mc * Mc : (size_t)Mc * Mc * Mc);
    for (size_t q = 0; q < ac.size(); ++q) {
      const int c1 = (int)(q % Mc);
      const size_t rr = q / Mc;
      const int c2 = (int)(dim == 2 ? rr : rr % Mc);
      const int c3 = dim == 3 ? (int)(rr / Mc) : 0;
      ac[q] = dim == 2 ? acur[(size_t)(2 * c2) * Mf + 2 * c1] : acur[((size_t)(2 * c3) * Mf + 2 * c2) * Mf + 2 * c1];
    }
    acur.swap(ac);
    m = mc;
  }
}

// interior values of the nodal coefficient, in vector ordering
static std::vector<double> interior_of(const std::vector<double>& a, int m1, int dim) {
  const int M = m1 + 2;
  const int64_t ms = dim == 2 ? (int64_t)m1 * m1 : (int64_t)m1 * m1 * m1;
  std::vector<double> ai((size_t)ms);
  for (int64_t s = 0; s < ms; ++s) {
    const int i1 = (int)(s % m1) + 1;
    const int64_t r = s / m1;
    const int i2 = (int)(dim == 2 ? r : r % m1) + 1;
    const int i3 = dim == 3 ? (int)(r / m1) + 1 : 0;
    ai[(size_t)s] = dim == 2 ? a[(size_t)i2 * M + i1] : a[((size_t)i3 * M + i2) * M + i1];
  }
  return ai;
}

// FST eigenvalues on the sine modes (i1, i2[, i3]) for a == c.  Finite differences:
// lam = tau c sum_axes 4 sin^2(pi i/(2(m+1)))/h^2 of tau K.  Finite elements: the 1D
// element matrices have the eigenvalues mu_M(i) = h/6 (4 + 2 cos(pi i/(m+1))) and
// mu_K(i) = 4 sin^2(pi i/(2(m+1)))/h, so M has prod_axes mu_M and K has
// c sum_axes mu_K prod_others mu_M; (sigma M + tau K)^{-1} is applied as
// rmass / (sigma + lam) with rmass = 1/eig(M) and lam = tau eig(K)/eig(M).
static std::vector<double> fst_eigenvalues(int m, int dim, double tau, double c, bool fe,
                                           std::vector<double>* rmass = nullptr) {
  const double h = 1.0 / (m + 1);
  std::vector<double> mu(m), muM(m, 1.0);
  for (int i = 0; i < m; ++i) {
    const double sv = std::sin(M_PI * (double)(i + 1) / (2.0 * (m + 1)));
    if (fe) {
      mu[i] = 4.0 * sv * sv / h;
      muM[i] = h / 6.0 * (4.0 + 2.0 * std::cos(M_PI * (double)(i + 1) / (m + 1)));
    } else {
      mu[i] = 4.0 * sv * sv / (h * h);
    }
  }
  const int64_t ms = dim == 2 ? (int64_t)m * m : (int64_t)m * m * m;
  std::vector<double> lam((size_t)ms);
  if (rmass) rmass->assign((size_t)ms, 1.0);
  for (int64_t s = 0; s < ms; ++s) {
    const int ix[3] = {(int)(s % m), (int)(dim == 2 ? s / m : (s / m) % m), dim == 3 ? (int)(s / m / m) : -1};
    double eM = 1.0, eK = 0.0;
    for (int a = 0; a < dim; ++a) {
      double t = mu[ix[a]];
      for (int b = 0; b < dim; ++b)
        if (b != a) t *= muM[ix[b]];
      eK += t;
      eM *= muM[ix[a]];
    }
    lam[(size_t)s] = tau * c * eK / eM;
    if (rmass) (*rmass)[(size_t)s] = 1.0 / eM;
  }
  return lam;
}

template <typename T>
static int upload(pc_handle* h, T** dst, const std::vector<double>& src, cudaStream_t st) {
  std::vector<T> tmp(src.begin(), src.end());
  int rc = dev_alloc_t(h, dst, tmp.size());
  if (rc) return rc;
  PC_CUDA(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

// face weights [4][np] (2D) packed per point for one-load access
// element coefficients of every multigrid level (2D): level l+1 takes level l's nodal
// values at even grid nodes (injection); an element gets the mean of its corner values
static std::vector<std::vector<double>> fe_level_elements(const std::vector<double>& a, int m1, int dim, int nlev) {
  // element value = mean of its 2^dim corner values; a: (m+2)^dim nodes, x1 fastest
  std::vector<std::vector<double>> out;
  std::vector<double> acur = a;
  int m = m1;
  for (int l = 0; l < nlev; ++l) {
    const size_t Mn = (size_t)m + 2, me = (size_t)m + 1;
    const size_t ne = dim == 2 ? me * me : me * me * me;
    std::vector<double> E(ne);
    for (size_t el = 0; el < ne; ++el) {
      const size_t k1 = el % me, k2 = (el / me) % me, k3 = dim == 2 ? 0 : el / (me * me);
      double v = 0.0;
      for (int c = 0; c < (1 << dim); ++c) {
        const size_t n1 = k1 + (c & 1), n2 = k2 + ((c >> 1) & 1), n3 = dim == 2 ? 0 : k3 + (c >> 2);
        v += acur[(n3 * Mn + n2) * Mn + n1];
      }
      E[el] = v / (1 << dim);
    }
    out.push_back(std::move(E));
    if (l + 1 == nlev) break;
    const size_t mc = ((size_t)m - 1) / 2, Mc = mc + 2;
    std::vector<double> ac(dim == 2 ? Mc * Mc : Mc * Mc * Mc);
    for (size_t q = 0; q < ac.size(); ++q) {
      const size_t I = q % Mc, J = (q / Mc) % Mc, K = dim == 2 ? 0 : q / (Mc * Mc);
      ac[q] = acur[((2 * K) * Mn + 2 * J) * Mn + 2 * I];
    }
    acur.swap(ac);
    m = (int)mc;
  }
  return out;
}

static std::vector<float4> pack_w4(const std::vector<double>& w, int64_t np) {
  std::vector<float4> t((size_t)np);
  for (int64_t i = 0; i < np; ++i)
    t[i] = make_float4((float)w[i], (float)w[np + i], (float)w[2 * np + i], (float)w[3 * np + i]);
  return t;
}

static int upload_c(pc_handle* h, void** dst, const std::vector<double>& re, const std::vector<double>& im, bool f32,
                    cudaStream_t st) {
  const size_t n = re.size();
  if (f32) {
    std::vector<float2> t(n);
    for (size_t i = 0; i < n; ++i) t[i] = make_float2((float)re[i], (float)im[i]);
    int rc = dev_alloc(h, dst, n * sizeof(float2));
    if (rc) return rc;
    PC_CUDA(cudaMemcpyAsync(*dst, t.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaStreamSynchronize(st));
  } else {
    std::vector<double2> t(n);
    for (size_t i = 0; i < n; ++i) t[i] = make_double2(re[i], im[i]);
    int rc = dev_alloc(h, dst, n * sizeof(double2));
    if (rc) return rc;
    PC_CUDA(cudaMemcpyAsync(*dst, t.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaStreamSynchronize(st));
  }
  return PC_OK;
}

// bytes of the Krylov basis V (cap + 1 vectors of the tiled layout, 8 bytes per
// unknown) and of the preconditioned vectors Z (cap vectors, FP32 or FP64), each
// part rounded up to 256 bytes; Z follows V
static size_t round256(size_t b) { return (b + 255) / 256 * 256; }
static size_t krylov_v_bytes(size_t U, int cap) { return round256((size_t)(cap + 1) * ((U + 511) / 512 * 512) * 8); }
static size_t krylov_bytes_of(size_t U, int cap, bool fp32) {
  return krylov_v_bytes(U, cap) + round256((size_t)cap * U * (fp32 ? sizeof(float) : sizeof(double)));
}
static int resolved_precision(const pc_params* p) {
  return p->precision == PC_PREC_AUTO ? (p->eps >= PC_AUTO_FP32_MIN_EPS ? PC_PREC_MIXED_FP32 : PC_PREC_FP64)
                                      : p->precision;
}

static int setup_impl(const pc_params* p, const double* a_nodes, void* krylov, size_t krylov_bytes, void* stream,
                      pc_handle** out);

extern "C" int pc_setup(const pc_params* p, const double* a_nodes, void* stream, pc_handle** out) {
  return setup_impl(p, a_nodes, nullptr, 0, stream, out);
}

extern "C" int pc_krylov_bytes(const pc_params* p, size_t* bytes) {
  if (!p || !bytes) return fail(PC_ERR_ARG, "pc_krylov_bytes: null argument");
  if (p->dim != 2 && p->dim != 3) return fail(PC_ERR_ARG, "dim must be 2 or 3");
  if (p->m1 < 1 || p->m1 > 4095) return fail(PC_ERR_ARG, "m1 must be in [1, 4095]");
  if (p->n < 1 || p->n > 4096) return fail(PC_ERR_ARG, "n must be in [1, 4096]");
  if (p->max_iter < 1 || p->max_iter > 1000) return fail(PC_ERR_ARG, "max_iter must be in [1, 1000]");
  if (!(p->eps > 0) || !(p->eps <= 1.0)) return fail(PC_ERR_ARG, "eps must lie in (0, 1]");
  const int prec = resolved_precision(p);
  if (prec != PC_PREC_FP64 && prec != PC_PREC_MIXED_FP32 && prec != PC_PREC_MIXED_BF16S)
    return fail(PC_ERR_ARG, "unknown precision");
  const size_t ms = p->dim == 2 ? (size_t)p->m1 * p->m1 : (size_t)p->m1 * p->m1 * p->m1;
  *bytes = krylov_bytes_of(2 * (size_t)p->n * ms, p->max_iter, prec != PC_PREC_FP64);
  return PC_OK;
}

extern "C" int pc_setup_shared(const pc_params* p, const double* a_nodes, void* krylov, size_t krylov_bytes,
                               void* stream, pc_handle** out) {
  if (!out) return fail(PC_ERR_ARG, "pc_setup_shared: null out pointer");
  *out = nullptr;
  if (!krylov) return fail(PC_ERR_ARG, "pc_setup_shared: null workspace");
  if (reinterpret_cast<uintptr_t>(krylov) % 256 != 0)
    return fail(PC_ERR_ARG, "pc_setup_shared: the workspace must be 256-byte aligned");
  size_t need = 0;
  if (int rc = pc_krylov_bytes(p, &need)) return rc;
  if (krylov_bytes < need)
    return fail(PC_ERR_ARG, "pc_setup_shared: workspace of " + std::to_string(krylov_bytes) + " bytes, " +
                                std::to_string(need) + " needed");
  return setup_impl(p, a_nodes, krylov, krylov_bytes, stream, out);
}

static int setup_impl(const pc_params* p, const double* a_nodes, void* krylov, size_t krylov_bytes, void* stream,
                      pc_handle** out) {
  if (!p || !out) return fail(PC_ERR_ARG, "pc_setup: null params or out pointer");
  *out = nullptr;
  if (p->dim != 2 && p->dim != 3) return fail(PC_ERR_ARG, "dim must be 2 or 3");
  if (p->m1 < 1 || p->m1 > 4095) return fail(PC_ERR_ARG, "m1 must be in [1, 4095]");
  if (p->n < 1) return fail(PC_ERR_ARG, "n must be >= 1");
  if (p->n > 4096) return fail(PC_ERR_ARG, "n must be <= 4096");
  if (!(p->T > 0) || !std::isfinite(p->T)) return fail(PC_ERR_ARG, "T must be finite and > 0");
  if (!(p->gamma > 0) || !std::isfinite(p->gamma)) return fail(PC_ERR_ARG, "gamma must be finite and > 0");
  if (!(p->eps > 0) || !(p->eps <= 1.0)) return fail(PC_ERR_ARG, "eps must lie in (0, 1]");
  if (p->precision != PC_PREC_FP64 && p->precision != PC_PREC_MIXED_FP32 && p->precision != PC_PREC_MIXED_BF16S &&
      p->precision != PC_PREC_AUTO)
    return fail(PC_ERR_ARG, "unknown precision");
  if (p->spatial < 0 || p->spatial > 2) return fail(PC_ERR_ARG, "unknown spatial solver");
  if (p->max_iter < 1 || p->max_iter > 1000) return fail(PC_ERR_ARG, "max_iter must be in [1, 1000]");
  if (p->space != PC_SPACE_FD && p->space != PC_SPACE_FE) return fail(PC_ERR_ARG, "unknown space discretisation");
  if (p->smoother != PC_SMOOTHER_RED_BLACK && p->smoother != PC_SMOOTHER_LEXICOGRAPHIC)
    return fail(PC_ERR_ARG, "unknown smoother");

  const int dim = p->dim, m1 = p->m1;
  const int M = m1 + 2;
  const size_t nodes = dim == 2 ? (size_t)M * M : (size_t)M * M * M;
  std::vector<double> a(nodes, 1.0);
  bool constant = true;
  if (a_nodes) {
    if (int rc = check_coefficient(a_nodes, m1, dim)) return rc;
    for (size_t i = 0; i < nodes; ++i) {
      a[i] = a_nodes[i];
      if (a_nodes[i] != a_nodes[0]) constant = false;
    }
  }
  int spatial = p->spatial;
  const bool fe = p->space == PC_SPACE_FE;
  if (fe && p->smoother == PC_SMOOTHER_LEXICOGRAPHIC)
    return fail(PC_ERR_UNSUPPORTED, "finite elements: the element multigrid smooths in colour order only");
  if (fe && p->precision == PC_PREC_MIXED_BF16S && (!constant || spatial == PC_SPATIAL_MG))
    return fail(PC_ERR_UNSUPPORTED, "finite elements: no BF16-storage element multigrid");
  if (spatial == PC_SPATIAL_AUTO) spatial = constant ? PC_SPATIAL_FST : PC_SPATIAL_MG;
  if (spatial == PC_SPATIAL_FST && !constant) return fail(PC_ERR_ARG, "FST needs a constant coefficient a");
  if (spatial == PC_SPATIAL_MG && ((m1 + 1) & m1) != 0) return fail(PC_ERR_ARG, "multigrid needs m1 = 2^k - 1");

  pc_handle* h = new (std::nothrow) pc_handle();
  if (!h) return fail(PC_ERR_OOM, "host allocation failed");
  h->prm = *p;
  h->dim = dim;
  h->m1 = m1;
  h->n = p->n;
  h->nf = p->n / 2 + 1;
  h->planes = 2 * h->nf;
  h->logn = 0;
  while ((1 << h->logn) < h->n) h->logn++;
  h->ms = dim == 2 ? (int64_t)m1 * m1 : (int64_t)m1 * m1 * m1;
  h->U = (size_t)2 * h->n * h->ms;
  h->tau = p->T / (p->n + 1);
  h->alpha = h->tau / std::sqrt(p->gamma);
  h->sqrtg = std::sqrt(p->gamma);
  h->h = 1.0 / (m1 + 1);
  h->spatial = spatial;
  const int prec = resolved_precision(p);
  h->prm.precision = prec;
  h->fp32 = prec != PC_PREC_FP64;
  h->bf16s = prec == PC_PREC_MIXED_BF16S && spatial == PC_SPATIAL_MG;
  h->cap = p->max_iter;
  h->a_const = a[0];
  h->fe = fe;
  h->fevar = fe && spatial == PC_SPATIAL_MG;
  h->fes = fe_scale(dim, m1, h->a_const);
  h->lex = spatial == PC_SPATIAL_MG && p->smoother == PC_SMOOTHER_LEXICOGRAPHIC;
  h->prof.on = false;
  cudaStream_t st = (cudaStream_t)stream;

  int rc = PC_OK;
  const size_t cb = h->fp32 ? sizeof(float2) : sizeof(double2);
  const size_t ub = h->bf16s ? sizeof(__nv_bfloat162) : cb;  // storage of the multigrid iterates
  // ---- level hierarchy: level 0 always (matvec), coarser ones for multigrid
  {
    std::vector<std::vector<double>> ws, ds;
    std::vector<int> mlev;
    all_level_stencils(a, m1, dim, h->tau, spatial == PC_SPATIAL_MG, ws, ds, mlev);
    const std::vector<std::vector<double>> els =
        h->fevar ? fe_level_elements(a, m1, dim, (int)mlev.size()) : std::vector<std::vector<double>>();
    for (size_t l = 0; l < mlev.size(); ++l) {
      LevelBuf L;
      L.m = mlev[l];
      L.np = dim == 2 ? (int64_t)L.m * L.m : (int64_t)L.m * L.m * L.m;
      if ((rc = upload(h, &L.w64, ws[l], st))) goto fail_out;
      if ((rc = upload(h, &L.d64, ds[l], st))) goto fail_out;
      if ((rc = upload(h, &L.w32, ws[l], st))) goto fail_out;
      if ((rc = upload(h, &L.d32, ds[l], st))) goto fail_out;
      if (h->fevar) {
        if ((rc = upload(h, &L.e64, els[l], st))) goto fail_out;
        if ((rc = upload(h, &L.e32, els[l], st))) goto fail_out;
      }
      if (dim == 2 && h->fp32) {
        const std::vector<float4> w4 = pack_w4(ws[l], L.np);
        if ((rc = dev_alloc_t(h, &L.w4, w4.size()))) goto fail_out;
        if (cudaMemcpyAsync(L.w4, w4.data(), w4.size() * sizeof(float4), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          rc = fail(PC_ERR_CUDA, "upload of packed face weights failed");
          goto fail_out;
        }
      }
      if ((rc = dev_alloc(h, &L.r, (size_t)h->planes * L.np * cb))) goto fail_out;
      if ((rc = dev_alloc(h, &L.u, (size_t)h->planes * L.np * ub))) goto fail_out;
      // per-level residual planes: the 3D path and the natural-order smoother write them
      // (the 2D red-black down leg fuses the residual away)
      if ((dim == 3 || h->lex || h->fevar) && l + 1 < mlev.size() &&
          (rc = dev_alloc(h, &L.res, (size_t)h->planes * L.np * cb)))
        goto fail_out;
      h->lv.push_back(L);
    }
    // double-float copies of the level-0 stencil for the inner matvec of flexible GMRES
    {
      auto split = [](const std::vector<double>& v) {
        std::vector<float2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
          const float hi = (float)v[i];
          o[i] = make_float2(hi, (float)(v[i] - (double)hi));
        }
        return o;
      };
      const std::vector<float2> wsp = split(ws[0]), dsp = split(ds[0]);
      if ((rc = dev_alloc_t(h, &h->wdf, wsp.size()))) goto fail_out;
      if ((rc = dev_alloc_t(h, &h->ddf, dsp.size()))) goto fail_out;
      cudaError_t ce = cudaMemcpyAsync(h->wdf, wsp.data(), wsp.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(h->ddf, dsp.data(), dsp.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) {
        rc = cuda_fail(ce, "pc_setup: double-float stencil");
        goto fail_out;
      }
      const float ah = (float)h->alpha;
      h->alpha_df = make_float2(ah, (float)(h->alpha - (double)ah));
    }
    // the fused lower cycle takes every level from the first with m <= 63 (2D, FP32
    // iterates: one in-place array per level), 31 (2D, FP64 iterates or BF16 storage)
    // or 15 (3D).  (The in-place kernel also runs FP64 iterates, but one CTA of 133 KB
    // per plane made the ideal preconditioner's two-plane steps slower: 29.6 -> 34.8
    // ms per apply at 255^2 x 256.)
    h->tail2 = dim == 2 && h->fp32 && !h->bf16s && !h->fevar;
    const int mthr = h->tail2 ? kMgTailMaxM : (dim == 2 ? 31 : 15);
    int l0 = (int)h->lv.size() - 1;
    while (l0 > 0 && h->lv[l0 - 1].m <= mthr) --l0;
    if ((int)h->lv.size() - l0 > kMaxCoarseLevels) l0 = (int)h->lv.size() - kMaxCoarseLevels;
    h->coarse_l0 = l0;
    h->coarse32.count = h->coarse64.count = (int)h->lv.size() - l0;
    for (int l = l0; l < (int)h->lv.size(); ++l) {
      const int q = l - l0;
      h->coarse32.m[q] = h->coarse64.m[q] = h->lv[l].m;
      h->coarse32.np[q] = h->coarse64.np[q] = h->lv[l].np;
      h->coarse32.w[q] = h->lv[l].w32;
      h->coarse32.diag[q] = h->lv[l].d32;
      h->coarse64.w[q] = h->lv[l].w64;
      h->coarse64.diag[q] = h->lv[l].d64;
    }
  }
  // ---- time FFT tables
  {
    const int n = h->n;
    // full circle of twiddles exp(-2 pi i k / n), k = 0..n-1
    std::vector<double> dp(n), di(n), twr(n), twi(n);
    for (int j = 0; j < n; ++j) {
      dp[j] = std::pow(p->eps, (double)j / n);
      di[j] = std::pow(p->eps, -(double)j / n);
    }
    for (int k = 0; k < n; ++k) {
      const double th = 2.0 * M_PI * (double)k / n;
      twr[k] = std::cos(th);
      twi[k] = -std::sin(th);
    }
    std::vector<double> sr(h->planes), si(h->planes);
    const double e1n = std::pow(p->eps, 1.0 / n);
    for (int q = 0; q < h->planes; ++q) {
      const int k = q / 2;
      const double th = 2.0 * M_PI * (double)k / n;
      // sigma_k = lambda_k + alpha, lambda_k = 1 - eps^{1/n} exp(-2 pi i k / n)
      sr[q] = 1.0 + h->alpha - e1n * std::cos(th);
      si[q] = (k == 0 || 2 * k == n) ? 0.0 : e1n * std::sin(th);
    }
    if ((rc = upload(h, &h->dpow64, dp, st))) goto fail_out;
    if ((rc = upload(h, &h->dpow32, dp, st))) goto fail_out;
    if ((rc = upload(h, &h->dinv64, di, st))) goto fail_out;
    if ((rc = upload(h, &h->dinv32, di, st))) goto fail_out;
    if ((rc = upload_c(h, (void**)&h->tw64, twr, twi, false, st))) goto fail_out;
    if ((rc = upload_c(h, (void**)&h->tw32, twr, twi, true, st))) goto fail_out;
    if ((rc = upload_c(h, (void**)&h->sig64, sr, si, false, st))) goto fail_out;
    if ((rc = upload_c(h, (void**)&h->sig32, sr, si, true, st))) goto fail_out;
    const std::vector<double> one{1.0}, zero{0.0};
    if ((rc = upload_c(h, (void**)&h->sig1_64, one, zero, false, st))) goto fail_out;
    if ((rc = upload_c(h, (void**)&h->sig1_32, one, zero, true, st))) goto fail_out;
    const std::vector<double> shiftP(2, 1.0 + h->alpha), zero2(2, 0.0);
    if ((rc = upload_c(h, (void**)&h->sigP64, shiftP, zero2, false, st))) goto fail_out;
    if ((rc = upload_c(h, (void**)&h->sigP32, shiftP, zero2, true, st))) goto fail_out;
  }
  // ---- FST tables (constant a)
  if (spatial == PC_SPATIAL_FST) {
    const int m = m1;
    std::vector<double> S((size_t)m * m);
    const double sc = std::sqrt(2.0 / (m + 1));
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) S[(size_t)i * m + j] = sc * std::sin(M_PI * (double)(i + 1) * (j + 1) / (m + 1));
    std::vector<double> rmass;
    const std::vector<double> lam = fst_eigenvalues(m, dim, h->tau, h->a_const, fe, &rmass);
    if ((rc = upload(h, &h->S64, S, st))) goto fail_out;
    if ((rc = upload(h, &h->S32, S, st))) goto fail_out;
    if ((rc = upload(h, &h->lamK64, lam, st))) goto fail_out;
    if ((rc = upload(h, &h->lamK32, lam, st))) goto fail_out;
    if (fe && (rc = upload(h, &h->rmass64, rmass, st))) goto fail_out;
    if (fe && (rc = upload(h, &h->rmass32, rmass, st))) goto fail_out;
    if (fst_fast_supported<float>(m)) {
      const int Lf = 2 * (m + 1);
      std::vector<double> twr(Lf), twi(Lf);
      for (int q = 0; q < Lf; ++q) {
        twr[q] = std::cos(2.0 * M_PI * q / Lf);
        twi[q] = -std::sin(2.0 * M_PI * q / Lf);
      }
      if ((rc = upload_c(h, (void**)&h->fst_tw64, twr, twi, false, st))) goto fail_out;
      if ((rc = upload_c(h, (void**)&h->fst_tw32, twr, twi, true, st))) goto fail_out;
    }
    if ((rc = dev_alloc(h, &h->fst_tmp, (size_t)h->planes * h->ms * cb))) goto fail_out;
  }
  // ---- interior coefficient (gradient) and its scratch
  {
    if ((rc = upload(h, &h->a_int, interior_of(a, m1, dim), st))) goto fail_out;
    if ((rc = upload(h, &h->a_nodes_dev, a, st))) goto fail_out;
    const int nch = (h->n + h->grad_tj - 1) / h->grad_tj;
    if ((rc = dev_alloc_t(h, &h->grad_partial, (size_t)nch * h->ms))) goto fail_out;
    if (fe && (rc = dev_alloc_t(h, &h->fe_gpart, (size_t)kFeGradChunks * (m1 + 1) * (m1 + 1) *
                                                   (dim == 3 ? (size_t)(m1 + 1) : 1))))
      goto fail_out;
  }
  // ---- Krylov workspace
  {
    const size_t U = h->U;
    const int cap = h->cap;
    h->nblocks = num_sms() * kMaxBlocksPerSM;
    // basis: cap + 1 vectors; a double-float basis stores each as two FP32 planes in
    // tiles of 512 unknowns (the last tile padded), i.e. ceil(U/512) * 512 doubles per vector
    const size_t tiled = (U + 511) / 512 * 512;
    if (krylov) {
      // V and Z in the caller's memory (checked by pc_setup_shared), Z after V
      h->kws = static_cast<const unsigned char*>(krylov);
      h->kws_bytes = krylov_bytes_of(U, cap, h->fp32);
      h->V = static_cast<double*>(krylov);
      h->Z = static_cast<unsigned char*>(krylov) + krylov_v_bytes(U, cap);
    } else {
      if ((rc = dev_alloc_t(h, &h->V, (size_t)(cap + 1) * tiled))) goto fail_out;
      if ((rc = dev_alloc(h, &h->Z, (size_t)cap * U * (h->fp32 ? sizeof(float) : sizeof(double))))) goto fail_out;
    }
    if (h->fp32 && (rc = dev_alloc_t(h, &h->vf32, U))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->wbuf, U))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->tbuf, U))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->adjbuf, U))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->H, (size_t)(cap + 1) * cap))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->cs, (size_t)cap + 1))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->sn, (size_t)cap + 1))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->gvec, (size_t)cap + 2))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->hcol, (size_t)2 * (cap + 1)))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->ycoef, (size_t)cap + 1))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->scal, 16))) goto fail_out;
    if (cudaMemsetAsync(h->scal, 0, 16 * sizeof(double), st) != cudaSuccess) {
      rc = fail(PC_ERR_CUDA, "pc_setup: scalar workspace");
      goto fail_out;
    }
    if ((rc = dev_alloc_t(h, &h->partial, (size_t)h->nblocks * (cap + 2)))) goto fail_out;
    if ((rc = dev_alloc_t(h, &h->idx, 4))) goto fail_out;
    // scalars come back through mapped pinned memory written by a kernel, so the
    // solver's per-iteration reads never queue behind bulk copies on a copy engine
    cudaError_t e = cudaHostAlloc((void**)&h->host, 18 * sizeof(double), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&h->host_dev, h->host, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = fail(PC_ERR_OOM, "mapped pinned host allocation failed");
      goto fail_out;
    }
  }
  {
    {
      int dev = 0;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&h->tiles.sms, cudaDevAttrMultiProcessorCount, dev);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->scal_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "pc_setup");
      goto fail_out;
    }
  }
  *out = h;
  return PC_OK;
fail_out:
  release(h);
  delete h;
  return rc;
}

template <typename T>
static int refill(T* dst, const std::vector<double>& src, cudaStream_t st, std::vector<T>& stage) {
  stage.assign(src.begin(), src.end());
  PC_CUDA(cudaMemcpyAsync(dst, stage.data(), stage.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

extern "C" int pc_set_coefficient(pc_handle* h, const double* a_nodes, void* stream) {
  if (!h) return fail(PC_ERR_ARG, "pc_set_coefficient: null handle");
  const int dim = h->dim, m1 = h->m1, M = m1 + 2;
  const size_t nodes = dim == 2 ? (size_t)M * M : (size_t)M * M * M;
  std::vector<double> a(nodes, 1.0);
  bool constant = true;
  if (a_nodes) {
    if (int rc = check_coefficient(a_nodes, m1, dim)) return rc;
    for (size_t i = 0; i < nodes; ++i) {
      a[i] = a_nodes[i];
      if (a_nodes[i] != a_nodes[0]) constant = false;
    }
  }
  if (h->spatial == PC_SPATIAL_FST && !constant) return fail(PC_ERR_ARG, "FST handle needs a constant coefficient");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<std::vector<double>> ws, ds;
  std::vector<int> mlev;
  all_level_stencils(a, m1, dim, h->tau, h->spatial == PC_SPATIAL_MG, ws, ds, mlev);
  if (mlev.size() != h->lv.size()) return fail(PC_ERR_ARG, "pc_set_coefficient: level mismatch");
  std::vector<double> s64;
  std::vector<float> s32;
  int rc;
  for (size_t l = 0; l < mlev.size(); ++l) {
    if ((rc = refill(h->lv[l].w64, ws[l], st, s64))) return rc;
    if ((rc = refill(h->lv[l].d64, ds[l], st, s64))) return rc;
    if ((rc = refill(h->lv[l].w32, ws[l], st, s32))) return rc;
    if ((rc = refill(h->lv[l].d32, ds[l], st, s32))) return rc;
    if (h->lv[l].w4) {
      const std::vector<float4> w4 = pack_w4(ws[l], h->lv[l].np);
      PC_CUDA(cudaMemcpyAsync(h->lv[l].w4, w4.data(), w4.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
      PC_CUDA(cudaStreamSynchronize(st));
    }
  }
  if (h->fevar) {
    const std::vector<std::vector<double>> els = fe_level_elements(a, m1, dim, (int)mlev.size());
    for (size_t l = 0; l < mlev.size(); ++l) {
      if ((rc = refill(h->lv[l].e64, els[l], st, s64))) return rc;
      if ((rc = refill(h->lv[l].e32, els[l], st, s32))) return rc;
    }
  }
  {
    std::vector<float2> wsp(ws[0].size()), dsp(ds[0].size());
    for (size_t i = 0; i < wsp.size(); ++i) {
      const float hi = (float)ws[0][i];
      wsp[i] = make_float2(hi, (float)(ws[0][i] - (double)hi));
    }
    for (size_t i = 0; i < dsp.size(); ++i) {
      const float hi = (float)ds[0][i];
      dsp[i] = make_float2(hi, (float)(ds[0][i] - (double)hi));
    }
    PC_CUDA(cudaMemcpyAsync(h->wdf, wsp.data(), wsp.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(h->ddf, dsp.data(), dsp.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaStreamSynchronize(st));
  }
  if ((rc = refill(h->a_int, interior_of(a, m1, dim), st, s64))) return rc;
  if ((rc = refill(h->a_nodes_dev, a, st, s64))) return rc;
  h->a_const = a[0];
  h->fes = fe_scale(dim, m1, h->a_const);
  if (h->spatial == PC_SPATIAL_FST) {
    const std::vector<double> lam = fst_eigenvalues(m1, dim, h->tau, h->a_const, h->fe);
    if ((rc = refill(h->lamK64, lam, st, s64))) return rc;
    if ((rc = refill(h->lamK32, lam, st, s32))) return rc;
  }
  return PC_OK;
}

extern "C" int pc_set_log_coefficient(pc_handle* h, const double* log_a, void* stream) {
  if (!h || !log_a) return fail(PC_ERR_ARG, "pc_set_log_coefficient: null argument");
  if (h->spatial != PC_SPATIAL_MG)
    return fail(PC_ERR_UNSUPPORTED, "pc_set_log_coefficient: variable-coefficient (multigrid) handles only");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  cudaError_t e = launch_set_log_coefficient(L, h->dim, h->m1, log_a, h->a_nodes_dev, h->a_int);
  if (h->fevar) {
    int st = 1;
    for (size_t l = 0; l < h->lv.size() && e == cudaSuccess; ++l, st *= 2)
      e = h->dim == 3
              ? launch_fevar3_level_elements(L, h->a_nodes_dev, h->m1 + 2, st, h->lv[l].m, h->lv[l].e64, h->lv[l].e32)
              : launch_fevar_level_elements(L, h->a_nodes_dev, h->m1 + 2, st, h->lv[l].m, h->lv[l].e64, h->lv[l].e32);
    return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_set_log_coefficient");
  }
  int stride = 1;
  for (size_t l = 0; l < h->lv.size() && e == cudaSuccess; ++l, stride *= 2) {
    LevelBuf& B = h->lv[l];
    e = launch_level_stencil(L, h->dim, h->m1 + 2, stride, B.m, h->tau, B.w64, B.d64, B.w32, B.d32, B.w4,
                             l == 0 ? h->wdf : nullptr, l == 0 ? h->ddf : nullptr, h->a_nodes_dev);
  }
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_set_log_coefficient");
}

extern "C" int pc_set_preconditioner(pc_handle* h, int kind) {
  if (!h) return fail(PC_ERR_ARG, "pc_set_preconditioner: null handle");
  if (kind != PC_PRECOND_EPS_CIRCULANT && kind != PC_PRECOND_IDEAL_RBD)
    return fail(PC_ERR_ARG, "pc_set_preconditioner: unknown kind");
  if (kind == PC_PRECOND_IDEAL_RBD && h->fe)
    return fail(PC_ERR_UNSUPPORTED, "pc_set_preconditioner: the ideal RBD preconditioner needs finite differences");
  if (kind != h->precond_kind) drop_graphs(h);
  h->precond_kind = kind;
  return PC_OK;
}

extern "C" int pc_set_arnoldi(pc_handle* h, int mode) {
  if (!h) return fail(PC_ERR_ARG, "pc_set_arnoldi: null handle");
  if (mode < PC_ARNOLDI_AUTO || mode > PC_ARNOLDI_DOUBLE_FLOAT) return fail(PC_ERR_ARG, "pc_set_arnoldi: unknown mode");
  if (mode == PC_ARNOLDI_DOUBLE_FLOAT && !h->fp32)
    return fail(PC_ERR_UNSUPPORTED, "pc_set_arnoldi: the double-float basis serves the FP32 preconditioner");
  if (mode != h->arnoldi) drop_graphs(h);
  h->arnoldi = mode;
  return PC_OK;
}

extern "C" int pc_destroy(pc_handle* h) {
  if (!h) return PC_OK;
  cudaDeviceSynchronize();
  release(h);
  delete h;
  return PC_OK;
}

extern "C" int pc_precision_of(const pc_handle* h, int* precision) {
  if (!h || !precision) return fail(PC_ERR_ARG, "pc_precision_of: null argument");
  *precision = h->prm.precision;
  return PC_OK;
}

extern "C" int pc_sizes(const pc_handle* h, int64_t* ms, int64_t* vec_len) {
  if (!h) return fail(PC_ERR_ARG, "null handle");
  if (ms) *ms = h->ms;
  if (vec_len) *vec_len = (int64_t)h->U;
  return PC_OK;
}

// ---------------------------------------------------------------------------
// internal operators
// ---------------------------------------------------------------------------
static Grid grid_of(const pc_handle* h, int l) {
  Grid g;
  g.dim = h->dim;
  g.m = h->lv[l].m;
  g.np = h->lv[l].np;
  return g;
}

template <typename Tc>
static const Tc* lvw(const LevelBuf& L);
template <>
const double* lvw<double>(const LevelBuf& L) { return L.w64; }
template <>
const float* lvw<float>(const LevelBuf& L) { return L.w32; }
template <typename Tc>
static const Tc* lvd(const LevelBuf& L);
template <>
const double* lvd<double>(const LevelBuf& L) { return L.d64; }
template <>
const float* lvd<float>(const LevelBuf& L) { return L.d32; }

template <typename Tc>
static const Tc* lve(const LevelBuf& L);
template <>
const double* lve<double>(const LevelBuf& L) { return L.e64; }
template <>
const float* lve<float>(const LevelBuf& L) { return L.e32; }

// element multigrid (k_fevar.cu in 2D, k_fevar3.cu in 3D): on every level a
// colour-ordered Gauss-Seidel sweep from zero, residual and restriction by P^T; the
// one-point level is solved by its sweep; then the (bi/tri)linear corrections from the
// coarsest level up
template <typename Tc>
static cudaError_t fevar_spatial(pc_handle* h, Launch& L, int P, const typename Cx<Tc>::t* sig) {
  typedef typename Cx<Tc>::t C;
  const int nl = (int)h->lv.size();
  const Tc tau = (Tc)h->tau;
  cudaError_t e;
  for (int l = 0; l < nl; ++l) {
    const LevelBuf& B = h->lv[l];
    const Tc hl = Tc(1) / Tc(B.m + 1);
    const Tc* E = lve<Tc>(B);
    e = h->dim == 3 ? launch_fevar3_smooth<Tc>(L, B.m, P, hl, tau, E, sig, (const C*)B.r, (C*)B.u)
                    : launch_fevar_smooth<Tc>(L, B.m, P, hl * hl, tau, E, sig, (const C*)B.r, (C*)B.u);
    if (e != cudaSuccess) return e;
    if (l + 1 == nl) break;
    e = h->dim == 3 ? launch_fevar3_resid_restrict<Tc>(L, B.m, P, hl, tau, E, sig, (const C*)B.r, (const C*)B.u,
                                                       (C*)B.res, (C*)h->lv[l + 1].r)
                    : launch_fevar_resid_restrict<Tc>(L, B.m, P, hl * hl, tau, E, sig, (const C*)B.r,
                                                      (const C*)B.u, (C*)B.res, (C*)h->lv[l + 1].r);
    if (e != cudaSuccess) return e;
  }
  for (int l = nl - 2; l >= 0; --l)
    if ((e = launch_mg_prolong<Tc, C>(L, grid_of(h, l), P, (const C*)h->lv[l + 1].u, (C*)h->lv[l].u)) != cudaSuccess)
      return e;
  return cudaSuccess;
}

template <typename Tc>
struct Tables;
template <>
struct Tables<double> {
  static const double* dpow(const pc_handle* h) { return h->dpow64; }
  static const double* dinv(const pc_handle* h) { return h->dinv64; }
  static const double2* tw(const pc_handle* h) { return h->tw64; }
  static const double2* sig(const pc_handle* h) { return h->sig64; }
  static const double2* sig1(const pc_handle* h) { return h->sig1_64; }
  static const double2* sigP(const pc_handle* h) { return h->sigP64; }
  static const double* S(const pc_handle* h) { return h->S64; }
  static const double* lamK(const pc_handle* h) { return h->lamK64; }
  static const double* rmass(const pc_handle* h) { return h->rmass64; }
  static const double2* fst_tw(const pc_handle* h) { return h->fst_tw64; }
};
template <>
struct Tables<float> {
  static const float* dpow(const pc_handle* h) { return h->dpow32; }
  static const float* dinv(const pc_handle* h) { return h->dinv32; }
  static const float2* tw(const pc_handle* h) { return h->tw32; }
  static const float2* sig(const pc_handle* h) { return h->sig32; }
  static const float2* sig1(const pc_handle* h) { return h->sig1_32; }
  static const float2* sigP(const pc_handle* h) { return h->sigP32; }
  static const float* S(const pc_handle* h) { return h->S32; }
  static const float* lamK(const pc_handle* h) { return h->lamK32; }
  static const float* rmass(const pc_handle* h) { return h->rmass32; }
  static const float2* fst_tw(const pc_handle* h) { return h->fst_tw32; }
};

template <typename Tc>
static const CoarseLevels<Tc>& coarse_of(const pc_handle* h);
template <>
const CoarseLevels<float>& coarse_of<float>(const pc_handle* h) { return h->coarse32; }
template <>
const CoarseLevels<double>& coarse_of<double>(const pc_handle* h) { return h->coarse64; }

// step 2: every plane of lv[0].r solved into lv[0].u (iterates stored as TU)
template <typename Tc, typename TU>
static cudaError_t spatial_solve(pc_handle* h, Launch& L, int nplanes = 0,
                                 const typename Cx<Tc>::t* sig_override = nullptr, bool complete = false) {
  // nplanes / sig_override: solve only the first planes with other shifts; complete:
  // also apply the finest correction that the inverse time FFT otherwise adds
  typedef typename Cx<Tc>::t C;
  const int P = nplanes > 0 ? nplanes : h->planes;
  const C* sig = sig_override ? sig_override : Tables<Tc>::sig(h);
  cudaError_t e;
  if constexpr (std::is_same<TU, C>::value) {
    if (h->spatial == PC_SPATIAL_FST && Tables<Tc>::fst_tw(h) && fst_fast_supported<Tc>(h->m1)) {
      // fast transforms: forward along x1 (.. x_{d-1}), the last axis fused with the
      // divide, inverse back down to x1
      const Grid g = grid_of(h, 0);
      const C* tw = Tables<Tc>::fst_tw(h);
      C* tmp = (C*)h->fst_tmp;
      const int last = h->dim - 1;
      for (int ax = 0; ax < last; ++ax)
        if ((e = launch_fst_fast<Tc>(L, g, P, ax, false, tw, nullptr, nullptr, nullptr, ax == 0 ? (const C*)h->lv[0].r : tmp,
                                     tmp)) != cudaSuccess)
          return e;
      if ((e = launch_fst_fast<Tc>(L, g, P, last, true, tw, Tables<Tc>::lamK(h), Tables<Tc>::rmass(h), sig, tmp,
                                   last == 0 ? (C*)h->lv[0].u : tmp)) != cudaSuccess)
        return e;
      for (int ax = last - 1; ax >= 0; --ax)
        if ((e = launch_fst_fast<Tc>(L, g, P, ax, false, tw, nullptr, nullptr, nullptr, tmp,
                                     ax == 0 ? (C*)h->lv[0].u : tmp)) != cudaSuccess)
          return e;
      return cudaSuccess;
    }
    if (h->spatial == PC_SPATIAL_FST) {
      const Grid g = grid_of(h, 0);
      C* bufs[2] = {(C*)h->lv[0].r, (C*)h->fst_tmp};
      int cur = 0;
      for (int ax = 0; ax < h->dim; ++ax) {
        if ((e = launch_fst_axis<Tc>(L, g, P, ax, Tables<Tc>::S(h), bufs[cur], bufs[1 - cur])) != cudaSuccess) return e;
        cur = 1 - cur;
      }
      if ((e = launch_fst_divide<Tc>(L, g, P, Tables<Tc>::lamK(h), Tables<Tc>::rmass(h), sig, bufs[cur])) != cudaSuccess) return e;
      for (int ax = h->dim - 1; ax >= 0; --ax) {
        C* dst = ax == 0 ? (C*)h->lv[0].u : bufs[1 - cur];
        if ((e = launch_fst_axis<Tc>(L, g, P, ax, Tables<Tc>::S(h), bufs[cur], dst)) != cudaSuccess) return e;
        cur = 1 - cur;
      }
      return cudaSuccess;
    }
  }
  if (h->fevar) {
    if constexpr (std::is_same<TU, C>::value) return fevar_spatial<Tc>(h, L, P, sig);
    return cudaErrorNotSupported;
  }
  // multigrid V(1,0): per-level kernels on the fine levels, one fused kernel for the rest
  const int nl = (int)h->lv.size();
  const int l0 = h->coarse_l0;
  if (h->lex) {
    // smoother in the natural order: per-level kernels on every level, explicit residuals,
    // the one-point level solved exactly, every prolongation here
    for (int l = 0; l + 1 < nl; ++l) {
      const LevelBuf& Lb = h->lv[l];
      Stencil<Tc> st{lvw<Tc>(Lb), lvd<Tc>(Lb)};
      const Grid g = grid_of(h, l);
      if ((e = launch_mg_smooth_lex<Tc, TU>(L, g, P, st, sig, (const C*)Lb.r, (TU*)Lb.u)) != cudaSuccess) return e;
      if ((e = launch_mg_resid_restrict<Tc, TU>(L, g, P, st, sig, (const C*)Lb.r, (const TU*)Lb.u, (C*)Lb.res,
                                                (C*)h->lv[l + 1].r, false)) != cudaSuccess)
        return e;
    }
    if ((e = launch_mg_coarsest<Tc, TU>(L, P, lvd<Tc>(h->lv[nl - 1]), sig, (const C*)h->lv[nl - 1].r,
                                        (TU*)h->lv[nl - 1].u)) != cudaSuccess)
      return e;
    for (int l = nl - 2; l >= 0; --l)
      if ((e = launch_mg_prolong<Tc, TU>(L, grid_of(h, l), P, (const TU*)h->lv[l + 1].u, (TU*)h->lv[l].u)) !=
          cudaSuccess)
        return e;
    return cudaSuccess;
  }
  for (int l = 0; l < l0; ++l) {
    const LevelBuf& Lb = h->lv[l];
    Stencil<Tc> st{lvw<Tc>(Lb), lvd<Tc>(Lb)};
    const Grid g = grid_of(h, l);
    if (g.dim == 2) {
      if ((e = launch_mg_down<Tc, TU>(L, g, P, st, sig, (const C*)Lb.r, (TU*)Lb.u, (C*)h->lv[l + 1].r, 0, 0,
                                      Lb.w4)) != cudaSuccess)
        return e;
      continue;
    }
    if ((e = launch_mg_smooth<Tc, TU>(L, g, P, st, sig, (const C*)Lb.r, (TU*)Lb.u)) != cudaSuccess) return e;
    if ((e = launch_mg_resid_restrict<Tc, TU>(L, g, P, st, sig, (const C*)Lb.r, (const TU*)Lb.u, (C*)Lb.res,
                                              (C*)h->lv[l + 1].r)) != cudaSuccess)
      return e;
  }
  {
    const CoarseLevels<Tc>& cl = coarse_of<Tc>(h);
    bool done = false;
    if constexpr (std::is_same<Tc, float>::value && std::is_same<TU, float2>::value) {
      if (h->tail2) {
        if ((e = launch_mg_tail2(L, P, cl, sig, (const C*)h->lv[l0].r, (C*)h->lv[l0].u)) != cudaSuccess) return e;
        done = true;
      }
    }
    if (!done && (e = launch_mg_coarse_cycle<Tc, TU>(L, h->dim, P, cl, sig, (const C*)h->lv[l0].r,
                                                     (TU*)h->lv[l0].u)) != cudaSuccess)
      return e;
  }
  // in 2D the finest level's correction is added by the inverse time transform
  // (fine_correction); in 3D (eight coarse parents per point) by the prolongation kernel
  for (int l = l0 - 1; l >= (h->dim == 2 && !complete ? 1 : 0); --l) {
    if ((e = launch_mg_prolong<Tc, TU>(L, grid_of(h, l), P, (const TU*)h->lv[l + 1].u, (TU*)h->lv[l].u)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// correction u_0 += P u_1 still owed by spatial_solve (multigrid with at least one fine level)
template <typename TU>
static FineCorrection<TU> fine_correction(const pc_handle* h) {
  FineCorrection<TU> fc;
  if (h->spatial == PC_SPATIAL_FST || h->lex || h->fevar || h->coarse_l0 < 1 || h->dim != 2) return fc;
  const Grid g0 = grid_of(h, 0), g1 = grid_of(h, 1);
  fc.ec = (const TU*)h->lv[1].u;
  fc.dim = h->dim;
  fc.mf = g0.m;
  fc.mc = g1.m;
  fc.npc = g1.np;
  return fc;
}

// w = P^{-1} v; with jdev != nullptr the output is w + j*stride and, when index_input,
// the input v + j*stride (an FP32 input is the single rounded copy of the basis vector)
// w = P^{-1} v for the ideal RBD preconditioner of Eq. matrix_P: n sequential
// steps, each one spatial solve of two planes with the real shift 1 + alpha (half 2
// forward in time, half 1 backward), then the rotation [[I, -I], [I, I]]
template <typename Tc, typename TU, typename Tout, typename Tin>
static cudaError_t precond_ideal_t(pc_handle* h, Launch& L, const Tin* v, Tout* w) {
  typedef typename Cx<Tc>::t C;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j <= h->n; ++j) {
    if ((e = launch_ideal_step<Tc, TU, Tin, Tout>(L, v, (const TU*)h->lv[0].u, (C*)h->lv[0].r, w, h->ms, h->n, j)) !=
        cudaSuccess)
      return e;
    if (j == h->n) break;
    if ((e = spatial_solve<Tc, TU>(h, L, 2, Tables<Tc>::sigP(h), true)) != cudaSuccess) return e;
  }
  return launch_rbd_butterfly<Tout>(L, w, (int64_t)h->n * h->ms);
}

// (in_stride, when nonzero, indexes the input instead of stride: the hi planes of a
// double-float basis lie 2 U apart)
template <typename Tc, typename TU, typename Tout, typename Tin = double>
static cudaError_t precond_t(pc_handle* h, Launch& L, const Tin* v, Tout* w, size_t stride = 0,
                             const int* jdev = nullptr, bool index_input = true, size_t in_stride = 0) {
  typedef typename Cx<Tc>::t C;
  if (h->precond_kind == PC_PRECOND_IDEAL_RBD) {
    if (stride != 0 || jdev != nullptr) return cudaErrorNotSupported;  // graph solves reject it first
    return precond_ideal_t<Tc, TU, Tout, Tin>(h, L, v, w);
  }
  cudaError_t e = launch_tfft_forward<Tc>(L, h->ms, h->n, v, Tables<Tc>::dpow(h), Tables<Tc>::dinv(h),
                                          Tables<Tc>::tw(h), (C*)h->lv[0].r,
                                          index_input ? (in_stride ? in_stride : stride) : 0,
                                          index_input ? jdev : nullptr);
  if (e != cudaSuccess) return e;
  if ((e = spatial_solve<Tc, TU>(h, L)) != cudaSuccess) return e;
  return launch_tfft_inverse<Tc, TU, Tout>(L, h->ms, h->n, (const TU*)h->lv[0].u, Tables<Tc>::dpow(h),
                                           Tables<Tc>::dinv(h), Tables<Tc>::tw(h), w, stride, jdev,
                                           fine_correction<TU>(h));
}

// FP32 preconditioner into Tout, with the handle's iterate storage
template <typename Tout, typename Tin = double>
static cudaError_t precond32(pc_handle* h, Launch& L, const Tin* v, Tout* w, size_t stride = 0,
                             const int* jdev = nullptr, bool index_input = true, size_t in_stride = 0) {
  return h->bf16s ? precond_t<float, __nv_bfloat162, Tout, Tin>(h, L, v, w, stride, jdev, index_input, in_stride)
                  : precond_t<float, float2, Tout, Tin>(h, L, v, w, stride, jdev, index_input, in_stride);
}

// Arnoldi precision of flexible GMRES with the FP32 preconditioner: a double-float
// basis (the default) or an FP64 one; strict: FP64 products everywhere, including the
// re-orthogonalisation pass and the inner matvec of the FP32 basis
static bool arnoldi_df(const pc_handle* h) {
  return h->fp32 && (h->arnoldi == PC_ARNOLDI_AUTO || h->arnoldi == PC_ARNOLDI_DOUBLE_FLOAT);
}
static bool arnoldi_strict(const pc_handle* h) { return h->arnoldi == PC_ARNOLDI_FP64_STRICT; }

// w (FP64) = P^{-1} v in the handle's precision
static cudaError_t precond64(pc_handle* h, Launch& L, const double* v, double* w) {
  return h->fp32 ? precond32<double>(h, L, v, w) : precond_t<double, double2, double>(h, L, v, w);
}

static cudaError_t matvec_any(pc_handle* h, Launch& L, const void* x, bool x_f32, double* y, bool transpose) {
  Stencil<double> st{h->lv[0].w64, h->lv[0].d64};
  const Grid g = grid_of(h, 0);
  if (h->fevar) {
    const double h2 = h->h * h->h;
    if (h->dim == 3)
      return x_f32 ? launch_matvec_fevar3<float>(L, h->m1, h->n, h->h, h->alpha, h->tau, h->lv[0].e64,
                                                 (const float*)x, y, transpose)
                   : launch_matvec_fevar3<double>(L, h->m1, h->n, h->h, h->alpha, h->tau, h->lv[0].e64,
                                                  (const double*)x, y, transpose);
    if (x_f32)
      return launch_matvec_fevar<float>(L, h->m1, h->n, h2, h->alpha, h->tau, h->lv[0].e64, (const float*)x, y,
                                        transpose);
    return launch_matvec_fevar<double>(L, h->m1, h->n, h2, h->alpha, h->tau, h->lv[0].e64, (const double*)x, y,
                                       transpose);
  }
  if (h->fe) {
    if (x_f32) return launch_matvec_fe<float>(L, g, h->n, h->alpha, h->fes, h->tau, (const float*)x, y, transpose);
    return launch_matvec_fe<double>(L, g, h->n, h->alpha, h->fes, h->tau, (const double*)x, y, transpose);
  }
  if (x_f32) return launch_matvec<float>(L, g, h->n, st, h->alpha, (const float*)x, y, transpose);
  return launch_matvec<double>(L, g, h->n, st, h->alpha, (const double*)x, y, transpose);
}

// y = A z for the preconditioned basis vector z of flexible GMRES (FP32 in the
// mixed modes: double-float arithmetic for finite differences, FP64 for elements);
// with jdev: z += (*jdev) zs, y += (*jdev + 1) ys
static cudaError_t matvec_basis(pc_handle* h, Launch& L, const void* z, double* y, size_t zs = 0, size_t ys = 0,
                                const int* jdev = nullptr) {
  const Grid g = grid_of(h, 0);
  if (h->fevar && h->dim == 3)
    return h->fp32 ? launch_matvec_fevar3<float>(L, h->m1, h->n, h->h, h->alpha, h->tau, h->lv[0].e64,
                                                 (const float*)z, y, false, zs, ys, jdev)
                   : launch_matvec_fevar3<double>(L, h->m1, h->n, h->h, h->alpha, h->tau, h->lv[0].e64,
                                                  (const double*)z, y, false, zs, ys, jdev);
  if (h->fevar)
    return h->fp32 ? launch_matvec_fevar<float>(L, h->m1, h->n, h->h * h->h, h->alpha, h->tau, h->lv[0].e64,
                                                (const float*)z, y, false, zs, ys, jdev)
                   : launch_matvec_fevar<double>(L, h->m1, h->n, h->h * h->h, h->alpha, h->tau, h->lv[0].e64,
                                                 (const double*)z, y, false, zs, ys, jdev);
  if (h->fe)
    return h->fp32 ? launch_matvec_fe<float>(L, g, h->n, h->alpha, h->fes, h->tau, (const float*)z, y, false, zs, ys,
                                             jdev)
                   : launch_matvec_fe<double>(L, g, h->n, h->alpha, h->fes, h->tau, (const double*)z, y, false, zs,
                                              ys, jdev);
  if (h->fp32 && arnoldi_strict(h))
    return launch_matvec<float>(L, g, h->n, Stencil<double>{h->lv[0].w64, h->lv[0].d64}, h->alpha, (const float*)z,
                                y, false, zs, ys, jdev);
  if (h->fp32) return launch_matvec_df(L, g, h->n, h->wdf, h->ddf, h->alpha_df, (const float*)z, y, zs, ys, jdev);
  return launch_matvec<double>(L, g, h->n, Stencil<double>{h->lv[0].w64, h->lv[0].d64}, h->alpha,
                               (const double*)z, y, false, zs, ys, jdev);
}

// ---------------------------------------------------------------------------
// public operators
// ---------------------------------------------------------------------------
extern "C" int pc_matvec(pc_handle* h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return fail(PC_ERR_ARG, "pc_matvec: null argument");
  if (x == y) return fail(PC_ERR_ARG, "pc_matvec: x and y must not overlap");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  cudaError_t e = matvec_any(h, L, x, false, y, false);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_matvec");
}

extern "C" int pc_matvec_f32(pc_handle* h, const float* x, double* y, void* stream) {
  if (!h || !x || !y) return fail(PC_ERR_ARG, "pc_matvec_f32: null argument");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  cudaError_t e = h->fe ? matvec_any(h, L, x, true, y, false)
                        : launch_matvec_df(L, grid_of(h, 0), h->n, h->wdf, h->ddf, h->alpha_df, x, y);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_matvec_f32");
}

extern "C" int pc_matvec_transpose(pc_handle* h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return fail(PC_ERR_ARG, "pc_matvec_transpose: null argument");
  if (x == y) return fail(PC_ERR_ARG, "pc_matvec_transpose: x and y must not overlap");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  cudaError_t e = matvec_any(h, L, x, false, y, true);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_matvec_transpose");
}

extern "C" int pc_apply_precond(pc_handle* h, const double* v, double* w, void* stream) {
  if (!h || !v || !w) return fail(PC_ERR_ARG, "pc_apply_precond: null argument");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  cudaError_t e = precond64(h, L, v, w);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_apply_precond");
}

extern "C" int pc_build_rhs(pc_handle* h, const double* f, const double* g, const double* y0, double* b,
                            void* stream) {
  if (!h || !g || !b) return fail(PC_ERR_ARG, "pc_build_rhs: null g or b");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  cudaError_t e;
  if (!h->fe) {
    e = launch_build_rhs(L, h->ms, h->n, h->tau, h->sqrtg, f, g, y0, b);
  } else {
    // b = [tau (I(x)M) g; -sqrt(gamma) (tau (I(x)M) f + M y0 e_1)]
    const Grid gr = grid_of(h, 0);
    const size_t half = (size_t)h->n * h->ms;
    e = launch_fe_apply(L, gr, h->n, h->tau * h->fes.wM, 0.0, g, 0.0, b);
    if (e == cudaSuccess)
      e = f ? launch_fe_apply(L, gr, h->n, -h->sqrtg * h->tau * h->fes.wM, 0.0, f, 0.0, b + half)
            : cudaMemsetAsync(b + half, 0, half * sizeof(double), L.stream);
    if (e == cudaSuccess && y0) e = launch_fe_apply(L, gr, 1, -h->sqrtg * h->fes.wM, 0.0, y0, 1.0, b + half);
  }
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_build_rhs");
}

extern "C" int pc_grad_log_a(pc_handle* h, const double* x, const double* lam, double* grad, void* stream) {
  if (!h || !x || !lam || !grad) return fail(PC_ERR_ARG, "pc_grad_log_a: null argument");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  if (h->fe) {
    // -tau a_P / 2^d sum over P's elements and the time blocks of (lam1^T K_e x2 - lam2^T K_e x1)
    cudaError_t e =
        h->dim == 3
            ? launch_fevar3_grad(L, h->m1, h->n, h->h, h->tau, h->a_int, x, lam, h->fe_gpart, kFeGradChunks, grad)
            : launch_fevar_grad(L, h->m1, h->n, h->tau, h->a_int, x, lam, h->fe_gpart, kFeGradChunks, grad);
    return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_grad_log_a");
  }
  // -tau * a_P / (2 h^2) * sum_j sum_faces [...]
  const double scale = -h->tau * 0.5 / (h->h * h->h);
  cudaError_t e =
      launch_grad_chunked(L, grid_of(h, 0), h->n, scale, h->a_int, x, lam, h->grad_partial, h->grad_tj, grad);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_grad_log_a");
}

extern "C" int pc_grad_g(pc_handle* h, const double* lam, double* grad_g, void* stream) {
  if (!h || !lam || !grad_g) return fail(PC_ERR_ARG, "pc_grad_g: null argument");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  if (h->fe) {  // b1_j = tau M g_j: the gradient is tau M lam1_j
    cudaError_t e = launch_fe_apply(L, grid_of(h, 0), h->n, h->tau * h->fes.wM, 0.0, lam, 0.0, grad_g);
    return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_grad_g");
  }
  cudaError_t e = launch_grad_g(L, lam, (int64_t)h->n * h->ms, h->tau, grad_g);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_grad_g");
}

// c = h^d tau, the quadrature weight of the discrete objective
static double objective_weight(const pc_handle* h) { return std::pow(h->h, h->dim) * h->tau; }

extern "C" int pc_objective(pc_handle* h, const double* x, const double* g, double* J, void* stream) {
  if (!h || !x || !g || !J) return fail(PC_ERR_ARG, "pc_objective: null argument");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  if (h->fe) {  // tau [1/2 sum e^T M e + 1/(2 gamma) sum p^T M p]
    cudaError_t e = h->dim == 3 ? launch_fevar3_objective(L, h->m1, h->n, h->h, h->tau, h->prm.gamma, x, g,
                                                          h->partial, h->nblocks * (h->cap + 2), J)
                                : launch_fevar_objective(L, h->m1, h->n, h->h * h->h, h->tau, h->prm.gamma, x, g,
                                                         h->partial, h->nblocks * (h->cap + 2), J);
    return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_objective");
  }
  cudaError_t e = launch_objective(L, x, g, (int64_t)h->n * h->ms, h->prm.gamma, objective_weight(h), h->partial,
                                   h->nblocks * (h->cap + 2), J);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_objective");
}

extern "C" int pc_objective_grad(pc_handle* h, const double* x, const double* g, const double* gJ, double* gx,
                                 double* gg, void* stream) {
  if (!h || !x || !g || (!gx && !gg)) return fail(PC_ERR_ARG, "pc_objective_grad: null argument");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  if (h->fe) {
    cudaError_t e =
        h->dim == 3 ? launch_fevar3_objective_grad(L, h->m1, h->n, h->h, h->tau, h->prm.gamma, x, g, gJ, gx, gg)
                    : launch_fevar_objective_grad(L, h->m1, h->n, h->h * h->h, h->tau, h->prm.gamma, x, g, gJ, gx, gg);
    return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_objective_grad");
  }
  cudaError_t e = launch_objective_grad(L, x, g, (int64_t)h->n * h->ms, h->prm.gamma, objective_weight(h), gJ, gx, gg);
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_objective_grad");
}

// ---------------------------------------------------------------------------
// GMRES (Section 3: zero initial guess, relative tolerance; Lemma 2.1)
// ---------------------------------------------------------------------------
// copy n doubles (and optionally one int, stored as a double after them) from device
// memory into the mapped host buffer
__global__ void to_mapped_kernel(const double* __restrict__ src, int n, const int* __restrict__ isrc,
                                 double* __restrict__ dst) {
  const int t = threadIdx.x;
  if (t < n) dst[t] = src[t];
  if (t == 0 && isrc) dst[n] = (double)isrc[0];
}

// host[off .. off+n) = src[0 .. n) (+ host[off+n] = *isrc), visible to the host after `st`
// is synchronised
static int fetch_scalars(pc_handle* h, cudaStream_t st, const double* src, int n, int off,
                         const int* isrc = nullptr) {
  Launch L{st, &h->prof, &h->tiles};
  L.begin(KC_REDUCE);
  to_mapped_kernel<<<1, 32, 0, st>>>(src, n, isrc, h->host_dev + off);
  PC_CUDA(L.end(KC_REDUCE, 8.0 * (n + (isrc ? 1 : 0)), 0.0));
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

// host[0] = est, host[1] = ref, host[8] = re-orthogonalisation flag of the last step,
// host[9] = error word of the bounded waits (scal[10]; nonzero: a wait ran out)
static int read_scalars(pc_handle* h, cudaStream_t st, double* est, double* ref, bool* reorth = nullptr) {
  if (int rc = fetch_scalars(h, st, h->scal + 1, 10, 0)) return rc;
  if (h->host[9] != 0.0) return fail(PC_ERR_TIMEOUT, "a bounded device wait ran out (streamed basis copy)");
  if (est) *est = h->host[0];
  if (ref) *ref = h->host[1];
  if (reorth) *reorth = h->host[8] != 0.0;
  return PC_OK;
}

// the same scalars as read_scalars, in two halves: post_scalars queues their copy into
// mapped host memory and records the handle's event; take_scalars waits for that event
// only (work queued after it keeps running) and reads them
static int post_scalars(pc_handle* h, cudaStream_t st) {
  Launch L{st, &h->prof, &h->tiles};
  L.begin(KC_REDUCE);
  to_mapped_kernel<<<1, 32, 0, st>>>(h->scal + 1, 10, nullptr, h->host_dev);
  PC_CUDA(L.end(KC_REDUCE, 80.0, 0.0));
  PC_CUDA(cudaEventRecord(h->scal_ev, st));
  return PC_OK;
}

static int take_scalars(pc_handle* h, double* est, double* ref, bool* reorth) {
  PC_CUDA(cudaEventSynchronize(h->scal_ev));
  if (h->host[9] != 0.0) return fail(PC_ERR_TIMEOUT, "a bounded device wait ran out (streamed basis copy)");
  if (est) *est = h->host[0];
  if (ref) *ref = h->host[1];
  if (reorth) *reorth = h->host[8] != 0.0;
  return PC_OK;
}

static int gmres_impl(pc_handle* h, const double* b, double* x, double rtol, int maxit, int mode, int* iters,
                      double* relres, cudaStream_t st) {
  if (!h || !b || !x) return fail(PC_ERR_ARG, "gmres: null argument");
  if (!(rtol > 0)) return fail(PC_ERR_ARG, "gmres: rtol must be > 0");
  if (maxit < 1 || maxit > h->cap) return fail(PC_ERR_ARG, "gmres: maxit must be in [1, max_iter]");
  if (mode != PC_GMRES_RIGHT && mode != PC_GMRES_LEFT) return fail(PC_ERR_ARG, "gmres: unknown mode");
  if (mode == PC_GMRES_LEFT && h->fp32) return fail(PC_ERR_ARG, "gmres: LEFT mode needs the FP64 preconditioner");
  Launch L{st, &h->prof, &h->tiles};
  h->last_k = -1;
  const size_t U = h->U;
  const int ldh = h->cap + 1;
  double* nrm2 = h->scal + 0;
  double* est = h->scal + 1;
  double* ref = h->scal + 2;
  double* V = h->V;
  const ArnoldiScalars AS{h->scal + 4, h->scal + 5, h->scal + 6, h->scal + 7, h->scal + 8, h->scal + 9};
  cudaError_t e;
#define GM_CUDA(...)                                   \
  do {                                                 \
    if ((e = (__VA_ARGS__)) != cudaSuccess) return cuda_fail(e, #__VA_ARGS__); \
  } while (0)

  // is x0 zero?  (one norm + readback)
  GM_CUDA(launch_norm2(L, x, U, h->partial, h->scal + 3));
  if (int rc = fetch_scalars(h, st, h->scal + 3, 1, 2)) return rc;
  PC_CUDA(cudaStreamSynchronize(st));
  const bool x0_zero = h->host[2] == 0.0;

  // double-float basis: two FP32 planes per vector, tiled layout (flexible GMRES only)
  const bool df = mode == PC_GMRES_RIGHT && arnoldi_df(h);
  const bool lp_reorth = !arnoldi_strict(h);
  float* Vf = reinterpret_cast<float*>(V);
  const int nvt = h->cap + 1;  // vectors per tile block of the double-float layout
  double* werr = h->scal + 10;
  PC_CUDA(cudaMemsetAsync(werr, 0, sizeof(double), st));
  const double* r0 = V;  // r0 before normalisation (double-float basis: b itself or tbuf)

  // reference norm and r0 (stored unnormalised in V_0)
  if (mode == PC_GMRES_RIGHT) {
    GM_CUDA(launch_norm2(L, b, U, h->partial, nrm2));
    GM_CUDA(launch_arnoldi_start(L, h->gvec, nrm2, est, ref, 1));  // ref = ||b||
    double* r0w = df ? h->tbuf : V;
    if (x0_zero) {
      if (df)
        r0 = b;
      else
        PC_CUDA(cudaMemcpyAsync(V, b, U * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      GM_CUDA(matvec_any(h, L, x, false, h->wbuf, false));
      PC_CUDA(cudaMemcpyAsync(r0w, b, U * sizeof(double), cudaMemcpyDeviceToDevice, st));
      GM_CUDA(launch_axpby<double>(L, -1.0, h->wbuf, 1.0, r0w, U));
      r0 = r0w;
    }
    GM_CUDA(launch_norm2(L, r0, U, h->partial, nrm2));
    GM_CUDA(launch_arnoldi_start(L, h->gvec, nrm2, est, ref, 0));
  } else {
    GM_CUDA(precond64(h, L, b, V));  // P^{-1} b
    GM_CUDA(launch_norm2(L, V, U, h->partial, nrm2));
    GM_CUDA(launch_arnoldi_start(L, h->gvec, nrm2, est, ref, 1));  // ref = ||P^{-1} b||
    if (!x0_zero) {
      GM_CUDA(matvec_any(h, L, x, false, h->wbuf, false));
      PC_CUDA(cudaMemcpyAsync(h->tbuf, b, U * sizeof(double), cudaMemcpyDeviceToDevice, st));
      GM_CUDA(launch_axpby<double>(L, -1.0, h->wbuf, 1.0, h->tbuf, U));
      GM_CUDA(precond64(h, L, h->tbuf, V));
      GM_CUDA(launch_norm2(L, V, U, h->partial, nrm2));
      GM_CUDA(launch_arnoldi_start(L, h->gvec, nrm2, est, ref, 0));
    }
  }
  double est_h = 0, ref_h = 0;
  if (int rc = read_scalars(h, st, &est_h, &ref_h)) return rc;
  h->last_res0 = ref_h == 0.0 ? 0.0 : est_h;
  h->last_k = 0;
  if (ref_h == 0.0) {
    // b == 0 (or P^{-1}b == 0): the solution is x = 0
    PC_CUDA(cudaMemsetAsync(x, 0, U * sizeof(double), st));
    PC_CUDA(cudaStreamSynchronize(st));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return PC_OK;
  }
  if (!std::isfinite(est_h) || !std::isfinite(ref_h)) return fail(PC_ERR_BREAKDOWN, "gmres: non-finite initial residual");
  if (est_h <= rtol) {
    if (iters) *iters = 0;
    if (relres) *relres = est_h;
    return PC_OK;
  }
  // flexible GMRES with the FP32 preconditioner reads the FP32 rounding of each new
  // basis vector, written by the kernels that finish it (scale / update)
  float* vf = (mode == PC_GMRES_RIGHT && h->fp32) ? h->vf32 : nullptr;
  if (df)
    GM_CUDA(launch_split_scale(L, r0, Vf, nvt, vf, U, nrm2));
  else
    GM_CUDA(launch_scale_by_inv_norm(L, V, U, nrm2, nullptr, vf));

  // Iteration j = front (z_j = P^{-1} v_j and w = A z_j, or the left-preconditioned
  // pair; it needs only v_j) + back (Arnoldi passes, Givens, the estimate copied to
  // mapped host memory behind an event, which the host waits for).  Queuing the next
  // front before that wait was tried: the GPU never idled long enough for it to pay
  // (0.0852 vs 0.0849 s per solve at 255^2 x 256), so the next front waits for the decision.
  auto front = [&](int j) -> cudaError_t {
    double* vj = V + (size_t)j * U;
    double* vn = V + (size_t)(j + 1) * U;
    cudaError_t e2;
    if (df) {
      // double-float basis: the preconditioner reads the FP32 rounding of v_j (vf32),
      // A z_j goes to wbuf (FP64)
      float* zj = (float*)h->Z + (size_t)j * U;
      if ((e2 = precond32<float, float>(h, L, vf, zj)) != cudaSuccess) return e2;
      return matvec_basis(h, L, zj, h->wbuf);
    }
    if (mode == PC_GMRES_RIGHT) {
      if (h->fp32) {
        float* zj = (float*)h->Z + (size_t)j * U;
        if ((e2 = precond32<float, float>(h, L, vf, zj)) != cudaSuccess) return e2;
        return matvec_basis(h, L, zj, vn);
      }
      double* zj = (double*)h->Z + (size_t)j * U;
      if ((e2 = precond_t<double, double2, double>(h, L, vj, zj)) != cudaSuccess) return e2;
      return matvec_any(h, L, zj, false, vn, false);
    }
    if ((e2 = matvec_any(h, L, vj, false, h->wbuf, false)) != cudaSuccess) return e2;
    return precond64(h, L, h->wbuf, vn);
  };
  int k = 0;
  bool converged = false;
  GM_CUDA(front(0));
  for (int j = 0; j < maxit; ++j) {
    double* vn = V + (size_t)(j + 1) * U;
    if (df) {
      // the update writes v_{j+1} and its FP32 rounding
      GM_CUDA(launch_multidot_df(L, Vf, nvt, j + 1, h->wbuf, U, h->partial, h->hcol, AS.ww, nullptr, werr));
      GM_CUDA(launch_arnoldi_prep(L, j + 1, h->hcol, AS));
      GM_CUDA(launch_update_df(L, Vf, nvt, j + 1, h->hcol, h->wbuf, vf, U, AS.inv, h->partial, AS.q, nullptr, werr));
      GM_CUDA(launch_arnoldi_check(L, AS));
      GM_CUDA(launch_multidot_df(L, Vf, nvt, j + 1, nullptr, U, h->partial, h->hcol + ldh, nullptr, AS.flag, werr));
      GM_CUDA(launch_update_df(L, Vf, nvt, j + 1, h->hcol + ldh, nullptr, vf, U, nullptr, h->partial, AS.rho2,
                               AS.flag, werr));
      GM_CUDA(launch_scale_df(L, Vf, nvt, j + 1, vf, U, AS.rho2, AS.flag));
    } else {
      // classical Gram-Schmidt with Pythagorean normalisation, re-orthogonalised only
      // when the check flags cancellation (the gated kernels then do the work)
      GM_CUDA(launch_multidot(L, V, U, j + 1, vn, U, h->partial, h->hcol, AS.ww, nullptr));
      GM_CUDA(launch_arnoldi_prep(L, j + 1, h->hcol, AS));
      GM_CUDA(launch_update(L, V, U, j + 1, h->hcol, vn, U, AS.inv, h->partial, AS.q, nullptr, vf));
      GM_CUDA(launch_arnoldi_check(L, AS));
      GM_CUDA(launch_multidot(L, V, U, j + 1, vn, U, h->partial, h->hcol + ldh, nullptr, AS.flag, lp_reorth));
      GM_CUDA(launch_update(L, V, U, j + 1, h->hcol + ldh, vn, U, nullptr, h->partial, AS.rho2, AS.flag, nullptr,
                            lp_reorth));
      GM_CUDA(launch_scale_by_inv_norm(L, vn, U, AS.rho2, AS.flag, vf));
    }
    GM_CUDA(launch_givens(L, j, ldh, h->H, h->cs, h->sn, h->gvec, h->hcol, h->hcol + ldh, AS, est, ref));
    if (int rc = post_scalars(h, st)) return rc;
    bool reorth = false;
    if (int rc = take_scalars(h, &est_h, nullptr, &reorth)) return rc;
    if (reorth) {  // book the second Gram-Schmidt pass that ran
      // double-float basis: hi planes read twice (4 B each), the new vector's planes read
      // three times and written twice; FP64 basis: 8 B per basis read, 6 vector passes
      h->prof.bytes[KC_REORTH] += df ? 4.0 * U * (2.0 * (j + 1) + 11.0) : 8.0 * U * (2.0 * (j + 1) + 6.0);
      h->prof.flops[KC_REORTH] += 4.0 * U * (j + 1);
      h->prof.launches[KC_REORTH]++;
    }
    k = j + 1;
    h->last_k = k;
    if (!std::isfinite(est_h)) return fail(PC_ERR_BREAKDOWN, "gmres: non-finite residual estimate");
    if (est_h <= rtol) {
      converged = true;
      break;
    }
    if (j + 1 < maxit) GM_CUDA(front(j + 1));
  }
  GM_CUDA(launch_backsolve(L, k, ldh, h->H, h->gvec, h->ycoef));
  if (mode == PC_GMRES_RIGHT) {
    if (h->fp32)
      GM_CUDA(launch_xupdate<float>(L, (const float*)h->Z, U, k, h->ycoef, x, U));
    else
      GM_CUDA(launch_xupdate<double>(L, (const double*)h->Z, U, k, h->ycoef, x, U));
    // true residual ||b - A x|| / ||b||
    GM_CUDA(matvec_any(h, L, x, false, h->wbuf, false));
    GM_CUDA(launch_axpby<double>(L, 1.0, b, -1.0, h->wbuf, U));
    GM_CUDA(launch_norm2(L, h->wbuf, U, h->partial, h->scal + 3));
    if (int rc = fetch_scalars(h, st, h->scal + 3, 1, 2)) return rc;
    PC_CUDA(cudaStreamSynchronize(st));
    est_h = std::sqrt(h->host[2]) / ref_h;
  } else {
    GM_CUDA(launch_xupdate<double>(L, V, U, k, h->ycoef, x, U));
    PC_CUDA(cudaStreamSynchronize(st));
  }
#undef GM_CUDA
  if (iters) *iters = k;
  if (relres) *relres = est_h;
  if (!std::isfinite(est_h)) return fail(PC_ERR_BREAKDOWN, "gmres: non-finite final residual");
  if (!converged) return fail(PC_ERR_NOT_CONVERGED, "gmres: maxit reached before rtol");
  return PC_OK;
}

// residual estimates of the last solve: |g_{i}| / ref = res_0 * prod_{q < i} |s_q|, with
// the sines s_q of the Givens rotations (the rotated right-hand side itself is
// overwritten by later rotations)
extern "C" int pc_residual_history(pc_handle* h, double* out, int cap, int* count, void* stream) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return fail(PC_ERR_ARG, "pc_residual_history: bad argument");
  *count = 0;
  if (h->last_k < 0) return PC_OK;
  const int k = h->last_k;
  const int nout = std::min(cap, k + 1);
  *count = nout;
  if (nout == 0) return PC_OK;
  out[0] = h->last_res0;
  if (nout == 1) return PC_OK;
  std::vector<double> sn((size_t)nout - 1);
  cudaStream_t st = (cudaStream_t)stream;
  PC_CUDA(cudaMemcpyAsync(sn.data(), h->sn, sn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  for (int i = 1; i < nout; ++i) out[i] = out[i - 1] * std::fabs(sn[(size_t)i - 1]);
  return PC_OK;
}

// Right-preconditioned GMRES stops on the least-squares estimate of ||b - A x||; with
// an FP32 preconditioner and a double-float basis the true residual formed at exit can
// sit just above that estimate.  When it misses rtol and iterations remain, the solve
// continues from the current x in a fresh Krylov space (r0 = b - A x, the remaining
// iteration budget) until the true residual meets rtol or the budget is spent; `done`
// holds the iterations already spent (a graph solve's), and *iters counts all of them.
static int gmres_confirm(pc_handle* h, const double* b, double* x, double rtol, int maxit, int mode, int rc,
                         int done, double rr, int* iters, double* relres, cudaStream_t st) {
  while (rc == PC_OK && mode == PC_GMRES_RIGHT && rr > rtol && done < maxit) {
    int k = 0;
    rc = gmres_impl(h, b, x, rtol, maxit - done, mode, &k, &rr, st);
    done += k;
    if (k == 0) break;
  }
  if (iters) *iters = done;
  if (relres) *relres = rr;
  if (rc == PC_OK && mode == PC_GMRES_RIGHT && rr > rtol)
    return fail(PC_ERR_NOT_CONVERGED, "gmres: true residual above rtol after maxit iterations");
  return rc;
}

extern "C" int pc_gmres_solve(pc_handle* h, const double* b, double* x, double rtol, int maxit, int mode, int* iters,
                              double* relres, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int k = 0;
  double rr = 0.0;
  const int rc = gmres_impl(h, b, x, rtol, maxit, mode, &k, &rr, st);
  if (rc != PC_OK && rc != PC_ERR_NOT_CONVERGED) {
    if (iters) *iters = k;
    if (relres) *relres = rr;
    return rc;
  }
  return gmres_confirm(h, b, x, rtol, maxit, mode, rc, k, rr, iters, relres, st);
}

extern "C" int pc_adjoint_solve(pc_handle* h, const double* c, double* lam, double rtol, int maxit, int mode,
                                int* iters, double* relres, void* stream) {
  if (!h || !c || !lam) return fail(PC_ERR_ARG, "pc_adjoint_solve: null argument");
  if (c == lam) return fail(PC_ERR_ARG, "pc_adjoint_solve: c and lam must not overlap");
  cudaStream_t st = (cudaStream_t)stream;
  Launch L{st, &h->prof, &h->tiles};
  const size_t half = h->U / 2;
  // A^T lam = c  <=>  A (S lam) = S c,  S = diag(I, -I)
  PC_CUDA(cudaMemcpyAsync(h->adjbuf, c, h->U * sizeof(double), cudaMemcpyDeviceToDevice, st));
  cudaError_t e = launch_axpby<double>(L, -1.0, h->adjbuf + half, 0.0, h->adjbuf + half, half);
  if (e != cudaSuccess) return cuda_fail(e, "pc_adjoint_solve");
  if ((e = launch_axpby<double>(L, -1.0, lam + half, 0.0, lam + half, half)) != cudaSuccess)
    return cuda_fail(e, "pc_adjoint_solve");
  int k = 0;
  double rr = 0.0;
  int rc = gmres_impl(h, h->adjbuf, lam, rtol, maxit, mode, &k, &rr, st);
  if (rc == PC_OK || rc == PC_ERR_NOT_CONVERGED)
    rc = gmres_confirm(h, h->adjbuf, lam, rtol, maxit, mode, rc, k, rr, iters, relres, st);
  if ((e = launch_axpby<double>(L, -1.0, lam + half, 0.0, lam + half, half)) != cudaSuccess)
    return cuda_fail(e, "pc_adjoint_solve");
  cudaError_t se = cudaStreamSynchronize(st);
  if (se != cudaSuccess) return cuda_fail(se, "pc_adjoint_solve");
  return rc;
}

// ---------------------------------------------------------------------------
// Graph-captured solve (right-preconditioned FGMRES, zero initial guess): the
// whole solve is one graph; the iteration is the body of a WHILE conditional
// node whose condition the loop-control kernel sets on the device, so no host
// round trip happens per iteration.  Every launch of the body reads the Arnoldi
// index from h->idx, so one captured iteration serves all of them.
// ---------------------------------------------------------------------------
#define GR_CUDA(...)                                                             \
  do {                                                                           \
    cudaError_t _e = (__VA_ARGS__);                                              \
    if (_e != cudaSuccess) return cuda_fail(_e, #__VA_ARGS__);                   \
  } while (0)

static int graph_supported(const pc_handle* h, int maxit) {
  if (maxit < 1 || maxit > h->cap) return fail(PC_ERR_ARG, "graph solve: maxit must be in [1, max_iter]");
  if (h->precond_kind != PC_PRECOND_EPS_CIRCULANT)
    return fail(PC_ERR_UNSUPPORTED, "graph solve: the eps-circulant preconditioner only");
  if (!is_pow2(h->n)) return fail(PC_ERR_UNSUPPORTED, "graph solve: n must be a power of two");
  const int nmax = h->fp32 ? 1024 : 256;
  if (h->n > nmax) return fail(PC_ERR_UNSUPPORTED, "graph solve: n too large for the register FFT");
  return PC_OK;
}

// x = 0, r0 = b, ref = ||b||, g0 = beta, v0 = b / beta, enter the loop iff est > rtol
static int enqueue_pre(pc_handle* h, Launch& L, const double* b, double* x, double rtol,
                       cudaGraphConditionalHandle hc) {
  const size_t U = h->U;
  double* nrm2 = h->scal + 0;
  GR_CUDA(cudaMemsetAsync(x, 0, U * sizeof(double), L.stream));
  GR_CUDA(launch_norm2(L, b, U, h->partial, nrm2));
  GR_CUDA(launch_arnoldi_start(L, h->gvec, nrm2, h->scal + 1, h->scal + 2, 1));
  if (arnoldi_df(h)) {
    GR_CUDA(cudaMemsetAsync(h->scal + 10, 0, sizeof(double), L.stream));
    GR_CUDA(launch_split_scale(L, b, reinterpret_cast<float*>(h->V), h->cap + 1, h->vf32, U, nrm2));
  } else {
    GR_CUDA(cudaMemcpyAsync(h->V, b, U * sizeof(double), cudaMemcpyDeviceToDevice, L.stream));
    GR_CUDA(launch_scale_by_inv_norm(L, h->V, U, nrm2, nullptr, h->fp32 ? h->vf32 : nullptr));
  }
  GR_CUDA(launch_loop_start(L, h->idx, h->idx + 1, h->scal + 1, rtol, hc));
  return PC_OK;
}

// one FGMRES iteration with device-resident index j = h->idx[0]
static int enqueue_body(pc_handle* h, Launch& L, double rtol, int maxit, cudaGraphConditionalHandle hc) {
  const size_t U = h->U;
  const int ldh = h->cap + 1;
  const int* j = h->idx;
  const ArnoldiScalars AS{h->scal + 4, h->scal + 5, h->scal + 6, h->scal + 7, h->scal + 8, h->scal + 9};
  if (arnoldi_df(h)) {
    // double-float basis (tiled layout): see gmres_impl
    float* Z = (float*)h->Z;
    float* Vf = reinterpret_cast<float*>(h->V);
    const int nvt = h->cap + 1;
    double* werr = h->scal + 10;
    GR_CUDA((precond32<float, float>(h, L, h->vf32, Z, U, j, false)));
    GR_CUDA(matvec_basis(h, L, Z, h->wbuf, U, 0, j));
    GR_CUDA(launch_multidot_df_dev(L, Vf, nvt, maxit, j, h->wbuf, U, h->partial, h->hcol, AS.ww, nullptr, werr));
    GR_CUDA(launch_arnoldi_prep_dev(L, j, h->hcol, AS));
    GR_CUDA(launch_update_df_dev(L, Vf, nvt, maxit, j, h->hcol, h->wbuf, h->vf32, U, AS.inv, h->partial, AS.q,
                                 nullptr, werr));
    GR_CUDA(launch_arnoldi_check(L, AS));
    GR_CUDA(launch_multidot_df_dev(L, Vf, nvt, maxit, j, nullptr, U, h->partial, h->hcol + ldh, nullptr, AS.flag,
                                   werr));
    GR_CUDA(launch_update_df_dev(L, Vf, nvt, maxit, j, h->hcol + ldh, nullptr, h->vf32, U, nullptr, h->partial,
                                 AS.rho2, AS.flag, werr));
    GR_CUDA(launch_scale_df_dev(L, Vf, nvt, j, h->vf32, U, AS.rho2, AS.flag));
    GR_CUDA(launch_givens_dev(L, j, ldh, h->H, h->cs, h->sn, h->gvec, h->hcol, h->hcol + ldh, AS, h->scal + 1,
                              h->scal + 2));
    GR_CUDA(launch_loop_control(L, h->idx, h->idx + 1, h->scal + 1, rtol, maxit, hc));
    return PC_OK;
  }
  const bool lp_reorth = !arnoldi_strict(h);
  if (h->fp32) {
    float* Z = (float*)h->Z;
    GR_CUDA((precond32<float, float>(h, L, h->vf32, Z, U, j, false)));
    GR_CUDA(matvec_basis(h, L, Z, h->V, U, U, j));
  } else {
    double* Z = (double*)h->Z;
    GR_CUDA((precond_t<double, double2, double>(h, L, h->V, Z, U, j)));
    GR_CUDA(matvec_basis(h, L, Z, h->V, U, U, j));
  }
  GR_CUDA(launch_multidot_dev(L, h->V, U, maxit, j, h->V, U, U, h->partial, h->hcol, AS.ww, nullptr));
  GR_CUDA(launch_arnoldi_prep_dev(L, j, h->hcol, AS));
  float* vf = h->fp32 ? h->vf32 : nullptr;
  GR_CUDA(launch_update_dev(L, h->V, U, maxit, j, h->hcol, h->V, U, U, AS.inv, h->partial, AS.q, nullptr, vf));
  GR_CUDA(launch_arnoldi_check(L, AS));
  GR_CUDA(launch_multidot_dev(L, h->V, U, maxit, j, h->V, U, U, h->partial, h->hcol + ldh, nullptr, AS.flag,
                              lp_reorth));
  GR_CUDA(launch_update_dev(L, h->V, U, maxit, j, h->hcol + ldh, h->V, U, U, nullptr, h->partial, AS.rho2, AS.flag,
                            nullptr, lp_reorth));
  GR_CUDA(launch_scale_dev(L, h->V, U, j, U, AS.rho2, AS.flag, vf));
  GR_CUDA(launch_givens_dev(L, j, ldh, h->H, h->cs, h->sn, h->gvec, h->hcol, h->hcol + ldh, AS, h->scal + 1,
                            h->scal + 2));
  GR_CUDA(launch_loop_control(L, h->idx, h->idx + 1, h->scal + 1, rtol, maxit, hc));
  return PC_OK;
}

// x = Z y (k = h->idx[1] columns), true residual ||b - A x||^2 -> scal[3]
static int enqueue_post(pc_handle* h, Launch& L, const double* b, double* x, int maxit) {
  const size_t U = h->U;
  const int ldh = h->cap + 1;
  GR_CUDA(launch_backsolve_dev(L, h->idx + 1, ldh, h->H, h->gvec, h->ycoef));
  if (h->fp32)
    GR_CUDA(launch_xupdate_dev<float>(L, (const float*)h->Z, U, maxit, h->idx + 1, h->ycoef, x, U));
  else
    GR_CUDA(launch_xupdate_dev<double>(L, (const double*)h->Z, U, maxit, h->idx + 1, h->ycoef, x, U));
  GR_CUDA(matvec_any(h, L, x, false, h->wbuf, false));
  GR_CUDA(launch_axpby<double>(L, 1.0, b, -1.0, h->wbuf, U));
  GR_CUDA(launch_norm2(L, h->wbuf, U, h->partial, h->scal + 3));
  return PC_OK;
}

// Enqueue one complete solve into `st`, which must be capturing; the loop body is
// captured on the handle's auxiliary stream into the conditional node's graph.
static int capture_solve(pc_handle* h, const double* b, double* x, double rtol, int maxit, cudaStream_t st) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t G = nullptr;
  GR_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &G, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !G) return fail(PC_ERR_CUDA, "capture_solve: stream is not capturing");
  cudaGraphConditionalHandle hc;
  GR_CUDA(cudaGraphConditionalHandleCreate(&hc, G, 0, cudaGraphCondAssignDefault));
  Launch L{st, nullptr, &h->tiles};
  int rc;
  if ((rc = enqueue_pre(h, L, b, x, rtol, hc))) return rc;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  GR_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  // cudaGraphNodeParams holds a union without a default constructor: zeroed storage
  alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
  std::memset(cp_storage, 0, sizeof(cp_storage));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  GR_CUDA(cudaGraphAddNode(&cnode, G, dv.data(), nullptr, nd, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  GR_CUDA(cudaStreamUpdateCaptureDependencies(st, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  GR_CUDA(cudaStreamBeginCaptureToGraph(h->aux_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  Launch LB{h->aux_stream, nullptr, &h->tiles};
  rc = enqueue_body(h, LB, rtol, maxit, hc);
  cudaGraph_t body_out = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->aux_stream, &body_out);
  if (rc) return rc;
  GR_CUDA(e);
  return enqueue_post(h, L, b, x, maxit);
}

// read iterations and the true relative residual of a finished graph solve
static int graph_results(pc_handle* h, cudaStream_t st, double rtol, int* iters, double* relres) {
  if (arnoldi_df(h)) {
    if (int rc = fetch_scalars(h, st, h->scal + 10, 1, 12)) return rc;
    if (h->host[12] != 0.0) return fail(PC_ERR_TIMEOUT, "graph solve: a bounded device wait ran out");
  }
  if (int rc = fetch_scalars(h, st, h->scal + 1, 3, 0, h->idx + 1)) return rc;
  const int kdone = (int)h->host[3];
  const double ref = h->host[1], r2 = h->host[2];
  const double rr = ref > 0 ? std::sqrt(r2) / ref : 0.0;
  h->last_k = kdone;
  h->last_res0 = ref > 0 ? 1.0 : 0.0;  // zero initial guess
  if (iters) *iters = kdone;
  if (relres) *relres = rr;
  if (ref == 0.0) return PC_OK;  // b = 0: x = 0 is exact
  if (!std::isfinite(rr) || !std::isfinite(h->host[0])) return fail(PC_ERR_BREAKDOWN, "graph solve: non-finite residual");
  if (h->host[0] > rtol) return fail(PC_ERR_NOT_CONVERGED, "graph solve: maxit reached before rtol");
  return PC_OK;
}

extern "C" int pc_gmres_solve_graph(pc_handle* h, const double* b, double* x, double rtol, int maxit, int* iters,
                                    double* relres, void* stream) {
  if (!h || !b || !x) return fail(PC_ERR_ARG, "pc_gmres_solve_graph: null argument");
  if (!(rtol > 0)) return fail(PC_ERR_ARG, "pc_gmres_solve_graph: rtol must be > 0");
  if (int rc = graph_supported(h, maxit)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  h->last_k = -1;
  if (!h->gexec || h->g_b != b || h->g_x != x || h->g_rtol != rtol || h->g_maxit != maxit) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    GR_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
    int rc = capture_solve(h, b, x, rtol, maxit, h->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    GR_CUDA(e);
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    GR_CUDA(e);
    h->g_b = b;
    h->g_x = x;
    h->g_rtol = rtol;
    h->g_maxit = maxit;
  }
  GR_CUDA(cudaGraphLaunch(h->gexec, st));
  int k = 0;
  double rr = 0.0;
  const int rc = graph_results(h, st, rtol, &k, &rr);
  if (iters) *iters = k;
  if (relres) *relres = rr;
  if (rc != PC_OK) return rc;
  // a true residual above rtol continues host-driven from x (gmres_confirm)
  return gmres_confirm(h, b, x, rtol, maxit, PC_GMRES_RIGHT, rc, k, rr, iters, relres, st);
}

// ---------------------------------------------------------------------------
// Batch: many independent problems (uneven m1, n, gamma, a) solved by ONE graph
// launch; each problem is a parallel branch with its own WHILE loop.
// ---------------------------------------------------------------------------
struct pc_batch {
  std::vector<pc_handle*> hs;
  std::vector<const double*> b;  // right-hand sides and solutions of the problems
  std::vector<double*> x;
  double rtol = 0.0;
  int maxit = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t origin = nullptr;
  std::vector<cudaEvent_t> events;
};

// do two handles' Krylov workspaces (pc_setup_shared) share any byte?
static bool krylov_overlap(const pc_handle* a, const pc_handle* b) {
  if (!a->kws || !b->kws) return false;
  return a->kws < b->kws + b->kws_bytes && b->kws < a->kws + a->kws_bytes;
}

static void batch_release(pc_batch* bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  for (auto e : bt->events) cudaEventDestroy(e);
  if (bt->origin) cudaStreamDestroy(bt->origin);
}

extern "C" int pc_batch_create(pc_handle* const* hs, int count, const double* const* b, double* const* x, double rtol,
                               int maxit, pc_batch** out) {
  if (!hs || !b || !x || !out || count < 1) return fail(PC_ERR_ARG, "pc_batch_create: bad arguments");
  if (!(rtol > 0)) return fail(PC_ERR_ARG, "pc_batch_create: rtol must be > 0");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b[i] || !x[i]) return fail(PC_ERR_ARG, "pc_batch_create: null handle or vector");
    if (int rc = graph_supported(hs[i], maxit)) return rc;
    for (int q = 0; q < i; ++q)
      if (hs[q] == hs[i]) return fail(PC_ERR_ARG, "pc_batch_create: a handle appears twice");
  }
  pc_batch* bt = new (std::nothrow) pc_batch();
  if (!bt) return fail(PC_ERR_OOM, "host allocation failed");
  bt->hs.assign(hs, hs + count);
  bt->rtol = rtol;
  bt->maxit = maxit;
  bt->b.assign(b, b + count);
  bt->x.assign(x, x + count);
  int rc = PC_OK;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&bt->origin, cudaStreamNonBlocking);
  for (int i = 0; e == cudaSuccess && i < 2 * count + 1; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) bt->events.push_back(ev);
  }
  if (e != cudaSuccess) {
    batch_release(bt);
    delete bt;
    return cuda_fail(e, "pc_batch_create");
  }
  e = cudaStreamBeginCapture(bt->origin, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaEventRecord(bt->events[0], bt->origin);
  for (int i = 0; e == cudaSuccess && rc == PC_OK && i < count; ++i) {
    // fork: the problem's capture stream joins the capture, then runs its own solve
    e = cudaStreamWaitEvent(hs[i]->cap_stream, bt->events[0], 0);
    // a problem whose Krylov workspace overlaps an earlier problem's starts after it
    for (int q = 0; e == cudaSuccess && q < i; ++q)
      if (krylov_overlap(hs[q], hs[i])) e = cudaStreamWaitEvent(hs[i]->cap_stream, bt->events[1 + q], 0);
    if (e != cudaSuccess) break;
    rc = capture_solve(hs[i], b[i], x[i], rtol, maxit, hs[i]->cap_stream);
    if (rc) break;
    e = cudaEventRecord(bt->events[1 + i], hs[i]->cap_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->origin, bt->events[1 + i], 0);  // join
  }
  cudaError_t ee = cudaStreamEndCapture(bt->origin, &g);
  if (rc == PC_OK && e != cudaSuccess) rc = cuda_fail(e, "pc_batch_create: capture");
  if (rc == PC_OK && ee != cudaSuccess) rc = cuda_fail(ee, "pc_batch_create: end capture");
  if (rc == PC_OK) {
    e = cudaGraphInstantiate(&bt->exec, g, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "pc_batch_create: instantiate");
  }
  if (g) cudaGraphDestroy(g);
  if (rc != PC_OK) {
    batch_release(bt);
    delete bt;
    return rc;
  }
  *out = bt;
  return PC_OK;
}

extern "C" int pc_batch_solve(pc_batch* bt, int* iters, double* relres, void* stream) {
  if (!bt) return fail(PC_ERR_ARG, "pc_batch_solve: null batch");
  cudaStream_t st = (cudaStream_t)stream;
  for (pc_handle* h : bt->hs) h->last_k = -1;
  GR_CUDA(cudaGraphLaunch(bt->exec, st));
  int worst = PC_OK;
  for (size_t i = 0; i < bt->hs.size(); ++i) {
    int k = 0;
    double rr = 0.0;
    int rc = graph_results(bt->hs[i], st, bt->rtol, &k, &rr);
    if (rc == PC_OK)  // a true residual above rtol continues host-driven from x[i] (gmres_confirm)
      rc = gmres_confirm(bt->hs[i], bt->b[i], bt->x[i], bt->rtol, bt->maxit, PC_GMRES_RIGHT, rc, k, rr, &k, &rr, st);
    if (iters) iters[i] = k;
    if (relres) relres[i] = rr;
    if (rc == PC_ERR_CUDA) return rc;
    if (rc != PC_OK && worst == PC_OK) worst = rc;
  }
  return worst;
}

extern "C" int pc_batch_destroy(pc_batch* bt) {
  if (!bt) return PC_OK;
  cudaDeviceSynchronize();
  batch_release(bt);
  delete bt;
  return PC_OK;
}

// ---------------------------------------------------------------------------
// instrumentation and status
// ---------------------------------------------------------------------------
extern "C" int pc_profile(pc_handle* h, int on) {
  if (!h) return fail(PC_ERR_ARG, "null handle");
  h->prof.on = on != 0;
  return PC_OK;
}

extern "C" int pc_profile_classes(pc_handle* h, const char* names) {
  if (!h) return fail(PC_ERR_ARG, "null handle");
  if (!names || !*names) {
    h->prof.mask = ~0ull;
    return PC_OK;
  }
  uint64_t mask = 0;
  std::string list(names);
  size_t pos = 0;
  while (pos <= list.size()) {
    size_t end = list.find(',', pos);
    if (end == std::string::npos) end = list.size();
    const std::string nm = list.substr(pos, end - pos);
    int found = -1;
    for (int kc = 0; kc < KC_COUNT; ++kc)
      if (nm == kernel_class_name(kc)) found = kc;
    if (found < 0) return fail(PC_ERR_ARG, "pc_profile_classes: unknown kernel class '" + nm + "'");
    mask |= 1ull << found;
    pos = end + 1;
  }
  h->prof.mask = mask;
  return PC_OK;
}

extern "C" int pc_stats(pc_handle* h, pc_kernel_stat* out, int cap, int* count) {
  if (!h) return fail(PC_ERR_ARG, "null handle");
  cudaError_t e = h->prof.flush();
  if (e != cudaSuccess) return cuda_fail(e, "pc_stats");
  int c = 0;
  for (int k = 0; k < KC_COUNT && c < cap; ++k) {
    if (!out) break;
    std::memset(&out[c], 0, sizeof(pc_kernel_stat));
    std::snprintf(out[c].name, sizeof(out[c].name), "%s", kernel_class_name(k));
    out[c].launches = h->prof.launches[k];
    out[c].total_ms = h->prof.ms[k];
    out[c].bytes = h->prof.bytes[k];
    out[c].flops = h->prof.flops[k];
    ++c;
  }
  if (count) *count = KC_COUNT;
  return PC_OK;
}

extern "C" int pc_stats_reset(pc_handle* h) {
  if (!h) return fail(PC_ERR_ARG, "null handle");
  cudaError_t e = h->prof.flush();
  h->prof.reset();
  return e == cudaSuccess ? PC_OK : cuda_fail(e, "pc_stats_reset");
}

extern "C" int64_t pc_launch_count(const pc_handle* h) { return h ? h->prof.total : 0; }

extern "C" int pc_debug_status(int reset, int* code) {
  if (!code) return fail(PC_ERR_ARG, "pc_debug_status: null code");
  const int a = pcopt_debug_matvec(reset), b = pcopt_debug_krylov(reset), c = pcopt_debug_tfft(reset);
  *code = a ? a : (b ? b : c);
#ifdef PCOPT_DEBUG
  return PC_OK;
#else
  return PC_ERR_UNSUPPORTED;  // release build: no checks compiled in, *code is 0
#endif
}

extern "C" const char* pc_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* pc_status_string(int s) {
  switch (s) {
    case PC_OK: return "ok";
    case PC_ERR_ARG: return "invalid argument";
    case PC_ERR_CUDA: return "CUDA error";
    case PC_ERR_OOM: return "out of device memory";
    case PC_ERR_NOT_CONVERGED: return "not converged";
    case PC_ERR_BREAKDOWN: return "breakdown (non-finite value)";
    case PC_ERR_UNSUPPORTED: return "unsupported";
    case PC_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------
// tile shapes of the tunable kernels
// ---------------------------------------------------------------------------
static int check_tiles(const pc_tiles* t) {
  if (t->mg_cx != 0 && t->mg_cx != 8 && t->mg_cx != 16) return fail(PC_ERR_ARG, "mg_cx must be 0, 8 or 16");
  if (t->mg_ctas < 0 || t->mg_ctas > 64) return fail(PC_ERR_ARG, "mg_ctas must be in [0, 64]");
  if (t->mv_tj < 0 || t->mv_tj > 4096) return fail(PC_ERR_ARG, "mv_tj must be in [0, 4096]");
  if (t->pro_pch < 0 || t->pro_pch > 64) return fail(PC_ERR_ARG, "pro_pch must be in [0, 64]");
  if (t->fft_stream < 0 || t->fft_stream > 1) return fail(PC_ERR_ARG, "fft_stream must be 0 or 1");
  if (t->mg_march < 0 || t->mg_march > 1) return fail(PC_ERR_ARG, "mg_march must be 0 or 1");
  if (t->mg_seg < 0 || t->mg_seg > 1024) return fail(PC_ERR_ARG, "mg_seg must be in [0, 1024]");
  if (t->fst_stream < 0 || t->fst_stream > 3) return fail(PC_ERR_ARG, "fst_stream must be in [0, 3]");
  return PC_OK;
}

static void drop_graphs(pc_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
}

extern "C" int pc_get_tiles(const pc_handle* h, pc_tiles* out) {
  if (!h || !out) return fail(PC_ERR_ARG, "pc_get_tiles: null argument");
  out->mg_cx = h->tiles.mg_cx;
  out->mg_ctas = h->tiles.mg_ctas;
  out->mv_tj = h->tiles.mv_tj;
  out->pro_pch = h->tiles.pro_pch;
  out->fft_stream = h->tiles.fft_stream;
  out->mg_march = h->tiles.mg_march;
  out->mg_seg = h->tiles.mg_seg;
  out->fst_stream = h->tiles.fst_stream;
  return PC_OK;
}

extern "C" int pc_set_tiles(pc_handle* h, const pc_tiles* t) {
  if (!h || !t) return fail(PC_ERR_ARG, "pc_set_tiles: null argument");
  if (int rc = check_tiles(t)) return rc;
  h->tiles.mg_cx = t->mg_cx;
  h->tiles.mg_ctas = t->mg_ctas;
  h->tiles.mv_tj = t->mv_tj;
  h->tiles.pro_pch = t->pro_pch;
  h->tiles.fft_stream = t->fft_stream;
  h->tiles.mg_march = t->mg_march;
  h->tiles.mg_seg = t->mg_seg;
  h->tiles.fst_stream = t->fst_stream;
  drop_graphs(h);  // a cached solve graph holds the old launch shapes
  return PC_OK;
}

// mean device time of `reps` calls of f (after one untimed call); +inf on error
template <typename F>
static double time_reps(cudaStream_t st, int reps, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  double out = HUGE_VAL;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) goto done;
  if (f() != cudaSuccess) goto done;
  if (cudaEventRecord(a, st) != cudaSuccess) goto done;
  for (int i = 0; i < reps; ++i)
    if (f() != cudaSuccess) goto done;
  if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) goto done;
  {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) out = ms / reps;
  }
done:
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return out;
}

template <typename Tc, typename TU>
static cudaError_t spatial_any(pc_handle* h, Launch& L) {
  return spatial_solve<Tc, TU>(h, L);
}

static cudaError_t spatial_for(pc_handle* h, Launch& L) {
  if (!h->fp32) return spatial_any<double, double2>(h, L);
  return h->bf16s ? spatial_any<float, __nv_bfloat162>(h, L) : spatial_any<float, float2>(h, L);
}

extern "C" int pc_autotune(pc_handle* h, int reps, pc_tiles* chosen, void* stream) {
  if (!h) return fail(PC_ERR_ARG, "null handle");
  if (reps < 1 || reps > 100) return fail(PC_ERR_ARG, "reps must be in [1, 100]");
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  GR_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(PC_ERR_ARG, "pc_autotune: stream is capturing");
  // deterministic, finite contents for the workspace the candidates read
  const size_t cb = h->fp32 ? sizeof(float2) : sizeof(double2);
  GR_CUDA(cudaMemsetAsync(h->lv[0].r, 0x3e, (size_t)h->planes * h->lv[0].np * cb, st));
  GR_CUDA(cudaMemsetAsync(h->V, 0x3e, h->U * sizeof(double), st));
  GR_CUDA(cudaMemsetAsync(h->Z, 0x3e, h->U * (h->fp32 ? sizeof(float) : sizeof(double)), st));
  if (h->vf32) GR_CUDA(cudaMemsetAsync(h->vf32, 0x3e, h->U * sizeof(float), st));
  Tiles best = h->tiles;
  // spatial step: fused down-leg tile and grid, then the per-level plane chunk
  if (h->spatial != PC_SPATIAL_FST) {
    double tbest = HUGE_VAL;
    const bool fused = h->dim == 2 && h->coarse_l0 >= 1;
    const int cxs[2] = {8, 16};
    const int ctas[5] = {2, 4, 8, 16, 32};
    for (int ci = 0; ci < (fused ? 2 : 1); ++ci)
      for (int ki = 0; ki < (fused ? 5 : 1); ++ki) {
        Tiles t = best;
        if (fused) {
          t.mg_cx = cxs[ci];
          t.mg_ctas = ctas[ki];
          t.mg_march = 0;
        }
        Launch L{st, nullptr, &t};
        const double ms = time_reps(st, reps, [&] { return spatial_for(h, L); });
        if (ms < tbest) {
          tbest = ms;
          best.mg_cx = t.mg_cx;
          best.mg_ctas = t.mg_ctas;
          best.mg_march = 0;
        }
      }
    // the register-marching down leg (FP32 iterates), by coarse rows per segment
    const bool march = fused && h->fp32 && !h->bf16s && h->lv[0].w4;
    const int segs[4] = {8, 16, 32, 64};
    for (int si = 0; si < (march ? 4 : 0); ++si) {
      Tiles t = best;
      t.mg_march = 1;
      t.mg_seg = segs[si];
      Launch L{st, nullptr, &t};
      const double ms = time_reps(st, reps, [&] { return spatial_for(h, L); });
      if (ms < tbest) {
        tbest = ms;
        best.mg_march = 1;
        best.mg_seg = segs[si];
      }
    }
    const int pchs[5] = {2, 4, 8, 16, 32};
    if (h->coarse_l0 >= 2 || (h->dim == 3 && h->coarse_l0 >= 1)) {
      tbest = HUGE_VAL;
      for (int pi = 0; pi < 5; ++pi) {
        Tiles t = best;
        t.pro_pch = pchs[pi];
        Launch L{st, nullptr, &t};
        const double ms = time_reps(st, reps, [&] { return spatial_for(h, L); });
        if (ms < tbest) {
          tbest = ms;
          best.pro_pch = t.pro_pch;
        }
      }
    }
  }
  // sine-transform solves: one CTA per line tile or persistent streaming CTAs
  if (h->spatial == PC_SPATIAL_FST) {
    double tbest = HUGE_VAL;
    for (int mode = 0; mode < 4; ++mode) {
      Tiles t = best;
      t.fst_stream = mode;
      Launch L{st, nullptr, &t};
      const double ms = time_reps(st, reps, [&] { return spatial_for(h, L); });
      if (ms < tbest) {
        tbest = ms;
        best.fst_stream = mode;
      }
    }
  }
  // time FFTs: one CTA per column tile or persistent streaming CTAs (power-of-two n)
  if ((h->n & (h->n - 1)) == 0) {
    double tbest = HUGE_VAL;
    for (int mode = 0; mode < 2; ++mode) {
      Tiles t = best;
      t.fft_stream = mode;
      Launch L{st, nullptr, &t};
      const double ms = time_reps(st, reps, [&]() -> cudaError_t {
        typedef float2 C32;
        if (!h->fp32) {
          cudaError_t e = launch_tfft_forward<double>(L, h->ms, h->n, h->V, h->dpow64, h->dinv64, h->tw64,
                                                      (double2*)h->lv[0].r);
          if (e != cudaSuccess) return e;
          return launch_tfft_inverse<double, double2, double>(L, h->ms, h->n, (const double2*)h->lv[0].u, h->dpow64,
                                                              h->dinv64, h->tw64, (double*)h->Z);
        }
        // flexible GMRES feeds the FP32 transform with the FP32 copy of the basis vector
        cudaError_t e = launch_tfft_forward<float>(L, h->ms, h->n, (const float*)h->vf32, h->dpow32, h->dinv32,
                                                   h->tw32, (C32*)h->lv[0].r);
        if (e != cudaSuccess) return e;
        if (h->bf16s)
          return launch_tfft_inverse<float, __nv_bfloat162, float>(L, h->ms, h->n, (const __nv_bfloat162*)h->lv[0].u,
                                                                   h->dpow32, h->dinv32, h->tw32, (float*)h->Z);
        return launch_tfft_inverse<float, float2, float>(L, h->ms, h->n, (const float2*)h->lv[0].u, h->dpow32,
                                                         h->dinv32, h->tw32, (float*)h->Z);
      });
      if (ms < tbest) {
        tbest = ms;
        best.fft_stream = mode;
      }
    }
  }
  // the all-at-once matvec of the Arnoldi step: time blocks per thread
  {
    double tbest = HUGE_VAL;
    const int tjs[5] = {8, 16, 32, 64, 128};
    for (int ti = 0; ti < 5; ++ti) {
      if (tjs[ti] > h->n && ti > 0) break;
      Tiles t = best;
      t.mv_tj = tjs[ti];
      Launch L{st, nullptr, &t};
      const double ms = time_reps(st, reps, [&] {
        return matvec_basis(h, L, h->Z, h->V + h->U);
      });
      if (ms < tbest) {
        tbest = ms;
        best.mv_tj = t.mv_tj;
      }
    }
  }
  GR_CUDA(cudaGetLastError());
  h->tiles = best;
  drop_graphs(h);
  if (chosen) pc_get_tiles(h, chosen);
  return PC_OK;
}

// ---------------------------------------------------------------------------
// end-point solves (Section 1): y^(N) and p^(0) from a solution of A x = b
// ---------------------------------------------------------------------------
// z = (I + tau K)^{-1} r approximately: the handle's spatial solver at shift 1 on one plane
template <typename Tc, typename TU>
static cudaError_t shift1_solve(pc_handle* h, Launch& L, const double* r, double* z) {
  typedef typename Cx<Tc>::t C;
  cudaError_t e = launch_real_to_plane<Tc>(L, r, (C*)h->lv[0].r, h->ms);
  if (e != cudaSuccess) return e;
  if ((e = spatial_solve<Tc, TU>(h, L, 1, Tables<Tc>::sig1(h), true)) != cudaSuccess) return e;
  return launch_plane_to_real<TU>(L, (const TU*)h->lv[0].u, z, h->ms);
}

static cudaError_t shift1_any(pc_handle* h, Launch& L, const double* r, double* z) {
  if (!h->fp32) return shift1_solve<double, double2>(h, L, r, z);
  return h->bf16s ? shift1_solve<float, __nv_bfloat162>(h, L, r, z) : shift1_solve<float, float2>(h, L, r, z);
}

// flexible preconditioned conjugate gradients on (I + tau K) u = b (u, b: ms doubles)
static int pcg_E(pc_handle* h, Launch& L, const double* b, double* u, double rtol, int maxit, int* iters) {
  const int64_t ms = h->ms;
  const Grid g = grid_of(h, 0);
  const Stencil<double> st{h->lv[0].w64, h->lv[0].d64};
  cudaStream_t s = L.stream;
  double* r = h->V;
  double* z = h->V + ms;
  double* p = h->V + 2 * ms;
  double* q = h->V + 3 * ms;
  double* rold = h->tbuf;
  double* sc = h->scal + 10;  // [0] b.b, [1] r.z, [2] p.q, [3] r.r, [4] rold.z
  auto dot = [&](const double* a, const double* c, double* out) {
    return launch_multidot(L, a, (size_t)ms, 1, c, (size_t)ms, h->partial, out, nullptr, nullptr);
  };
  auto fetch = [&](int cnt) -> int {
    return fetch_scalars(h, s, sc, cnt, 0);
  };
  PC_CUDA(cudaMemsetAsync(u, 0, ms * sizeof(double), s));
  PC_CUDA(cudaMemcpyAsync(r, b, ms * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PC_CUDA(launch_norm2(L, b, ms, h->partial, sc));
  PC_CUDA(shift1_any(h, L, r, z));
  PC_CUDA(dot(r, z, sc + 1));
  PC_CUDA(launch_axpby<double>(L, 1.0, z, 0.0, p, ms));
  if (int rc = fetch(2)) return rc;
  const double bnorm = std::sqrt(h->host[0]);
  double rz = h->host[1];
  if (iters) *iters = 0;
  if (bnorm == 0.0) return PC_OK;
  if (!std::isfinite(bnorm) || !std::isfinite(rz)) return fail(PC_ERR_BREAKDOWN, "end-point solve: non-finite input");
  for (int it = 1; it <= maxit; ++it) {
    if (h->fevar && h->dim == 3)
      PC_CUDA(launch_fevar3_apply(L, h->m1, 1, h->h, h->lv[0].e64, 1.0, h->tau, p, 0.0, q));  // (M + tau K) p
    else if (h->fevar)
      PC_CUDA(launch_fevar_apply(L, h->m1, 1, h->h * h->h, h->lv[0].e64, 1.0, h->tau, p, 0.0, q));  // (M + tau K) p
    else if (h->fe)
      PC_CUDA(launch_fe_apply(L, g, 1, h->fes.wM, h->tau * h->fes.wK, p, 0.0, q));  // (M + tau K) p
    else
      PC_CUDA(launch_apply_E(L, g, st, p, q));
    PC_CUDA(dot(p, q, sc + 2));
    if (int rc = fetch(3)) return rc;
    const double pq = h->host[2];
    if (!(pq > 0) || !std::isfinite(pq)) return fail(PC_ERR_BREAKDOWN, "end-point solve: p.Ap not positive");
    const double alpha = rz / pq;
    PC_CUDA(launch_axpby<double>(L, alpha, p, 1.0, u, ms));
    PC_CUDA(launch_axpby<double>(L, 1.0, r, 0.0, rold, ms));
    PC_CUDA(launch_axpby<double>(L, -alpha, q, 1.0, r, ms));
    PC_CUDA(launch_norm2(L, r, ms, h->partial, sc + 3));
    if (int rc = fetch(4)) return rc;
    if (iters) *iters = it;
    const double rel = std::sqrt(h->host[3]) / bnorm;
    if (!std::isfinite(rel)) return fail(PC_ERR_BREAKDOWN, "end-point solve: non-finite residual");
    if (rel <= rtol) return PC_OK;
    PC_CUDA(shift1_any(h, L, r, z));
    PC_CUDA(dot(r, z, sc + 1));
    PC_CUDA(dot(rold, z, sc + 4));
    if (int rc = fetch(5)) return rc;
    const double rz_new = h->host[1];
    const double beta = (rz_new - h->host[4]) / rz;  // Polak-Ribiere: tolerates a varying preconditioner
    PC_CUDA(launch_axpby<double>(L, 1.0, z, beta, p, ms));
    rz = rz_new;
  }
  return fail(PC_ERR_NOT_CONVERGED, "end-point solve: not converged");
}

extern "C" int pc_end_point_solves(pc_handle* h, const double* x, const double* f_T, const double* g_0,
                                   const double* y0, const double* p_N, double* yN, double* p0, double rtol,
                                   int maxit, int* iters, void* stream) {
  if (!h || !x || !yN || !p0) return fail(PC_ERR_ARG, "pc_end_point_solves: null argument");
  if (!(rtol > 0)) return fail(PC_ERR_ARG, "pc_end_point_solves: rtol must be > 0");
  if (maxit < 1 || maxit > 10000) return fail(PC_ERR_ARG, "pc_end_point_solves: maxit must be in [1, 10000]");
  Launch L{(cudaStream_t)stream, &h->prof, &h->tiles};
  double* rhs_y = h->wbuf;
  double* rhs_p = h->wbuf + h->ms;
  if (!h->fe) {
    GR_CUDA(launch_endpoint_rhs(L, x, h->ms, h->n, h->tau, h->prm.gamma, f_T, g_0, y0, p_N, rhs_y, rhs_p));
  } else {  // the same combinations, multiplied by M
    GR_CUDA(launch_endpoint_rhs(L, x, h->ms, h->n, h->tau, h->prm.gamma, f_T, g_0, y0, p_N, h->tbuf,
                                h->tbuf + h->ms));
    GR_CUDA(launch_fe_apply(L, grid_of(h, 0), 2, h->fes.wM, 0.0, h->tbuf, 0.0, rhs_y));
  }
  int it_y = 0, it_p = 0;
  if (int rc = pcg_E(h, L, rhs_y, yN, rtol, maxit, &it_y)) return rc;
  if (int rc = pcg_E(h, L, rhs_p, p0, rtol, maxit, &it_p)) return rc;
  if (iters) *iters = it_y > it_p ? it_y : it_p;
  return PC_OK;
}
