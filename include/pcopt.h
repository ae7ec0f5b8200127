/*
 * pcopt -- GB300 (sm_103a) library for the all-at-once optimality system of
 * the parabolic optimal-control problem and its eps-circulant rotated
 * block-diagonal (RBD) preconditioner (Hon, Fung & Lin, arXiv 2410.22686).
 *
 * Problem (Eq. Cost_functional_heat, Eq. heat): minimise
 *   1/2 ||y - g||^2 + gamma/2 ||u||^2   s.t.  y_t - div(a grad y) = f + u,
 * homogeneous Dirichlet data on the unit square (dim 2) or cube (dim 3).
 * Backward Euler with tau = T/(n+1) and a conservative finite-difference
 * stencil (M = I, K = -L_h, face coefficient (a_P + a_Q)/2) give the scaled
 * all-at-once system A x = b of Eq. main_system / Eq. matrix_A:
 *
 *   A = [[alpha I, T^T], [-T, alpha I]],  T = B_n (x) I + tau I_n (x) K,
 *   x = [sqrt(gamma) y; p],  b = [g_vec; -sqrt(gamma) f_vec],  alpha = tau/sqrt(gamma).
 *
 * VECTOR LAYOUT.  Every all-at-once vector (x, b, v, w, lam, c) is a
 * contiguous FP64 array of 2*n*ms entries, ms = m1^dim, ordered
 * [half][time block][space]: half 0 is sqrt(gamma) y (resp. the first block
 * row), half 1 is p; time block j = 1..n is stored at index j-1; space is
 * C-ordered with x1 fastest, i.e. s = i1 + m1*i2 (+ m1*m1*i3), 0-based
 * interior indices.  Space-time source/target fields (f, g) are FP64 arrays
 * [time block][space] of n*ms entries; y0 is one spatial field of ms entries.
 *
 * MEMORY.  Vector arguments are DEVICE pointers owned by the caller (for
 * example torch CUDA tensors), 8-byte aligned, not overlapping unless stated.
 * The handle owns all workspace; it is allocated in pc_setup and released in
 * pc_destroy.  No other call allocates device memory.  Calls are asynchronous
 * on `stream` (a cudaStream_t, NULL = legacy default stream) except where a
 * host result (iteration count, residual) is returned: those synchronise the
 * stream before returning.  A handle must not be used from two host threads
 * at once.
 *
 * ERRORS.  Every entry point returns a pc_status; nothing throws across the
 * boundary.  pc_last_error() gives a human-readable message for the calling
 * thread's most recent failure.
 */
#ifndef PCOPT_H
#define PCOPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pc_status {
  PC_OK = 0,
  PC_ERR_ARG = 1,            /* invalid argument (see pc_last_error) */
  PC_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  PC_ERR_OOM = 3,            /* device allocation failed in pc_setup */
  PC_ERR_NOT_CONVERGED = 4,  /* Krylov solver hit max_iter; x holds the last iterate */
  PC_ERR_BREAKDOWN = 5,      /* NaN/Inf in a residual or Arnoldi coefficient */
  PC_ERR_UNSUPPORTED = 6,    /* valid request outside what this build implements */
  PC_ERR_TIMEOUT = 7         /* a bounded device-side wait (streamed copy) ran out; the result is invalid */
} pc_status;

typedef enum pc_spatial {
  PC_SPATIAL_AUTO = 0,  /* FST when a is constant (a_nodes == NULL), else multigrid */
  PC_SPATIAL_FST = 1,   /* exact sine-transform solves, constant a only (Example 1) */
  PC_SPATIAL_MG = 2     /* one V(1,0) multigrid cycle per shifted system (Example 2) */
} pc_spatial;

typedef enum pc_precision {
  PC_PREC_FP64 = 0,         /* preconditioner in FP64 */
  PC_PREC_MIXED_FP32 = 1,   /* preconditioner in FP32 (flexible GMRES keeps FP64 outside) */
  PC_PREC_MIXED_BF16S = 2,  /* as FP32, multigrid smoother iterates stored as BF16 */
  PC_PREC_AUTO = 3          /* FP32 when eps >= PC_AUTO_FP32_MIN_EPS, else FP64: the time
                               scaling D = diag(eps^{j/n}) amplifies the FP32 rounding of the
                               apply by up to 1/eps; down to this eps (the paper's eps = tau/2
                               included for n up to a few thousand) the FP32 preconditioner
                               needs at most about one iteration more than FP64;
                               pc_precision_of reports the choice */
} pc_precision;
#define PC_AUTO_FP32_MIN_EPS 1e-4

typedef enum pc_gmres_mode {
  PC_GMRES_RIGHT = 0,  /* flexible GMRES, right preconditioning, stops on ||b-Ax||/||b|| */
  PC_GMRES_LEFT = 1    /* GMRES on P^{-1}A x = P^{-1}b, stops on ||P^{-1}(b-Ax)||/||P^{-1}b|| */
} pc_gmres_mode;

typedef enum pc_space {
  PC_SPACE_FD = 0,  /* finite differences: M = I, conservative stencil of K (Eq. matrix_A as printed) */
  PC_SPACE_FE = 1   /* conforming bilinear (2D) / trilinear (3D) finite elements, mass matrix M
                       (Section 1: A = [[alpha I(x)M, T^T], [-T, alpha I(x)M]], T = B_n(x)M + tau I(x)K);
                       constant coefficient a only, sine-transform spatial solves */
} pc_space;

typedef enum pc_smoother {
  PC_SMOOTHER_RED_BLACK = 0,     /* one red-black Gauss-Seidel sweep from zero, red first (parallel) */
  PC_SMOOTHER_LEXICOGRAPHIC = 1  /* one sweep in the natural order, x1 fastest (Example 2's counts of
                                    Table 7 exactly; sequential along the grid diagonals, much slower) */
} pc_smoother;

/* Preconditioner of a handle (pc_set_preconditioner).
 *   PC_PRECOND_EPS_CIRCULANT: P_eps of Eq. matrix_P_eps, applied by the four
 *     steps of Section 2.1 (all time blocks in parallel; the default).
 *   PC_PRECOND_IDEAL_RBD: P of Eq. matrix_P (the paper's comparison, Tables 4
 *     and 8), applied by block substitution in time: n sequential steps, each
 *     one spatial solve ((1 + alpha) I + tau K) z = r per half by the handle's
 *     spatial solver (exact sine transforms or one V(1,0) cycle), half 2 forward
 *     and half 1 backward in time, then w = [[I, -I], [I, I]] [w1; w2]. */
typedef enum { PC_PRECOND_EPS_CIRCULANT = 0, PC_PRECOND_IDEAL_RBD = 1 } pc_precond_kind;

/* Arnoldi precision of GMRES (pc_set_arnoldi).  The paper fixes none (Section 3
 * runs MATLAB's FP64 gmres); these choose how the orthogonalisation of flexible
 * GMRES with the FP32 preconditioner uses GB300's small FP64 unit.
 *   PC_ARNOLDI_AUTO: FP64 handles as PC_ARNOLDI_FP64, mixed handles as
 *     PC_ARNOLDI_DOUBLE_FLOAT.
 *   PC_ARNOLDI_FP64: FP64 basis and FP64 products in the first Gram-Schmidt
 *     pass; on mixed handles the selective second pass takes FP32 products of
 *     20-bit truncations and the inner matvec of the FP32 basis is double-float.
 *   PC_ARNOLDI_FP64_STRICT: FP64 basis and FP64 products everywhere, the second
 *     pass and the inner matvec (FP32 input, FP64 arithmetic) included.
 *   PC_ARNOLDI_DOUBLE_FLOAT (mixed handles): each basis vector stored as two FP32
 *     planes, v = hi + lo to ~2^-48 relative (hi is the FP32 rounding the
 *     preconditioner reads); dot products and updates as error-free FP32
 *     transformations (FMA product errors, TwoSum), scalars and reductions in
 *     FP64; the second pass takes FP32 products of the hi planes. */
typedef enum {
  PC_ARNOLDI_AUTO = 0,
  PC_ARNOLDI_FP64 = 1,
  PC_ARNOLDI_FP64_STRICT = 2,
  PC_ARNOLDI_DOUBLE_FLOAT = 3
} pc_arnoldi;

typedef struct pc_params {
  int dim;          /* 2 or 3 */
  int m1;           /* interior grid points per dimension, h = 1/(m1+1); multigrid needs m1 = 2^k-1 */
  int n;            /* time blocks (FFT length), tau = T/(n+1); 1..4096.  Powers of two use the
                       register FFT; other lengths (the paper's n = 2^k - 1) a direct DFT */
  double T;         /* final time > 0 */
  double gamma;     /* regularisation parameter > 0 */
  double eps;       /* eps of C_{eps,n}, in (0, 1] */
  int spatial;      /* pc_spatial */
  int precision;    /* pc_precision */
  int max_iter;     /* Krylov capacity: basis storage for this many iterations (1..1000) */
  int space;        /* pc_space: spatial discretisation (0 = finite differences) */
  int smoother;     /* pc_smoother: Gauss-Seidel ordering of the multigrid pre-smoother (0 = red-black) */
} pc_params;

typedef struct pc_handle pc_handle;

/* Build a solver for one problem.  Section 1 (discretisation), Eq. matrix_A,
 * Eq. matrix_P_eps, Eq. decomposition_eps.
 *   a_nodes: HOST pointer to the coefficient a(x) sampled on all (m1+2)^dim
 *            grid nodes including the boundary, C-ordered with x1 fastest;
 *            NULL means a == 1.  Values must be finite, > 0 at interior nodes
 *            and >= 0 at boundary nodes.
 *   stream:  stream used for the coefficient upload.
 *   out:     receives the handle (caller releases it with pc_destroy).
 * With space = PC_SPACE_FE the matrices are the bilinear (2D) / trilinear (3D)
 * element matrices of the uniform grid with the consistent mass matrix
 * (M = (h/6)^dim [1 4 1]^(x)dim).  A constant a gives
 * K = a (h/6)^(dim-1)/h sum_axes [-1 2 -1] (x) [1 4 1].., and with the
 * sine-transform solver every spatial solve (sigma M + tau K) z = r is exact; a
 * nodal a gives K(a) = sum_e a_e K_e (a_e the mean of element e's corner values,
 * a 9-point stencil in 2D, 27-point in 3D), solved inside P_eps^{-1} by one
 * V(1,0) cycle of the element multigrid (Gauss-Seidel in 2^dim colours).
 * Errors: PC_ERR_ARG (dim not 2/3, m1 < 1, n outside 1..4096,
 * T <= 0, gamma <= 0, eps outside (0,1], a not as above, FST with non-constant a,
 * MG with m1 != 2^k-1, unknown space), PC_ERR_UNSUPPORTED (finite elements with
 * the natural-order smoother or BF16 storage), PC_ERR_OOM, PC_ERR_CUDA. */
int pc_setup(const pc_params* params, const double* a_nodes, void* stream, pc_handle** out);

/* Bytes of the Krylov storage a handle built from `params` needs: the basis of
 * max_iter + 1 vectors (8 bytes per unknown each, double-float or FP64) and the
 * max_iter preconditioned vectors of flexible GMRES (4 bytes per unknown with an
 * FP32 preconditioner, 8 with FP64), each part rounded up to 256 bytes.  This
 * storage is what full GMRES (Section 3: no restarts) needs to hold, and it
 * dominates a handle's memory.  Host arithmetic only.
 * Errors: PC_ERR_ARG (null argument; dim, m1, n, max_iter, eps or precision as
 * in pc_setup). */
int pc_krylov_bytes(const pc_params* params, size_t* bytes);

/* pc_setup with the Krylov storage in caller-provided device memory instead of
 * the handle's own: krylov (device, 256-byte aligned, at least
 * pc_krylov_bytes(params) bytes) holds the basis and then the preconditioned
 * vectors.  The caller owns that memory, keeps it alive while the handle exists
 * and may give overlapping ranges to several handles, which then must not solve
 * at the same time: a batch (pc_batch_create) starts a problem whose range
 * overlaps an earlier problem's after that problem has finished, so more
 * problems than fit in memory at once run in one graph launch.  Every
 * solve (and pc_autotune) overwrites the range.
 * Errors: as pc_setup; PC_ERR_ARG also for a null, misaligned or too small
 * workspace (checked before any device work). */
int pc_setup_shared(const pc_params* params, const double* a_nodes, void* krylov, size_t krylov_bytes,
                    void* stream, pc_handle** out);

/* The precision a handle resolved to (PC_PREC_FP64, PC_PREC_MIXED_FP32 or
 * PC_PREC_MIXED_BF16S; PC_PREC_AUTO is resolved at setup). */
int pc_precision_of(const pc_handle* h, int* precision);

/* Replace the coefficient a(x) of an existing handle without reallocating:
 * the stencil of every level (and the FST eigenvalues) is recomputed on the
 * host and copied into the handle's buffers.  a_nodes: HOST, (m1+2)^dim values
 * as in pc_setup (NULL means a == 1).  Synchronises `stream`.
 * Errors: PC_ERR_ARG (a not as in pc_setup; non-constant a on an FST handle). */
int pc_set_coefficient(pc_handle* h, const double* a_nodes, void* stream);

/* Replace a(x) at the interior nodes by exp(log_a), on the device (the
 * differentiable parameters of pc_grad_log_a: the nodal log-coefficient).  The
 * boundary nodes keep the values given at setup or by the last
 * pc_set_coefficient.  Rebuilds every multigrid level's face weights from the
 * nodal values by injection (as pc_setup does), so the handle then acts exactly
 * as one set up with those nodal values.  Asynchronous on `stream` (no host
 * work, no synchronisation).
 *   log_a: device, ms = m1^dim FP64, interior nodes in vector ordering.  The
 *          values must be finite (exp of them is the coefficient; no device-side
 *          check: NaN or Inf surfaces later as PC_ERR_BREAKDOWN of a solve).
 * Errors: PC_ERR_ARG (null), PC_ERR_UNSUPPORTED (sine-transform handles, whose
 * coefficient must stay constant). */
int pc_set_log_coefficient(pc_handle* h, const double* log_a, void* stream);

/* Select the preconditioner used by pc_apply_precond, pc_gmres_solve and
 * pc_adjoint_solve (pc_precond_kind).  The graph-launched and batched solves
 * take the eps-circulant one only (PC_ERR_UNSUPPORTED otherwise).  Errors:
 * PC_ERR_ARG (unknown kind), PC_ERR_UNSUPPORTED (ideal RBD on a finite-element
 * handle). */
int pc_set_preconditioner(pc_handle* h, int kind);

/* Select the Arnoldi precision (pc_arnoldi) of later solves on the handle.
 * Errors: PC_ERR_ARG (unknown mode), PC_ERR_UNSUPPORTED (double-float basis on an
 * FP64 handle). */
int pc_set_arnoldi(pc_handle* h, int mode);

/* Release the handle and its workspace (waits for its work to finish).  NULL is a no-op. */
int pc_destroy(pc_handle* h);

/* y = A x  (Eq. matrix_A, Section 2.1: two block-bidiagonal Toeplitz products, O(mn);
 * with finite elements the blocks carry M, see pc_space).
 * x, y: device, 2*n*ms FP64, must not overlap. */
int pc_matvec(pc_handle* h, const double* x, double* y, void* stream);

/* y = A x for an FP32 vector x (Eq. matrix_A): the product flexible GMRES forms
 * with its FP32 basis Z.  Evaluated in double-float arithmetic on the FP32 units
 * (each FP64 coefficient split into two floats, FMA error terms, TwoSum
 * accumulation); relative error of order 2^-46 of the largest term; FP64 output.
 * Finite-element handles use the same double-float scheme on the element stencils.
 * x: device, 2*n*ms FP32; y: device, 2*n*ms FP64. */
int pc_matvec_f32(pc_handle* h, const float* x, double* y, void* stream);

/* y = A^T x  (block transpose of Eq. matrix_A; equals S A S with S = diag(I, -I)).
 * x, y: device, 2*n*ms FP64, must not overlap. */
int pc_matvec_transpose(pc_handle* h, const double* x, double* y, void* stream);

/* w = P_eps^{-1} v by the four steps of Section 2.1: scaled FFT along time,
 * n independent complex-shifted spatial solves (FST or one V(1,0) cycle),
 * inverse scaled FFT, and w = [[I,-I],[I,I]] w~.  Computed in the handle's
 * precision (FP64, or FP32 for the mixed modes); input and output are FP64.
 * v, w: device, 2*n*ms FP64; v and w may be the same pointer. */
int pc_apply_precond(pc_handle* h, const double* v, double* w, void* stream);

/* b = [g_vec; -sqrt(gamma) f_vec] of Eq. main_system_before / Eq. main_system:
 * g_vec_j = tau g^(j) (j = 1..n; the final condition p^(N) = 0 adds nothing),
 * f_vec_1 = tau f^(1) + y0, f_vec_j = tau f^(j).  Finite elements: every term is
 * multiplied by M (g_vec_j = tau M g^(j), f_vec_1 = tau M f^(1) + M y0, ...).
 * f, g: device, n*ms FP64 (time levels t_j = j tau, j = 1..n); y0: device, ms
 * FP64 (NULL means 0); f may be NULL (means 0).  b: device, 2*n*ms FP64. */
int pc_build_rhs(pc_handle* h, const double* f, const double* g, const double* y0,
                 double* b, void* stream);

/* Solve A x = b by preconditioned GMRES without restarts (Section 3: MATLAB gmres,
 * zero initial guess, relative tolerance; Lemma 2.1), preconditioner P_eps.
 *   b: device rhs; x: device, in = initial guess x0, out = solution.
 *   rtol > 0; maxit in 1..params.max_iter; mode: pc_gmres_mode (LEFT needs PC_PREC_FP64).
 *   iters, relres: HOST outputs (may be NULL): iterations done and the final
 *   relative residual (true residual for RIGHT, preconditioned for LEFT).
 * Arnoldi (classical Gram-Schmidt with one re-orthogonalisation), the Givens
 * least-squares update, the matvec and the true residual are FP64 in every
 * precision mode.  RIGHT mode stops on the least-squares estimate of the
 * residual and then forms the true residual ||b - A x|| / ||b||; if that misses
 * rtol (an FP32 preconditioner can leave it just above the estimate) and
 * iterations remain, the solve continues from x in a fresh Krylov space until
 * the true residual meets rtol or maxit iterations in total are spent; iters
 * counts every iteration.  PC_OK therefore means relres <= rtol.
 * Synchronises `stream`.
 * Errors: PC_ERR_NOT_CONVERGED (x holds the maxit-th iterate), PC_ERR_BREAKDOWN. */
int pc_gmres_solve(pc_handle* h, const double* b, double* x, double rtol, int maxit,
                   int mode, int* iters, double* relres, void* stream);

/* Residual history of the handle's last solve (pc_gmres_solve, pc_adjoint_solve,
 * pc_gmres_solve_graph or its batch): out[0] = initial relative residual, out[i]
 * = the GMRES least-squares estimate ||r_i|| / ||b|| after iteration i (RIGHT:
 * of the true residual in exact arithmetic; LEFT: of the preconditioned one),
 * i.e. out[0] times the product of the first i Givens sines, non-increasing.
 *   out: HOST array of cap entries; *count (HOST) = entries written, min(cap,
 *   iterations + 1); 0 before any solve, or after one that failed before its
 *   first residual.  Copies the sines from the device on `stream` and
 *   synchronises it.
 * After a continuation (pc_gmres_solve) the history is that of the last Krylov
 * space, out[0] being its initial residual.
 * Errors: PC_ERR_ARG (null h or count, cap < 0, out NULL with cap > 0). */
int pc_residual_history(pc_handle* h, double* out, int cap, int* count, void* stream);

/* The same right-preconditioned (flexible) GMRES solve from a zero initial
 * guess, run as ONE CUDA-graph launch: the iteration is the body of a graph
 * WHILE node whose condition a kernel sets on the device from the residual
 * estimate, so no host round trip happens per iteration.  The graph is built
 * on the first call and reused while (b, x, rtol, maxit) are unchanged.
 *   x: device, overwritten (the initial guess is zero).  iters/relres as in
 *   pc_gmres_solve (relres is the true relative residual; a true residual above
 *   rtol is continued host-driven as in pc_gmres_solve).  Synchronises `stream`.
 * Errors: as pc_gmres_solve; PC_ERR_UNSUPPORTED for n not a power of two,
 * n > 1024 (FP32 preconditioner) or n > 256 (FP64 preconditioner). */
int pc_gmres_solve_graph(pc_handle* h, const double* b, double* x, double rtol, int maxit, int* iters,
                         double* relres, void* stream);

/* Batched solve of independent problems of uneven size (each with its own
 * handle: grid, n, gamma and a may all differ): pc_batch_create captures one
 * graph in which every problem is a parallel branch running its own device-
 * controlled FGMRES loop (as pc_gmres_solve_graph); pc_batch_solve runs the
 * whole batch with ONE graph launch and fills iters[count], relres[count]
 * (HOST arrays, may be NULL).  hs: distinct handles; b[i], x[i]: device
 * vectors of handle i (x overwritten, zero initial guess).  The batch keeps
 * pointers to everything it was created with; destroy it before those.
 * Problems whose Krylov storage overlaps (pc_setup_shared) are ordered: the
 * later one in hs starts when the earlier one has finished; all others run
 * concurrently.  A problem whose true residual misses rtol after the launch is
 * continued host-driven as in pc_gmres_solve.  pc_batch_solve returns the worst
 * status over the problems. */
typedef struct pc_batch pc_batch;
int pc_batch_create(pc_handle* const* hs, int count, const double* const* b, double* const* x, double rtol,
                    int maxit, pc_batch** out);
int pc_batch_solve(pc_batch* batch, int* iters, double* relres, void* stream);
int pc_batch_destroy(pc_batch* batch);

/* Solve the adjoint system A^T lam = c with the same preconditioner, using
 * A^T = S A S, S = diag(I, -I) (from the block form of Eq. matrix_A with K
 * symmetric): lam = S A^{-1} S c.  Arguments as pc_gmres_solve; lam in/out
 * (initial guess in). */
int pc_adjoint_solve(pc_handle* h, const double* c, double* lam, double rtol, int maxit,
                     int mode, int* iters, double* relres, void* stream);

/* Stencil derivative for the gradient with respect to the nodal log a:
 *   grad_P = -tau * sum_j [ lam1_j^T (dK/dlog a_P) x2_j - lam2_j^T (dK/dlog a_P) x1_j ],
 *   u^T (dK/dlog a_P) v = a_P/(2h^2) sum_{faces (P,Q)} (u_P-u_Q)(v_P-v_Q),
 * i.e. -lam^T (dA/dlog a_P) x for interior nodes P (boundary nodes fixed).
 * Finite elements: u^T (dK/dlog a_P) v = a_P / 2^dim sum over the 2^dim elements
 * e around P of u_e^T K_e v_e (K_e the element stiffness of a = 1).
 *   x, lam: device all-at-once vectors; grad: device, ms FP64 (interior nodes,
 *   same spatial ordering), overwritten. */
int pc_grad_log_a(pc_handle* h, const double* x, const double* lam, double* grad, void* stream);

/* Gradient with respect to the target g of a scalar L(x) through the solve
 * (b1_j = tau g_j in Eq. main_system): given the adjoint lam = A^{-T} dL/dx,
 *   grad_g[j][s] = tau * lam1[j][s],  j = 1..n (the first half of lam);
 * finite elements (b1_j = tau M g_j): grad_g[j] = tau M lam1[j].
 *   lam: device all-at-once vector; grad_g: device, n*ms FP64, overwritten. */
int pc_grad_g(pc_handle* h, const double* lam, double* grad_g, void* stream);

/* The discrete tracking objective (Eq. Cost_functional_heat on the grid, with
 * u = p/gamma):
 *   J_h = h^d tau [ 1/2 sum_{j=1..n} ||y_j - g_j||^2 + 1/(2 gamma) sum_{j=1..n} ||p_j||^2 ],
 * y = x1/sqrt(gamma), p = x2; the optimality system of Eq. main_system is its
 * KKT system.  Finite elements: h^d I replaced by the mass matrix M,
 * J_h = tau [1/2 sum (y_j - g_j)^T M (y_j - g_j) + 1/(2 gamma) sum p_j^T M p_j].
 * x: device all-at-once vector; g: device, n*ms; J: device, one
 * FP64, written asynchronously (deterministic reduction order).  Uses the
 * handle's reduction scratch: do not overlap with a solve on the same handle. */
int pc_objective(pc_handle* h, const double* x, const double* g, double* J, void* stream);

/* Gradient of J_h (pc_objective) times the scalar *gJ (device; NULL means 1):
 *   gx1 = gJ h^d tau (y - g)/sqrt(gamma),  gx2 = gJ h^d tau p/gamma   (dJ/dx)
 *   gg  = -gJ h^d tau (y - g)                                          (explicit dJ/dg)
 * (finite elements: h^d replaced by M applied to each time block).
 * gx: device all-at-once vector or NULL; gg: device n*ms or NULL (not both). */
int pc_objective_grad(pc_handle* h, const double* x, const double* g, const double* gJ, double* gx, double* gg,
                      void* stream);

/* Allocation-free variant of pc_grad_log_a (the paper has no counterpart: it
 * is a deployment feature of this library).  For callers that may not
 * allocate device memory at all -- e.g. code running under another
 * framework's memory pool or a fixed pre-allocated budget, where cudaMalloc is
 * forbidden after start-up -- and so cannot create a handle.  It needs no
 * handle and calls no cudaMalloc, cudaFree or allocating library routine; the
 * caller passes every input and the output:
 *   dim, m1, n, T: as in pc_params (tau = T/(n+1), h = 1/(m1+1));
 *   a_int:  device, ms = m1^dim FP64, the coefficient a at the interior nodes
 *           (same spatial ordering as the vectors);
 *   x, lam: device all-at-once vectors (2*n*ms FP64);
 *   grad:   device, ms FP64, overwritten with the same quantity as pc_grad_log_a.
 * Scratch: the per-time-chunk partial sums live in one file-scope device array
 * of PC_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB) that every GPU loading the
 * library holds until exit.  m1^dim above that size is rejected with
 * PC_ERR_ARG, and so is n above PC_NOALLOC_MAX_N (a handle's limit); larger
 * n only coarsens the time chunks.  All calls on a device share the array and
 * it keeps the last call's contents (every entry a call reads it first writes,
 * so nothing needs clearing); calls whose execution overlaps on the GPU
 * (different streams without ordering) race on it.
 * Every call looks up the array's device address (cudaGetSymbolAddress) in the
 * context current at the call, so the device and context the caller has made
 * current are the ones used; the first call on a device loads the module there,
 * so make it before any stream capture. */
#define PC_NOALLOC_SCRATCH_DOUBLES (1 << 21)
#define PC_NOALLOC_MAX_N 4096
int pc_grad_log_a_noalloc(int dim, int m1, int n, double T, const double* a_int, const double* x,
                          const double* lam, double* grad, void* stream);

/* End-point values of the time discretisation (Section 1), which the
 * all-at-once unknowns leave out: from a solution x of A x = b (device,
 * 2*n*ms; y = x1 / sqrt(gamma), p = x2),
 *   (I + tau K) y^(N) = y^(n) + tau f_T + (tau / gamma) p_N,
 *   (I + tau K) p^(0) = p^(1) + tau g_0 - tau y0
 * (finite elements: M + tau K on the left, each right-hand side multiplied by M),
 * each solved to relative residual rtol by flexible conjugate gradients
 * preconditioned with the handle's spatial solver at shift 1 (exact for the
 * sine-transform handle, one V(1,0) cycle otherwise).  f_T, g_0, y0, p_N:
 * device, ms doubles each, or NULL for zero.  yN, p0: device outputs, ms
 * doubles.  *iters (may be NULL) = the larger of the two CG iteration counts.
 * Synchronises `stream`; uses the handle's Krylov workspace.  Errors:
 * PC_ERR_ARG, PC_ERR_NOT_CONVERGED (after maxit, 1..10000), PC_ERR_BREAKDOWN. */
int pc_end_point_solves(pc_handle* h, const double* x, const double* f_T, const double* g_0, const double* y0,
                        const double* p_N, double* yN, double* p0, double rtol, int maxit, int* iters,
                        void* stream);

/* Problem sizes of a handle: ms = m1^dim and the all-at-once length 2*n*ms. */
int pc_sizes(const pc_handle* h, int64_t* ms, int64_t* vec_len);

/* Tile shapes of the tunable kernels (an implementation choice: the paper has no
 * counterpart).  0 in any field means the built-in default.
 *   mg_cx:   fused 2D multigrid down leg (red-black sweep, residual and
 *            restriction of one level in one launch): coarse points per tile
 *            axis, 8 or 16 (default 16 in FP32, 8 in FP64).
 *   mg_ctas: CTAs per SM the fused down leg's grid is sized for, 1..64; it sets
 *            the spectral planes each CTA sweeps on every level (default 8).
 *   mv_tj:   time blocks per thread of the all-at-once matvec, 1..4096 (default 32).
 *   pro_pch: spectral planes per CTA of the prolongation and the 3D per-level
 *            multigrid kernels, 1..64 (default 8).
 *   fft_stream: time FFTs (power-of-two n): 0 = one CTA per tile of spatial
 *            columns (default), 1 = persistent CTAs that copy the next tile into
 *            shared memory (cp.async) while transforming the current one.
 *   mg_march: fused 2D down leg with FP32 iterates: 0 = shared-memory tiles
 *            (default), 1 = register-marching warps (a warp walks the rows of one
 *            plane over a 64-column strip; neighbours by lane shuffles).
 *   mg_seg:  register-marching down leg: coarse rows per warp, 1..1024 (default 16).
 *   fst_stream: sine-transform spatial solves, 0..3: persistent CTAs that copy
 *            the next tile of grid lines into shared memory (cp.async) while
 *            transforming the current one, for the single-axis passes (bit 0)
 *            and for the fused last-axis pass with the spectral divide (bit 1);
 *            one CTA per tile otherwise (default 0).
 * pc_set_tiles validates (PC_ERR_ARG), applies the shapes to every later call on
 * the handle and drops its cached solve graph.  pc_autotune times candidate
 * shapes on the handle's own workspace (the multigrid spatial step for each
 * (mg_cx, mg_ctas) and, with FP32 iterates, the register-marching kernel for each
 * mg_seg, then pro_pch; with sine-transform solves the spatial step for each
 * fst_stream; the forward + inverse time FFT for each fft_stream; the matvec
 * for each mv_tj), `reps` timed calls
 * each (1..100) after one untimed call, keeps the fastest, applies it and copies
 * it to *chosen (may be NULL).  It synchronises `stream`, overwrites the
 * handle's Krylov and spectral workspace (not the caller's vectors) and must not
 * run while `stream` is capturing or another call on the handle is in flight. */
typedef struct pc_tiles {
  int mg_cx;
  int mg_ctas;
  int mv_tj;
  int pro_pch;
  int fft_stream;
  int mg_march;
  int mg_seg;
  int fst_stream;
} pc_tiles;

int pc_get_tiles(const pc_handle* h, pc_tiles* out);
int pc_set_tiles(pc_handle* h, const pc_tiles* tiles);
int pc_autotune(pc_handle* h, int reps, pc_tiles* chosen, void* stream);

/* Instrumentation.  pc_profile(h, 1) starts recording a CUDA-event pair around
 * every kernel the handle launches (per kernel class); pc_profile(h, 0) stops.
 * pc_stats fills up to `cap` records (name, launches, summed device ms,
 * summed algorithmic DRAM bytes) and returns the number of classes; it
 * synchronises the events.  For the class "arnoldi_reorth" (the second
 * Gram-Schmidt pass, launched flag-gated every iteration) `launches` counts the
 * iterations in which it actually ran and `bytes` only their traffic.  pc_launch_count returns the number of kernels the
 * handle has launched since setup or pc_stats_reset. */
typedef struct pc_kernel_stat {
  char name[32];
  int64_t launches;
  double total_ms;      /* 0 unless profiling was on */
  double bytes;         /* algorithmic bytes moved (reads + writes of DRAM-resident data) */
  double flops;         /* algorithmic floating-point operations */
} pc_kernel_stat;

int pc_profile(pc_handle* h, int on);
/* Restrict the timing of pc_profile to the named kernel classes (comma-separated,
 * as pc_stats names them, e.g. "arnoldi_dot,arnoldi_update_norm"; NULL or "" times
 * every class).  Untimed classes still count launches, bytes and flops.  Fewer
 * event pairs leave the timed work closer to an unprofiled run.  PC_ERR_ARG for an
 * unknown name. */
int pc_profile_classes(pc_handle* h, const char* names);
int pc_stats(pc_handle* h, pc_kernel_stat* out, int cap, int* count);
int pc_stats_reset(pc_handle* h);
int64_t pc_launch_count(const pc_handle* h);

/* Arithmetic-rate probes (instrumentation; the paper has no counterpart): the
 * best of five CUDA-event-timed launches of register-only FMA chains (eight
 * independent chains per thread, grid of a few CTAs per SM), in TFLOP/s
 * (2 flops per FMA).  *fp64_tflops bounds the FP64 Arnoldi and matvec
 * kernels, whose FP64 operations per byte exceed the ridge point of a GPU
 * with a small FP64 unit.  Either output may be NULL (not both).  Synchronises
 * `stream`; takes tens of milliseconds. */
int pc_measure_peaks(double* fp64_tflops, double* fp32_tflops, void* stream);

/* Self-test of the bounded device waits (no paper counterpart): one CTA waits on
 * an mbarrier phase that cannot complete (64 bytes announced, 32 copied), gives
 * up after budget_ms (0 < budget_ms <= 10000) of SM clock, records the timeout
 * and returns, as the streamed Arnoldi kernels do if a copy never arrives.
 * Returns PC_ERR_TIMEOUT when the wait ran out as intended (the CUDA context stays
 * usable); PC_ERR_CUDA on a CUDA error.  Allocates nothing.  Synchronises `stream`. */
int pc_selftest_wait_timeout(double budget_ms, void* stream);

/* Debug build only (compiled with -DPCOPT_DEBUG, libpcopt_debug.so; no paper
 * counterpart): kernels check their index arithmetic (neighbour indices of the
 * stencils, basis-vector and tile indices of the Krylov kernels, time and column
 * indices of the time transforms), record the first failing check's code in a
 * device word and skip the access instead of trapping.  *code = that code (0: no
 * check failed; 1xx matvec, 2xx Krylov, 3xx time FFT); reset != 0 clears it.
 * Returns PC_OK in the debug build, PC_ERR_UNSUPPORTED (and *code = 0) in the
 * release build. */
int pc_debug_status(int reset, int* code);

/* Message of the calling thread's last error (never NULL). */
const char* pc_last_error(void);
const char* pc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PCOPT_H */
