// pc_grad_log_a_noalloc: the stencil-gradient kernel of pc_grad_log_a with its
// scratch (per-time-chunk partial sums) in a fixed file-scope device array, so
// that the call needs no handle and performs no device allocation.
//
// Who needs it: code that must not call cudaMalloc at all -- for example a
// caller that runs inside another framework's memory pool or a strict
// pre-allocated budget, or one whose allocation calls are forbidden after
// start-up.  Such a caller cannot create a handle (pc_setup allocates the
// Krylov workspace), but it can still own the inputs and the output buffer.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/pcopt.h"
#include "common.cuh"

using namespace pcopt;

// Shared scratch of every call on a device: PC_NOALLOC_SCRATCH_DOUBLES doubles
// (16 MiB).  Each GPU that loads the library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[PC_NOALLOC_SCRATCH_DOUBLES];

namespace {

// Device address of the scratch array in the context that is current now.
// Host code must not use the symbol itself (it is a host-side stand-in, not a
// device address).  The lookup is a cheap host call and is repeated on every
// call: an address cached per device ordinal would go stale when the caller
// switches to another context on that device or after cudaDeviceReset.
cudaError_t scratch_for_current_context(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" int pc_grad_log_a_noalloc(int dim, int m1, int n, double T, const double* a_int, const double* x,
                                     const double* lam, double* grad, void* stream) {
  if (dim != 2 && dim != 3) return set_error(PC_ERR_ARG, "pc_grad_log_a_noalloc: dim must be 2 or 3");
  if (m1 < 1 || n < 1 || !(T > 0) || !std::isfinite(T))
    return set_error(PC_ERR_ARG, "pc_grad_log_a_noalloc: need m1 >= 1, n >= 1, finite T > 0");
  if (n > PC_NOALLOC_MAX_N)  // the same limit as a handle's n
    return set_error(PC_ERR_ARG, "pc_grad_log_a_noalloc: n = " + std::to_string(n) + " exceeds " +
                                     std::to_string(PC_NOALLOC_MAX_N));
  if (!a_int || !x || !lam || !grad) return set_error(PC_ERR_ARG, "pc_grad_log_a_noalloc: null pointer");
  const int64_t ms = dim == 2 ? (int64_t)m1 * m1 : (int64_t)m1 * m1 * m1;
  if (ms > (int64_t)PC_NOALLOC_SCRATCH_DOUBLES)  // one time chunk of partial sums must fit
    return set_error(PC_ERR_ARG, "pc_grad_log_a_noalloc: m1^dim = " + std::to_string(ms) +
                                     " exceeds the static scratch of " +
                                     std::to_string((long long)PC_NOALLOC_SCRATCH_DOUBLES) + " doubles");
  // time chunk of 16 blocks, as pc_grad_log_a, enlarged until the partial sums
  // fit the scratch and the chunk count fits the grid's y extent (65535)
  int64_t max_chunks = (int64_t)PC_NOALLOC_SCRATCH_DOUBLES / ms;
  if (max_chunks > 65535) max_chunks = 65535;
  int64_t tj = 16;
  if (((int64_t)n + tj - 1) / tj > max_chunks) tj = ((int64_t)n + max_chunks - 1) / max_chunks;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_context(&scratch);
  if (e != cudaSuccess)
    return set_error(PC_ERR_CUDA, std::string("pc_grad_log_a_noalloc: scratch address: ") + cudaGetErrorString(e));
  Launch L{(cudaStream_t)stream, nullptr};
  Grid g;
  g.dim = dim;
  g.m = m1;
  g.np = ms;
  const double tau = T / (n + 1);
  const double h = 1.0 / (m1 + 1);
  e = launch_grad_chunked(L, g, n, -tau * 0.5 / (h * h), a_int, x, lam, scratch, (int)tj, grad);
  if (e != cudaSuccess)
    return set_error(PC_ERR_CUDA, std::string("pc_grad_log_a_noalloc: ") + cudaGetErrorString(e));
  return PC_OK;
}
