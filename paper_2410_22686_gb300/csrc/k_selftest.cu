// Self-tests of the library's failure paths, run on the GPU without faulting it.
//
// pc_selftest_wait_timeout: one CTA announces 64 bytes on an mbarrier and
// copies only 32 with a bulk asynchronous copy, so the phase can never
// complete; its bounded wait must give up after the budget, record the
// timeout in the error word and return.  The copy that was issued has landed
// by then, so nothing is in flight when the CTA exits.  This is the path the
// streamed Arnoldi kernels take if a copy ever fails to arrive.  No device
// memory is allocated: source and error word are file-scope device variables.
#include <cuda_runtime.h>

#include <string>

#include "../../include/pcopt.h"
#include "common.cuh"
#include "tma.cuh"

using namespace pcopt;

namespace {

__device__ __align__(16) float g_probe_src[8];
__device__ double g_probe_err;

__global__ void wait_timeout_probe_kernel(const float* src, double* err, long long budget) {
  __shared__ __align__(16) float buf[16];
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    *err = 0.0;
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, 64);      // 64 bytes announced ...
    bulk_copy_g2s(buf, src, 32, &bar);    // ... 32 delivered
  }
  // every thread's wait is bounded; the first to give up records the timeout
  if (!mbar_wait_bounded(&bar, 0, nullptr, 0.0, budget)) *err = kErrWaitTimeout;
  __syncthreads();
}

}  // namespace

extern "C" int pc_selftest_wait_timeout(double budget_ms, void* stream) {
  if (!(budget_ms > 0.0) || budget_ms > 10000.0)
    return set_error(PC_ERR_ARG, "pc_selftest_wait_timeout: budget_ms must be in (0, 10000]");
  int dev = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  void* src = nullptr;
  void* err = nullptr;
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&src, g_probe_src);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&err, g_probe_err);
  if (e != cudaSuccess) return set_error(PC_ERR_CUDA, std::string("pc_selftest_wait_timeout: ") + cudaGetErrorString(e));
  const long long budget = (long long)(budget_ms * (khz > 0 ? khz : 2000000));
  cudaStream_t st = (cudaStream_t)stream;
  wait_timeout_probe_kernel<<<1, 64, 0, st>>>((const float*)src, (double*)err, budget);
  double h = 0.0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(PC_ERR_CUDA, std::string("pc_selftest_wait_timeout: ") + cudaGetErrorString(e));
  if (h != 0.0) return set_error(PC_ERR_TIMEOUT, "pc_selftest_wait_timeout: the bounded wait ran out (as intended)");
  return set_error(PC_ERR_ARG, "pc_selftest_wait_timeout: the wait completed although it could not");
}
