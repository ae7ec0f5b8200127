// pc_measure_peaks: arithmetic-rate probes of the GPU the library runs on.
//
// The Arnoldi passes of the solver do two FP64 operations per 8 bytes they
// read, which is above the FP64 ridge point of a GPU whose FP64 unit is small
// next to its HBM bandwidth; their roofline is then the FP64 FMA rate, which
// these kernels measure: long independent FMA chains per thread, registers
// only, no memory traffic in the timed loop.  The paper has no counterpart.
#include <cuda_runtime.h>

#include <string>

#include "../../include/pcopt.h"
#include "common.cuh"

using namespace pcopt;

namespace {

// Written only when a chain ends on a value the inputs cannot produce, so the
// compiler must keep every FMA; never read.
__device__ double g_peak_sink64;
__device__ float g_peak_sink32;

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma64_probe_kernel(int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0) g_peak_sink64 = s;
}

__global__ void __launch_bounds__(256) fma32_probe_kernel(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0f + 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) g_peak_sink32 = s;
}

// best-of-`reps` rate in TFLOP/s of one probe launch (2 flops per FMA)
template <typename Kern>
cudaError_t time_probe(Kern launch, cudaStream_t st, double flops, int reps, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  double best = 0.0;
  launch();  // warm-up (clocks ramp, module load)
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f) {
      const double t = flops / (ms * 1e-3) / 1e12;
      if (t > best) best = t;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return e;
}

}  // namespace

extern "C" int pc_measure_peaks(double* fp64_tflops, double* fp32_tflops, void* stream) {
  if (!fp64_tflops && !fp32_tflops) return set_error(PC_ERR_ARG, "pc_measure_peaks: no output");
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = num_sms();
  const int threads = 256;
  cudaError_t e = cudaSuccess;
  if (fp64_tflops) {
    // 4 CTAs of 8 warps per SM keep the small FP64 unit busy; ~10 ms per launch
    const int blocks = sms * 4, iters = 4096;
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    e = time_probe([&] { fma64_probe_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7); }, st, flops, 5,
                   fp64_tflops);
  }
  if (e == cudaSuccess && fp32_tflops) {
    const int blocks = sms * 8, iters = 65536;
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    e = time_probe([&] { fma32_probe_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-7f); }, st, flops, 5,
                   fp32_tflops);
  }
  if (e != cudaSuccess)
    return set_error(PC_ERR_CUDA, std::string("pc_measure_peaks: ") + cudaGetErrorString(e));
  return PC_OK;
}
