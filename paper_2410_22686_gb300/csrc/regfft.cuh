// Radix-2 FFT of a small power-of-two length held in registers (one thread
// owns the whole sequence) and the cp.async helpers, shared by the time FFTs and
// the sine transforms.
#pragma once

#include "common.cuh"

namespace pcopt {

template <int R>
__device__ __forceinline__ constexpr int brev_ct(int i) {
  int r = 0;
  for (int b = 1, rb = R >> 1; b < R; b <<= 1, rb >>= 1)
    if (i & b) r |= rb;
  return r;
}

// in-place R-point DFT of registers x (DIT, radix 2); twiddles exp(-+2 pi i q/R)
// are tw[q * tstride] from the full-circle table of length n = R * tstride
template <int R, bool INV, typename C>
__device__ __forceinline__ void reg_fft(C (&x)[R], const C* __restrict__ tw, int tstride) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = brev_ct<R>(i);
    if (j > i) {
      const C t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < R; half <<= 1) {
#pragma unroll
    for (int g = 0; g < R; g += 2 * half) {
#pragma unroll
      for (int p = 0; p < half; ++p) {
        const C a = x[g + p];
        C b = x[g + p + half];
        if (p != 0) {
          C w = tw[p * (R / (2 * half)) * tstride];
          if (INV) w.y = -w.y;
          b = cmul(w, b);
        }
        x[g + p] = a + b;
        x[g + p + half] = a - b;
      }
    }
  }
}

// cp.async (sm_80+ asynchronous global -> shared copy of B = 4, 8 or 16 bytes,
// bypassing registers); `ok == false` zero-fills the destination without reading
// global memory
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = ok ? B : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(B), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace pcopt
