// kc_probe.cu -- throughput probe of the FP32 and FP64 FMA pipes, the
// denominators of the rooflines (the FP64 rate of this GPU is not in the
// vendor's public tables at the precision needed, so it is measured).
//
// One CTA of 1024 threads per SM; every thread runs eight independent FMA
// chains, so issue is never latency-bound; thread 0 of each CTA reads the
// SM clock around the loop.  Rate = FMAs executed by the CTA / its cycles.
#include <cstdint>

#include "kc_internal.h"

namespace kc {

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(1024) fma_probe_kernel(int iters, T *__restrict__ sink,
                                                         long long *__restrict__ cycles) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x) * T(1e-7) + T(i);
  const T a = T(0.999999), b = T(1e-6);
  __syncthreads();
  const long long c0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  __syncthreads();
  const long long c1 = clock64();
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;       // keeps the chains live
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

}  // namespace

cudaError_t probe_fma_rate(bool f64, int n_sm, int iters, void *sink, long long *cycles,
                           cudaStream_t st) {
  if (f64)
    fma_probe_kernel<double><<<n_sm, 1024, 0, st>>>(iters, static_cast<double *>(sink), cycles);
  else
    fma_probe_kernel<float><<<n_sm, 1024, 0, st>>>(iters, static_cast<float *>(sink), cycles);
  return cudaGetLastError();
}

}  // namespace kc
