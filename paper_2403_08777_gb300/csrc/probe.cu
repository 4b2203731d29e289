// FMA-throughput probes for the roofline denominators (see nsrhs_probe.h).

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/nsrhs_probe.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int64_t iters, T a, T b, double* sink) {
  // 8 independent chains per thread hide the pipe latency.
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int64_t i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] =
      (double)(((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7)));
}

}  // namespace

extern "C" int nsrhs_probe_fma(int fp64, int64_t blocks, int64_t iters, double* sink,
                               void* stream) {
  if (blocks < 1 || blocks > (1 << 24) || iters < 1 || !sink) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  // a slightly below 1 keeps the chains bounded and away from denormals
  if (fp64)
    fma_chain_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(iters, 0.999999, 1e-6, sink);
  else
    fma_chain_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(iters, 0.999999f, 1e-6f, sink);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
