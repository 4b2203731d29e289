// FMA-throughput probes for the roofline denominators (see nsrhs_probe.h).

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/nsrhs_probe.h"
#include "fastmath.cuh"

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int64_t iters, T a, T b, double* sink) {
  // 16 independent dependent chains per thread, loop unrolled, so that the
  // FMA pipe (not latency or loop overhead) limits the rate.
  T x[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) x[c] = (T)threadIdx.x * (T)1e-3 + (T)c;
#pragma unroll 4
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 16; ++c) x[c] = fma(x[c], a, b);
  }
  T acc = (T)0;
#pragma unroll
  for (int c = 0; c < 16; ++c) acc += x[c];
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = (double)acc;
}

// y[i] = f(x[i]) with this library's function and with CUDA's.
__global__ void special_kernel(int which, int64_t n, const double* __restrict__ x,
                               double* __restrict__ ours, double* __restrict__ ref) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    switch (which) {
      case 0:
        ours[i] = nsrhs::rcp_pos(v);
        ref[i] = 1.0 / v;
        break;
      case 1:
        ours[i] = nsrhs::sqrt_nonneg(v);
        ref[i] = sqrt(v);
        break;
      case 2:
        ours[i] = nsrhs::rcbrt_pos(v);
        ref[i] = rcbrt(v);
        break;
      default: {
        const float f = __double2float_rn(v);
        ours[i] = nsrhs::widen_f32(f);
        ref[i] = (double)f;
      }
    }
  }
}

}  // namespace

extern "C" int nsrhs_probe_special(int which, int64_t n, const double* x, double* ours,
                                   double* ref, void* stream) {
  if (which < 0 || which > 3 || n < 1 || !x || !ours || !ref) return 1;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  special_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(which, n, x, ours, ref);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

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
