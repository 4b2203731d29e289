// Double-precision reciprocal, square root and reciprocal cube root for the
// element kernels, built for GB300's narrow FP64 pipe: a low-precision seed
// from the hardware approximation units (which run beside the FP64 pipe),
// then ONE cubically convergent correction in double precision.
//
// Methods (textbook series corrections, one step each):
//  * reciprocal 1/x: seed r, e = 1 - x r, r' = r (1 + e + e^2)
//    (the geometric series of 1/(1 - e) truncated after e^2); error O(e^3);
//  * square root sqrt(s): seed y ~ s^(-1/2), n = s y, e = 1 - n y (= 1 - s y^2),
//    n' = n (1 + e/2 + 3 e^2/8) (binomial series of (1 - e)^(-1/2)); O(e^3);
//  * reciprocal cube root x^(-1/3): seed y, e = 1 - x y^3,
//    y' = y (1 + e/3 + 2 e^2/9) (binomial series of (1 - e)^(-1/3)); O(e^3).
// With seeds good to about 2^-20 the corrected results are within a few
// units in the last place of the correctly rounded values (tests compare them
// with CUDA's own division, sqrt and rcbrt). Each costs 3, 5 and 6 FP64
// instructions (the inverse square root, 5).
//
// Domains: rcp_pos and rcbrt_pos take finite x > 0 (the callers guarantee
// it); sqrt_nonneg takes s >= 0 and returns 0 for zero and subnormal s.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

namespace nsrhs {

#if defined(__CUDA_ARCH__)

// Exact float -> double widening with integer operations only (keeps the
// conversion off the FP64 pipe). Subnormal floats are flushed to signed zero.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  unsigned lo = b << 29;
  if (ex == 0u) {
    hi = b & 0x80000000u;
    lo = 0u;
  } else if (ex == 255u) {
    hi = (b & 0x80000000u) | 0x7ff00000u | ((b & 0x7fffffu) >> 3);
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double rcp_pos(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  const double e2 = fma(e, e, e);
  return fma(r, e2, r);
}

__device__ __forceinline__ double sqrt_nonneg(double s) {
  // zero and subnormal inputs (high word below the smallest normal) -> 0
  const bool tiny = __double2hiint(s) < 0x00100000;
  const double ss = tiny ? 1.0 : s;
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(ss));
  const double n = ss * y;
  const double e = fma(-n, y, 1.0);
  const double p = fma(0.375, e, 0.5);
  const double r = fma(n * e, p, n);
  return tiny ? 0.0 : r;
}

// 1/sqrt(s): seed y, e = 1 - s y^2, y' = y (1 + e/2 + 3 e^2/8); 0 for zero and
// subnormal s (so that s * rsqrt_nonneg(s) = 0 there).
__device__ __forceinline__ double rsqrt_nonneg(double s) {
  const bool tiny = __double2hiint(s) < 0x00100000;
  const double ss = tiny ? 1.0 : s;
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(ss));
  const double e = fma(-ss, y * y, 1.0);
  const double p = fma(0.375, e, 0.5);
  const double r = fma(y * e, p, y);
  return tiny ? 0.0 : r;
}

__device__ __forceinline__ double rcbrt_pos(double x) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7ff;
  // float seed from the leading 20 mantissa bits; outside the float
  // exponent range use the library function
  if (ex < 897 || ex > 1150) return rcbrt(x);
  const float xf = __int_as_float(((ex - 896) << 23) | ((hi & 0xfffff) << 3));
  const double y = widen_f32(rcbrtf(xf));
  const double y3 = (y * y) * y;
  const double e = fma(-x, y3, 1.0);
  const double p = fma(2.0 / 9.0, e, 1.0 / 3.0);
  return fma(y * e, p, y);
}

#else  // host compilation of the same sources (flop census, host probes)

inline double widen_f32(float f) { return (double)f; }
inline double rcp_pos(double x) { return 1.0 / x; }
inline double sqrt_nonneg(double s) { return s > 0.0 ? sqrt(s) : 0.0; }
inline double rcbrt_pos(double x) { return 1.0 / cbrt(x); }
inline double rsqrt_nonneg(double s) { return s > 0.0 ? 1.0 / sqrt(s) : 0.0; }

#endif

}  // namespace nsrhs
