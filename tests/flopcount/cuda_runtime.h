// Host stand-in for <cuda_runtime.h>, used only to compile the element
// arithmetic as host code with a counting scalar type (flop census).
#pragma once
#include <cmath>
#define __device__
#define __forceinline__ inline
inline double rcbrt(double x) { return 1.0 / std::cbrt(x); }
inline float rcbrtf(float x) { return 1.0f / std::cbrt(x); }
inline float __frcp_rn(float x) { return 1.0f / x; }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
using std::sqrt;
