// The square root of the observables' lengths: an FP32 seed refined in FP64.
// Shared by the observables kernels and the accuracy test's export.
#pragma once

#include "log_fp64.cuh"

namespace gaps {

// sqrt(x) of the observables' lengths (|p|, |P|, |p x n_T|) to 1.5e-13
// relative: the FP32 reciprocal square root y0 = x^-1/2 (1 + e0) (two FP32
// ulps, plus the rounding of x to FP32: |e0| < 2.5 2^-23) refined by one
// Newton step in FP64, which leaves sqrt(x) (1 - 1.5 e0^2 + O(e0^3)) plus
// the step's own roundings.  Three FP64 operations against the ten-FMA cost
// of a correctly rounded FP64 square root on this part.  What it moves: T
// by 3e-13 at most; on y_ij = 2 min(E^2) (1 - cos)/s the cosine by 3e-13
// absolute, so y by 2 min(E^2)/s x 3e-13 <= 1.5e-13 absolute; B_T and B_W
// by 3e-13 relative.  Zero, negative, non-finite and extreme x (outside
// 2^-120 .. 2^120, where the FP32 seed would leave FP32's normal range)
// take the library square root.
__device__ __forceinline__ double sqrt_obs(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned ex = static_cast<unsigned>(b >> 52);  // sign and exponent field
  if (ex < 1023u - 120u || ex > 1023u + 120u) return sqrt(x);
  const unsigned y0f = __float_as_uint(rsqrtf(f32_from_f64(x)));
  // y0 and y0 / 2 as doubles, assembled from the FP32 bits (positive normal
  // floats: exponent rebiased by 1023 - 127, mantissa moved up 29 bits)
  const unsigned long long man = static_cast<unsigned long long>(y0f & 0x7fffffu) << 29;
  const unsigned long long e64 = static_cast<unsigned long long>((y0f >> 23) + 896u);
  const double y0 = __longlong_as_double(static_cast<long long>((e64 << 52) | man));
  const double y0h = __longlong_as_double(static_cast<long long>(((e64 - 1ull) << 52) | man));
  const double h = x * y0;                  // sqrt(x) (1 + e0)
  const double rh = fma(-h, y0h, 0.5);      // (1 - x y0^2) / 2
  return fma(h, rh, h);
}

}  // namespace gaps
