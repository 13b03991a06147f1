// Reciprocal of a pivot (device code shared by the factor kernels).
#pragma once

namespace kkt {

// FP64: the Newton-Raphson iteration for 1/d, y <- y + y (1 - d y), twice from
// a single-precision seed (each step squares the relative error: 2^-23 ->
// 2^-46 -> 2^-92, so the result is within an ulp or so of 1/d), about half the
// latency of a double division on this GPU.  Pivots outside the
// single-precision normal range use the division.
__device__ __forceinline__ double pivot_recip(double d) {
  const double ad = fabs(d);
  if (!(ad > 1e-36 && ad < 1e36)) return 1.0 / d;
  double y = (double)__frcp_rn((float)d);
  y = fma(y, fma(-d, y, 1.0), y);
  y = fma(y, fma(-d, y, 1.0), y);
  return y;
}
__device__ __forceinline__ float pivot_recip(float d) { return __frcp_rn(d); }

}  // namespace kkt
