// fp64_recip.cuh — the double-precision reciprocal and reciprocal square
// root of the FP64 flux arithmetic, and the wave-speed maximum taken on the
// integer pipes.
//
// Each takes the hardware's approximate value (rcp.approx.ftz.f64,
// rsqrt.approx.ftz.f64: correct to about 2^-23 relative) and refines it with
// one third-order Householder step, the cubic-convergence form of Newton's
// method for 1/x and 1/sqrt(x):
//   1/x       = y / (1 - e)         = y (1 + e + e^2 + ...),        e = 1 - x y,
//   1/sqrt(x) = y / sqrt(1 - e)     = y (1 + e/2 + 3 e^2 / 8 + ...), e = 1 - x y^2.
// Truncating after e^2 leaves a relative error near e^3 (about 2^-69), so the
// result is within about one unit in the last place of the exact value: not
// correctly rounded, and not required to be (the flux formulas round more
// than that in every step). The fused multiply-adds are explicit, so every
// kernel that includes this file rounds them identically. Subnormal inputs
// and results are flushed to zero; zero, negative, infinite and NaN inputs
// give a non-finite result, which the step's monitoring reports.
#pragma once

namespace mprk {

__device__ __forceinline__ double rcp_approx_f64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ double rsqrt_approx_f64(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

// 1/x: y (1 + e + e^2) as y + y (e + e^2)
__device__ __forceinline__ double recip_f64(double x) {
  const double y = rcp_approx_f64(x);
  const double e = __fma_rn(-x, y, 1.0);
  return __fma_rn(y, __fma_rn(e, e, e), y);
}

// 1/sqrt(x): y (1 + e/2 + 3 e^2/8) as y + (y e) (1/2 + 3 e/8)
__device__ __forceinline__ double rsqrt_f64(double x) {
  const double y = rsqrt_approx_f64(x);
  const double e = __fma_rn(-__dmul_rn(x, y), y, 1.0);
  return __fma_rn(__dmul_rn(y, e), __fma_rn(0.375, e, 0.5), y);
}

// sqrt(x) = x / sqrt(x): the same step applied to t = x y, the
// approximation of sqrt(x) that the rsqrt iteration forms anyway:
// t (1 + e/2 + 3 e^2/8) with e = 1 - t y.
__device__ __forceinline__ double sqrt_f64(double x) {
  const double y = rsqrt_approx_f64(x);
  const double t = __dmul_rn(x, y);
  const double e = __fma_rn(-t, y, 1.0);
  return __fma_rn(__dmul_rn(t, e), __fma_rn(0.375, e, 0.5), t);
}

// The larger of two wave speeds |u_n| + a, both >= 0. For doubles the IEEE
// bit patterns of non-negative values order as signed integers, so the
// comparison runs on the integer pipes and leaves the FP64 pipe (two
// operations per clock per SM on this GPU) to the arithmetic; the result is
// the same value.
__device__ __forceinline__ double max_speed(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}
__device__ __forceinline__ float max_speed(float a, float b) { return fmaxf(a, b); }

}  // namespace mprk
