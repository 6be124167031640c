/* FP64 helpers that keep work off the GB300's narrow FP64 pipe.
 *
 * Comparisons, min/max and sign tests of doubles run on the integer pipe: for non-NaN
 * doubles the map okey(x) = bits(x) XOR (sign(x) ? 0x7fff...f : 0) is monotone, so
 * x < y  <=>  okey(x) < okey(y) as signed 64-bit integers (with -0 ordered just below +0).
 * For non-negative doubles the raw bit patterns are already ordered.
 *
 * Reciprocals use Newton-Raphson iteration for 1/x (y <- y + y (1 - x y), quadratic
 * convergence) started from the PTX rcp.approx.ftz.f64 estimate; two steps reach the
 * rounding level (checked against CUDA's 1.0/x by the GPU tests).  Square root and its
 * reciprocal use Newton iteration for 1/sqrt(x) (y <- y + y (1/2 - x y^2 / 2)) from the
 * PTX rsqrt.approx.ftz.f64 estimate.
 */
#pragma once
#include <cstdint>

namespace tenom {

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

/* x < y for non-NaN doubles, on the integer pipe */
__device__ __forceinline__ bool ilt(double x, double y) { return okey(x) < okey(y); }
__device__ __forceinline__ double imin(double a, double b) { return ilt(b, a) ? b : a; }
__device__ __forceinline__ double imax(double a, double b) { return ilt(a, b) ? b : a; }
/* strict sign tests (+0 and -0 are neither positive nor negative) */
__device__ __forceinline__ bool ipos(double x) { return dbits(x) > 0; }
__device__ __forceinline__ bool ineg(double x) { return (unsigned long long)dbits(x) > 0x8000000000000000ull; }
__device__ __forceinline__ double iabs(double x) { return __longlong_as_double(dbits(x) & 0x7fffffffffffffffll); }
/* max of non-negative doubles: raw bits are ordered */
__device__ __forceinline__ double imax_nonneg(double a, double b) { return dbits(a) < dbits(b) ? b : a; }
/* a < b for non-negative doubles (including +inf) */
__device__ __forceinline__ bool ilt_nonneg(double a, double b) { return dbits(a) < dbits(b); }

__device__ __forceinline__ double rcp_approx(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ double rsqrt_approx(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

/* 1/x by two Newton-Raphson steps (finite, normal, nonzero x) */
__device__ __forceinline__ double rcp_nr(double x) {
  double y = rcp_approx(x);
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

/* 1/x by one Newton-Raphson step: for quantities that only feed a comparison
   (the cutoff's gamma_k, TENO8A's eta); accuracy checked by the GPU tests */
__device__ __forceinline__ double rcp_nr1(double x) {
  const double y = rcp_approx(x);
  return fma(y, fma(-x, y, 1.0), y);
}

/* 1/sqrt(x) by two Newton steps for positive normal x; sqrt(x) = x * rsqrt(x) */
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = rsqrt_approx(x);
  const double h = 0.5 * x;
  double r = fma(-h, y * y, 0.5);
  y = fma(y, r, y);
  r = fma(-h, y * y, 0.5);
  return fma(y, r, y);
}

/* FP64 -> FP32 rounded toward zero, on the integer pipe (the F2F conversion instruction runs
   on the FP64 pipe, the scarce unit here).  |x - f| < 2^-23 |x| in the FP32 normal range;
   magnitudes below it become a signed zero, above it (and NaN) infinity. */
__device__ __forceinline__ float f32_rz(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | m);
}

}  // namespace tenom
