// af_math.cuh -- FP64 helpers for an FP64-starved GPU.
//
// On GB300 the FP64 pipe issues about 1.65 DFMA/DADD/DMUL per SM per clock,
// and a compiler double division or square root costs about 8.6 of those,
// while FP32 and integer work is ~67x cheaper.  The helpers below keep the
// FP64 instruction count down:
//   * rcp/ddiv/dsqrt: an FP32 hardware seed (rcp.approx / rsqrt.approx on the
//     double's leading bits, converted with integer bit operations) refined by
//     Newton-Raphson iterations in FP64 (the classical Newton reciprocal and
//     Heron square-root iterations, e.g. P. Markstein, IBM J. Res. Dev. 34(1),
//     1990).  Each costs 4-5 FP64 instructions and is accurate to about one
//     ulp; outside the FP32 exponent range they fall back to the exact
//     operators.
//   * maxnn/minnn/absd: min/max/abs of doubles on the integer pipe (valid for
//     non-negative, non-NaN operands where stated).
#pragma once
#include <cuda_runtime.h>

namespace afm {

__device__ __forceinline__ unsigned hi32(double x) { return (unsigned)__double2hiint(x); }

// x == +0 or -0, on the integer pipe
__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }

// true when the FP32 seed path is valid: 2^-123 <= |x| < 2^124
__device__ __forceinline__ bool seed_ok(double x) {
  unsigned e = (hi32(x) >> 20) & 0x7ffu;
  return (e - 900u) <= 246u;
}

// leading 24 bits of a double in seed_ok range, as an FP32 value (truncated)
__device__ __forceinline__ float seed_f32(double x) {
  unsigned hi = hi32(x), lo = (unsigned)__double2loint(x);
  unsigned fb = ((((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29)) | (hi & 0x80000000u);
  return __uint_as_float(fb);
}

// exact widening of a normal FP32 value to FP64
__device__ __forceinline__ double widen_f32(float f) {
  unsigned fb = __float_as_uint(f);
  unsigned hi = (((fb & 0x7fffffffu) >> 3) + (896u << 20)) | (fb & 0x80000000u);
  return __hiloint2double((int)hi, (int)(fb << 29));
}

__device__ __forceinline__ float rcp_approx_f32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx_f32(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/x: two Newton steps y <- y + y (1 - x y) from the FP32 seed.
__device__ __forceinline__ double rcp(double x) {
  if (!seed_ok(x)) return 1.0 / x;
  double y = widen_f32(rcp_approx_f32(seed_f32(x)));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// a/b: one Newton step on the seed, then one residual correction of the quotient.
__device__ __forceinline__ double ddiv(double a, double b) {
  if (!seed_ok(b)) return a / b;
  double y = widen_f32(rcp_approx_f32(seed_f32(b)));
  double e = fma(-b, y, 1.0);
  y = fma(y, e, y);
  double q = a * y;
  double r = fma(-b, q, a);
  return fma(r, y, q);
}

// sqrt(x): s = x * rsqrt-seed, then two Heron corrections s <- s + (x - s^2)/(2 s)
// with 1/(2 s) taken from the seed.
__device__ __forceinline__ double dsqrt(double x) {
  if (!seed_ok(x)) return is_zero(x) ? x : sqrt(x);   // sqrt(+-0) = +-0
  float yf = rsqrt_approx_f32(seed_f32(x));
  double y = widen_f32(yf), h = widen_f32(0.5f * yf);
  double s = x * y;
  double r = fma(-s, s, x);
  s = fma(r, h, s);
  r = fma(-s, s, x);
  return fma(r, h, s);
}

// max/min of non-negative, non-NaN doubles via their bit patterns
__device__ __forceinline__ double maxnn(double a, double b) {
  long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}
__device__ __forceinline__ double minnn(double a, double b) {
  long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x < y ? x : y);
}
__device__ __forceinline__ double absd(double a) {
  return __hiloint2double(__double2hiint(a) & 0x7fffffff, __double2loint(a));
}
// finite (neither infinite nor NaN), from the exponent bits
__device__ __forceinline__ bool finite_bits(double a) { return ((hi32(a) >> 20) & 0x7ffu) != 0x7ffu; }
// a == 1.0 and a < 1.0 for non-negative a, +NaN included (bit-pattern comparisons on the
// integer pipe)
__device__ __forceinline__ bool is_one(double a) { return __double_as_longlong(a) == 0x3ff0000000000000LL; }
__device__ __forceinline__ bool lt_one(double a) { return __double_as_longlong(a) < 0x3ff0000000000000LL; }
// a < 0 for non-NaN a (negative zero is not negative)
__device__ __forceinline__ bool isneg(double a) {
  long long x = __double_as_longlong(a);
  return x < 0 && (x & 0x7fffffffffffffffLL) != 0;
}

}  // namespace afm
