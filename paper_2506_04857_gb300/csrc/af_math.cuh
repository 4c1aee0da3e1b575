// af_math.cuh -- FP64 helpers for an FP64-starved GPU.
//
// On GB300 the FP64 pipe issues about 1.65 DFMA/DADD/DMUL per SM per clock,
// and a compiler double division or square root costs about 8.6 of those,
// while FP32 and integer work is ~67x cheaper.  The helpers below keep the
// FP64 instruction count down:
//   * rcp/ddiv/dsqrt: an FP32 hardware seed (rcp.approx / rsqrt.approx on the
//     double's leading bits, converted with integer bit operations) refined by
//     one Newton-Raphson step in FP32 on the double split into two floats and
//     one in FP64 (the classical Newton reciprocal and Heron square-root
//     iterations, e.g. P. Markstein, IBM J. Res. Dev. 34(1), 1990).  Each costs
//     2 FP64 instructions and is within one ulp; outside 2^-63 <= |x| < 2^78
//     they take two FP64 steps (4 instructions), outside the FP32 exponent
//     range the exact operators.
//   * maxnn/minnn/absd and the compares ge_pos/gt_pos/ge_zero/ge_i: on the
//     integer pipe, through an opaque move of the bit pattern (valid for
//     non-negative, non-NaN operands where stated; the compares for every input).
//   * mul_i/add_i: correctly rounded binary64 product and sum computed with
//     integer instructions only, for code that is bound by the FP64 pipe while
//     the integer pipes idle (GB300 has 2 FP64 lanes per SM against 64 integer
//     ones).  Their results are bitwise those of DMUL/DADD; a kernel that moves
//     part of its products and sums onto them runs both pipes at once.
#pragma once
#include <cuda_runtime.h>

namespace afm {

__device__ __forceinline__ unsigned hi32(double x) { return (unsigned)__double2hiint(x); }

// The bit pattern of a double and back.  The move is opaque to the compiler, so
// integer tests on the pattern stay integer instructions (a plain bit cast lets
// the compiler turn e.g. (bits << 1) == 0 back into an FP64 compare).
__device__ __forceinline__ unsigned long long bits(double x) {
  unsigned long long r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double from_bits(unsigned long long u) {
  double r;
  asm("mov.b64 %0, %1;" : "=d"(r) : "l"(u));
  return r;
}

// x == +0 or -0, on the integer pipe
__device__ __forceinline__ bool is_zero(double x) { return (bits(x) << 1) == 0; }
// x > 0 (false for NaN), on the integer pipe: the patterns of +min subnormal .. +inf
__device__ __forceinline__ bool gt_zero(double x) { return bits(x) - 1ULL < 0x7ff0000000000000ULL; }

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
__device__ __forceinline__ double rcp_nr2(double x) {
  if (!seed_ok(x)) return 1.0 / x;
  double y = widen_f32(rcp_approx_f32(seed_f32(x)));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// a/b: one Newton step on the seed, then one residual correction of the quotient.
__device__ __forceinline__ double ddiv_nr(double a, double b) {
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
__device__ __forceinline__ double dsqrt_nr2(double x) {
  if (!seed_ok(x)) return is_zero(x) ? x : sqrt(x);   // sqrt(+-0) = +-0
  float yf = rsqrt_approx_f32(seed_f32(x));
  double y = widen_f32(yf), h = widen_f32(0.5f * yf);
  double s = x * y;
  double r = fma(-s, s, x);
  s = fma(r, h, s);
  r = fma(-s, s, x);
  return fma(r, h, s);
}

// ---- seeds refined once in FP32 ------------------------------------------
// A double x is split into two floats, xh (its leading 24 significand bits) and xl
// (the next 24, truncated): |x - xh - xl| < 2^-47 |x|.  One Newton (or Heron) step
// taken in FP32 on the pair carries the FP32 seed from about 23 to about 44 bits;
// one FP64 step then leaves the result within one ulp (its error is the square of
// 2^-44 plus the final rounding), so a reciprocal, quotient or square root costs
// two FP64 instructions instead of four.  Valid for 2^-63 <= |x| < 2^78, where
// every float involved is normal; elsewhere the two-step forms above.
__device__ __forceinline__ bool split_f32(double x, float &xh, float &xl) {
  const unsigned long long b = bits(x);
  const unsigned hi = (unsigned)(b >> 32), e = (hi >> 20) & 0x7ffu;
  if (e - 960u > 140u) return false;
  xh = seed_f32(x);
  // the 29 significand bits below xh, times 2^(e - 1075) (an exact power of two)
  const float scale = __uint_as_float(((e - 948u) << 23) | (hi & 0x80000000u));
  xl = __uint2float_rn((unsigned)b & 0x1fffffffu) * scale;
  return true;
}
// y + c as a double for floats with |c| <= 2^-20 |y|, y normal: the significand of
// c aligned to that of y and added as an integer (bits of c below 2^-52 |y| are
// dropped, which the FP64 step that follows absorbs).
__device__ __forceinline__ double join_f32(float y, float c) {
  const unsigned a = __float_as_uint(y), bc = __float_as_uint(c);
  const unsigned ea = (a >> 23) & 0xffu, eb = (bc >> 23) & 0xffu;
  unsigned long long M = (unsigned long long)((a & 0x7fffffu) | 0x800000u) << 29;   // leading one at bit 52
  const unsigned sh = ea - eb;                                                        // c's at bit 52 - sh
  const unsigned long long mc0 = (unsigned long long)((bc & 0x7fffffu) | 0x800000u);
  unsigned long long mc = sh <= 29u ? (mc0 << (29u - sh)) : (sh < 53u ? (mc0 >> (sh - 29u)) : 0ULL);
  mc = eb == 0u ? 0ULL : mc;
  M = ((a ^ bc) >> 31) ? M - mc : M + mc;
  unsigned e = ea;
  if (M >> 53) {
    M >>= 1;
    ++e;
  } else if (!(M >> 52)) {
    M <<= 1;
    --e;
  }
  return from_bits(((unsigned long long)(a >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                   (M & 0x000fffffffffffffULL));
}
// 1/x to about 44 bits: y0 + y0 (1 - x y0) in FP32 on the split of x
__device__ __forceinline__ double rcp44(float xh, float xl) {
  const float y0 = rcp_approx_f32(xh);
  const float e1 = fmaf(-xl, y0, fmaf(-xh, y0, 1.0f));
  return join_f32(y0, e1 * y0);
}

__device__ __forceinline__ double mul_i(double a, double b);

// 1/x: the 44-bit reciprocal and one FP64 Newton step
__device__ __forceinline__ double rcp(double x) {
  float xh, xl;
  if (!split_f32(x, xh, xl)) return rcp_nr2(x);
  const double y = rcp44(xh, xl);
  const double e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// a/b: q = a y with the 44-bit reciprocal y of b (product on the integer pipes),
// then one residual correction
__device__ __forceinline__ double ddiv(double a, double b) {
  float bh, bl;
  if (!split_f32(b, bh, bl)) return ddiv_nr(a, b);
  const double y = rcp44(bh, bl);
  const double q = mul_i(a, y);
  const double r = fma(-b, q, a);
  return fma(r, y, q);
}

// sqrt(x), x > 0 in range: s0 = xh / sqrt(xh) from the rsqrt seed, one Heron step
// s0 + (x - s0^2) / (2 s0) in FP32 on the split, one FP64 Heron step (1/(2 s) from
// the seed)
__device__ __forceinline__ double dsqrt(double x) {
  float xh, xl;
  if ((long long)bits(x) <= 0 || !split_f32(x, xh, xl)) return dsqrt_nr2(x);
  const float r0 = rsqrt_approx_f32(xh);
  const float s0 = xh * r0, h0 = 0.5f * r0;
  const float d = fmaf(-s0, s0, xh) + xl;
  const double s = join_f32(s0, d * h0);
  const double r = fma(-s, s, x);
  return fma(r, widen_f32(h0), s);
}

// max/min of non-negative, non-NaN doubles via their bit patterns
__device__ __forceinline__ double maxnn(double a, double b) {
  const long long x = (long long)bits(a), y = (long long)bits(b);
  return from_bits((unsigned long long)(x > y ? x : y));
}
__device__ __forceinline__ double minnn(double a, double b) {
  const long long x = (long long)bits(a), y = (long long)bits(b);
  return from_bits((unsigned long long)(x < y ? x : y));
}
__device__ __forceinline__ double absd(double a) { return from_bits(bits(a) & 0x7fffffffffffffffULL); }
// finite (neither infinite nor NaN), from the exponent bits
__device__ __forceinline__ bool finite_bits(double a) { return ((hi32(a) >> 20) & 0x7ffu) != 0x7ffu; }
// a == 1.0 and a < 1.0 for non-negative a, +NaN included (bit-pattern comparisons on the
// integer pipe)
__device__ __forceinline__ bool is_one(double a) { return bits(a) == 0x3ff0000000000000ULL; }
__device__ __forceinline__ bool lt_one(double a) { return (long long)bits(a) < 0x3ff0000000000000LL; }
// a < 0 for non-NaN a (negative zero is not negative)
__device__ __forceinline__ bool isneg(double a) {
  const long long x = (long long)bits(a);
  return x < 0 && (x & 0x7fffffffffffffffLL) != 0;
}


// ---------------------------------------------------------------------------
// Binary64 product and sum on the integer pipes (IEEE 754-2008 round to nearest,
// ties to even).  Method: the exact integer product or sum of the significands,
// normalised, then rounded with a half bit and a sticky bit (the textbook
// construction, e.g. D. Goldberg, ACM Comput. Surv. 23(1), 1991, Sec. 1.4 and
// Theorem 2; J.-M. Muller et al., Handbook of Floating-Point Arithmetic, 2018,
// ch. 7).  A fast path covers every finite case whose result cannot be
// subnormal; the rest (infinities, NaN, subnormal operands or results) takes
// the FP64 instruction in a function that is not inlined: a branch around an
// inlined one is turned into a predicated FP64 instruction that still takes
// its issue slot on the FP64 pipe.
// ---------------------------------------------------------------------------
static __device__ __noinline__ double mul_hw(double a, double b) { return __dmul_rn(a, b); }
static __device__ __noinline__ double add_hw(double a, double b) { return __dadd_rn(a, b); }

// a * b.  Fast path: both finite with normal exponent fields and a product
// exponent field in [1, 2045], or a zero factor times a finite one (+-0).
__device__ __forceinline__ double mul_i(double a, double b) {
  const unsigned long long ia = bits(a), ib = bits(b);
  const unsigned s = (unsigned)((ia ^ ib) >> 32) & 0x80000000u;
  const unsigned ea = (unsigned)(ia >> 52) & 0x7ffu, eb = (unsigned)(ib >> 52) & 0x7ffu;
  const bool za = (ia << 1) == 0, zb = (ib << 1) == 0;
  const int esum = (int)(ea + eb) - 1023;   // product exponent field when the significand product is < 2
  const bool fast = ((ea - 1u < 2046u) && (eb - 1u < 2046u) && esum >= 1 && esum <= 2045) ||
                    ((za || zb) && ea != 0x7ffu && eb != 0x7ffu);
  if (!fast) return mul_hw(a, b);
  // significands with the leading one at bit 63: x, y in [2^63, 2^64)
  const unsigned long long x = ((ia & 0x000fffffffffffffULL) | 0x0010000000000000ULL) << 11;
  const unsigned long long y = ((ib & 0x000fffffffffffffULL) | 0x0010000000000000ULL) << 11;
  const unsigned x0 = (unsigned)x, x1 = (unsigned)(x >> 32), y0 = (unsigned)y, y1 = (unsigned)(y >> 32);
  unsigned r0, r1, r2, r3;   // the 128-bit product r3:r2:r1:r0, in [2^126, 2^128)
  asm("mul.lo.u32 %0, %4, %6;\n\t"
      "mul.hi.u32 %1, %4, %6;\n\t"
      "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
      "madc.hi.u32 %2, %4, %7, 0;\n\t"
      "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32 %3, 0, 0;\n\t"
      "mad.lo.cc.u32 %2, %5, %7, %2;\n\t"
      "madc.hi.u32 %3, %5, %7, %3;"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
      : "r"(x0), "r"(x1), "r"(y0), "r"(y1));
  const bool top = (r3 >> 31) != 0;   // significand product in [2, 4)
  // the 53-bit significand (leading one at bit 52) and the bits below it scaled
  // to 11 bits (half = 0x400); the low 64 bits of the product are sticky
  const unsigned sh = top ? 11u : 10u;
  const unsigned qlo = __funnelshift_r(r2, r3, sh), qhi = r3 >> sh;
  const unsigned rem = top ? (r2 & 0x7ffu) : ((r2 & 0x3ffu) << 1);
  const bool st = (r0 | r1) != 0;
  const unsigned up = (rem > 0x400u || (rem == 0x400u && (st || (qlo & 1u)))) ? 1u : 0u;
  // exponent field minus one plus sign into the high word; the leading one of the
  // significand adds the missing one, and a rounding carry out of it the next
  const unsigned eh = ((unsigned)(esum + (top ? 1 : 0) - 1) << 20) | s;
  unsigned lo, hi;
  asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, %5;" : "=r"(lo), "=r"(hi) : "r"(qlo), "r"(qhi), "r"(up), "r"(eh));
  const unsigned long long r = (za || zb) ? ((unsigned long long)s << 32) : (((unsigned long long)hi << 32) | lo);
  return from_bits(r);
}

// IEEE compares on the integer pipe (the same result as the FP64 compare for every
// input, NaN and +-0 included).
// x >= c and x > c for a constant c > 0: x in [c, +inf] (resp. (c, +inf]) by pattern
__device__ __forceinline__ bool ge_pos(double x, double c) {
  const unsigned long long bc = bits(c);
  return bits(x) - bc <= 0x7ff0000000000000ULL - bc;
}
__device__ __forceinline__ bool gt_pos(double x, double c) {
  const unsigned long long bc = bits(c);
  return bits(x) - bc - 1ULL < 0x7ff0000000000000ULL - bc;
}
// x >= 0: +-0, the positive finite values and +inf
__device__ __forceinline__ bool ge_zero(double x) {
  const unsigned long long b = bits(x);
  return b <= 0x7ff0000000000000ULL || b == 0x8000000000000000ULL;
}
// x >= y: the patterns mapped to an order-preserving unsigned key (negative values
// complemented, positive ones with the sign bit set); +-0 compare equal, NaN false
__device__ __forceinline__ bool ge_i(double x, double y) {
  const unsigned long long bx = bits(x), by = bits(y);
  const unsigned long long ax = bx & 0x7fffffffffffffffULL, ay = by & 0x7fffffffffffffffULL;
  if (ax > 0x7ff0000000000000ULL || ay > 0x7ff0000000000000ULL) return false;
  if ((ax | ay) == 0) return true;
  const unsigned long long kx = (bx >> 63) ? ~bx : (bx | 0x8000000000000000ULL);
  const unsigned long long ky = (by >> 63) ? ~by : (by | 0x8000000000000000ULL);
  return kx >= ky;
}

// -x on the integer pipe
__device__ __forceinline__ double neg_i(double x) { return from_bits(bits(x) ^ 0x8000000000000000ULL); }

// x * 2^K for a small constant K (an exact scaling): the exponent field moved by
// K on the integer pipes when x and the result are normal, +-0 kept, the rest
// (infinities, NaN, subnormal operand or result) by the FP64 product.
template <int K>
__device__ __forceinline__ double ldexp_i(double x) {
  static_assert(K >= -8 && K <= 8, "small scalings only");
  const unsigned long long ix = bits(x);
  const unsigned e = (unsigned)(ix >> 52) & 0x7ffu;
  if ((ix << 1) == 0) return x;
  const bool ok = K >= 0 ? (e - 1u < (unsigned)(2046 - K)) : (e - (unsigned)(1 - K) < (unsigned)(2046 + K));
  if (!ok) return mul_hw(x, K >= 0 ? (double)(1 << (K >= 0 ? K : 0)) : 1.0 / (double)(1 << (K < 0 ? -K : 0)));
  return from_bits(ix + ((unsigned long long)(long long)K << 52));
}

// a + b.  Fast path: the operand of larger magnitude finite and normal with an
// exponent field <= 2045, the other zero or with an exponent field >= 54 (no
// result is then subnormal), or both zero.
__device__ __forceinline__ double add_i(double a, double b) {
  const unsigned long long SGN = 0x8000000000000000ULL;
  const unsigned long long ia = bits(a), ib = bits(b);
  const unsigned long long ma = ia & ~SGN, mb = ib & ~SGN;
  const bool swp = ma < mb;
  const unsigned long long X = swp ? mb : ma, Y = swp ? ma : mb;   // |x| >= |y|
  const unsigned long long sx = (swp ? ib : ia) & SGN;
  const unsigned ex = (unsigned)(X >> 52), ey = (unsigned)(Y >> 52);
  const bool fast = (ex - 1u < 2045u && (ey >= 54u || Y == 0)) || X == 0;
  if (!fast) return add_hw(a, b);
  // significands with the leading one at bit 62 (10 guard bits below)
  const unsigned long long fx = ((X & 0x000fffffffffffffULL) | 0x0010000000000000ULL) << 10;
  const unsigned long long fy = Y == 0 ? 0ULL : ((Y & 0x000fffffffffffffULL) | 0x0010000000000000ULL) << 10;
  unsigned dsh = ex - ey;
  dsh = dsh < 63u ? dsh : 63u;
  unsigned long long al = fy >> dsh;
  al |= (unsigned long long)((al << dsh) != fy);   // sticky: some bit of y was shifted out
  const bool sub = ((ia ^ ib) & SGN) != 0;
  unsigned long long m = sub ? fx - al : fx + al;
  const int lz = __clzll((long long)m);
  m <<= (lz & 63);
  const unsigned long long q0 = m >> 11;   // leading one at bit 52
  const unsigned rem = (unsigned)m & 0x7ffu;   // half = 0x400
  const unsigned long long q = q0 + (unsigned long long)(rem > 0x400u || (rem == 0x400u && (q0 & 1ULL)));
  const unsigned long long e = (unsigned long long)(ex - (unsigned)lz);   // exponent field minus one
  unsigned long long r = sx | ((e << 52) + q);
  r = (m == 0) ? 0ULL : r;                // exact cancellation: +0
  r = (X == 0) ? (ia & ib) : r;           // +-0 + +-0: -0 only for -0 + -0
  return from_bits(r);
}

// a - b on the integer pipes
__device__ __forceinline__ double sub_i(double a, double b) { return add_i(a, neg_i(b)); }

}  // namespace afm
