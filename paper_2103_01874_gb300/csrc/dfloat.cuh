// Double-float ("float-float") arithmetic and exact-ish FP64 <-> pair
// conversions done with integer operations.
//
// Why: on a GB300 an FP64 FMA, and also every f64<->f32 conversion, issues at
// about 1/64 of the FP32 rate (measured: 1.19 TFLOP/s FP64 against 72.9 FP32;
// cvt f64<->f32 at ~1.9 per clock per SM; cvt u32->f32 at ~34).  The stencils
// of the projection (Eq. (34) right-hand side, the residual f - L p of the
// refinement, Eq. (33) correction) need FP64-level accuracy but few ops per
// byte, so they read and write IEEE FP64 at the API boundary and compute on
// pairs (hi, lo) of floats carrying ~48 significant bits.
//
// Published methods used (restated, not copied):
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and FastTwoSum (Dekker 1971) give
//     a + b = s + e exactly;
//   * TwoProd with a fused multiply-add (as in Dekker 1971 / the FMA
//     formulation of Ogita, Rump and Oishi 2005) gives a * b = p + e exactly;
//   * one Newton-Raphson step y1 = y0 + y0 (1 - a y0) for the reciprocal.
//
// Representation: value = hi + lo, |lo| <= ulp(hi)/2 after normalisation.
// Relative precision ~2^-48 (3.6e-15).  Range: magnitudes in [2^-74, 2^127];
// smaller inputs are flushed to zero (their contribution is below 1e-22 in
// absolute value), larger ones are out of scope.
//
// d2df(x): hi = x truncated to 24 significant bits (exponent rebias and
// mantissa shift on the bit pattern), lo = the remaining 29 mantissa bits as an
// integer, converted with one int->float conversion and scaled by 2^(e-1075).
// df2d(a): the exact doubles of hi and lo from their bit patterns, added by
// one FP64 add (correctly rounded; four per cell in the correction, well
// within the FP64 pipe those kernels otherwise leave idle).  df2d_alu(a), for
// kernels whose FP64 pipe is busy: exact double of hi from its bits, plus lo
// expressed in units of the double ulp of hi (a float scaling by a power of
// two and one float->int conversion) added to the bit pattern.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define PPE_HD __host__ __device__ __forceinline__
#else
#define PPE_HD inline
#endif

namespace ppe {

// 8-byte aligned, so that a pair moves as one 64-bit load or store
struct alignas(8) df {
  float hi, lo;
};

PPE_HD uint32_t f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}
PPE_HD float f_from(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}
PPE_HD uint64_t d_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}
PPE_HD double d_from(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
PPE_HD float rcp_rn(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}
PPE_HD int f2i_rn(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(x);
#else
  return (int)lrintf(x);
#endif
}

// a + b = s + e exactly (any magnitudes)
PPE_HD df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
// a + b = s + e exactly when |a| >= |b| (or a == 0)
PPE_HD df fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}
// a * b = p + e exactly
PPE_HD df two_prod(float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  return {p, e};
}

PPE_HD df df_make(float x) { return {x, 0.0f}; }
PPE_HD df df_neg(df a) { return {-a.hi, -a.lo}; }
PPE_HD df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}
PPE_HD df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
PPE_HD df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo += a.lo;
  return fast_two_sum(s.hi, s.lo);
}
PPE_HD df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
PPE_HD df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// exact scaling by a power of two
PPE_HD df df_ldexp2(df a) { return {2.0f * a.hi, 2.0f * a.lo}; }
// 1/a: correctly rounded float seed, one Newton step carried in pairs
PPE_HD df df_recip(df a) {
  const float y0 = rcp_rn(a.hi);
  df p = two_prod(a.hi, y0);                  // a.hi*y0 = p.hi + p.lo exactly, p.hi ~ 1
  const float e = ((1.0f - p.hi) - p.lo) - a.lo * y0;  // 1 - a*y0 to float precision
  return fast_two_sum(y0, y0 * e);
}
PPE_HD float df_to_f(df a) { return a.hi + a.lo; }

// "Lazy" variants for chains of operations: the hi parts are combined exactly
// (TwoSum / TwoProd) and the low parts are summed in plain FP32, without the
// renormalising FastTwoSum after each step.  The result is an unnormalised
// pair whose low part stays tiny against the high part; its error is that of
// the normalised operation plus a few ulps of the low part (relative ~2^-47).
// Normalise (df_norm) before storing or converting.
PPE_HD df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }
PPE_HD df df_addz(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return s;
}
PPE_HD df df_subz(df a, df b) { return df_addz(a, df_neg(b)); }
PPE_HD df df_mulz(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return p;
}
PPE_HD df df_mulz_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return p;
}
// Approximate float reciprocal seed (about 1 ulp on the device; exact on the host).
PPE_HD float rcp_seed(float x) {
#ifdef __CUDA_ARCH__
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / x;
#endif
}
// 1/a as an unnormalised pair: seed y0 ~ 1/a.hi, one Newton step (relative
// error ~ seed error squared, about 2^-44 with the device seed)
PPE_HD df df_recipz(df a) {
  const float y0 = rcp_seed(a.hi);
  df p = two_prod(a.hi, y0);
  const float e = ((1.0f - p.hi) - p.lo) - a.lo * y0;
  return {y0, y0 * e};
}

// IEEE double -> pair (see header comment).  Relative error <= 2^-48.
// hi: the 9 bits below the sign of (hw << 3 | lw >> 29) hold the exponent
// modulo 512 and the top 23 mantissa bits follow, so adding 128 << 23
// rebiases 1023 -> 127 (modulo 512) for every in-range exponent and the sign
// is or-ed back.  lo: the 29 low mantissa bits, converted once, times
// 2^(e - 1075) = 2^(E_hi - 52), whose bit pattern (with the sign of x) is hi's
// sign and exponent field minus 52 << 23.  |x| < 2^-74 gives (0, 0).
PPE_HD df d2df(double x) {
  const uint64_t b = d_bits(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t hb = (((hw << 3) | (lw >> 29)) + 0x40000000u) | (hw & 0x80000000u);
  const float sc = f_from((hb & 0xFF800000u) - 0x1A000000u);
  const float lo = (float)(lw & 0x1FFFFFFFu) * sc;
  const bool ok = (hw & 0x7FF00000u) >= (949u << 20);
  df r;
  r.hi = ok ? f_from(hb) : 0.0f;
  r.lo = ok ? lo : 0.0f;
  return r;
}

// exact double of a float from its bit pattern: exponent rebias 127 -> 1023
// and the 23 mantissa bits moved to the top of the 52 (zero for |x| < 2^-126)
PPE_HD uint64_t f2d_bits(float x) {
  const uint32_t b = f_bits(x);
  const uint32_t m = b & 0x7FFFFFFFu;
  if (m < 0x00800000u) return (uint64_t)(b & 0x80000000u) << 32;
  const uint32_t hw = ((m >> 3) + 0x38000000u) | (b & 0x80000000u);
  return ((uint64_t)hw << 32) | (uint64_t)(b << 29);
}

// pair -> IEEE double: the exact doubles of hi and lo added once, so the
// result is hi + lo correctly rounded (one FP64 add, on a pipe the pair
// kernels otherwise leave idle, in place of a float -> int conversion and
// the integer carry of the previous form)
PPE_HD double df2d(df a) { return d_from(f2d_bits(a.hi)) + d_from(f2d_bits(a.lo)); }

// pair -> IEEE double with integer and FP32 operations only (see header
// comment), for kernels whose FP64 pipe is already the limit.  Relative error
// ~2^-53.
PPE_HD double df2d_alu(df a) {
  a = fast_two_sum(a.hi, a.lo);
  const uint32_t hb = f_bits(a.hi);
  const uint32_t eh = (hb >> 23) & 0xFFu;  // biased float exponent of hi
  if (eh == 0u) return 0.0;                // |hi| < 2^-126: flushed
  // exact double of hi: rebias 127 -> 1023, mantissa to the top of 52 bits
  const uint64_t Hb = ((uint64_t)(hb >> 31) << 63) | ((uint64_t)(eh + 896u) << 52) |
                      ((uint64_t)(hb & 0x7FFFFFu) << 29);
  // lo in units of the double ulp of hi, 2^(E_h - 52) with E_h = eh - 127;
  // a negative lo below a power of two counts in the next binade down
  const bool down = ((hb & 0x7FFFFFu) == 0u) && ((a.lo < 0.0f) != (a.hi < 0.0f)) && a.lo != 0.0f;
  const uint32_t se = (down ? 307u : 306u) - eh;  // biased exponent of 2^(52 - E_h) (+1 if down)
  if (se >= 255u || se == 0u) return d_from(Hb);
  const float sc = f_from(se << 23);
  int k = f2i_rn(a.lo * sc);
  if (a.hi < 0.0f) k = -k;  // the bit pattern counts magnitude
  return d_from((uint64_t)((int64_t)Hb + (int64_t)k));
}

// ---------------------------------------------------------------------------
// dd: a double-float number with arithmetic operators, so that templates
// written for float and double (the FFT passes, the cosine-transform y solve)
// run in pair arithmetic.  Each operator is the normalised pair operation
// above (relative error about 2^-47 per operation).  Construction from a
// double splits it into the nearest float and the float of the remainder
// (exact to 2^-48 relative; used for compile-time constants and host tables --
// device code converts FP64 data with d2df, which needs no FP64 instruction).
// ---------------------------------------------------------------------------
struct alignas(8) dd {
  float hi, lo;
  dd() = default;
  PPE_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
  PPE_HD constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  PPE_HD constexpr dd(int x) : hi((float)x), lo(0.0f) {}  // exact for |x| < 2^24
  PPE_HD constexpr dd(df a) : hi(a.hi), lo(a.lo) {}
  PPE_HD explicit operator double() const { return (double)hi + (double)lo; }
  PPE_HD df pair() const { return {hi, lo}; }
};
PPE_HD dd operator+(dd a, dd b) { return dd(df_add(a.pair(), b.pair())); }
PPE_HD dd operator-(dd a, dd b) { return dd(df_sub(a.pair(), b.pair())); }
PPE_HD dd operator-(dd a) { return dd(-a.hi, -a.lo); }
PPE_HD dd operator*(dd a, dd b) { return dd(df_mul(a.pair(), b.pair())); }
PPE_HD dd operator/(dd a, dd b) { return dd(df_mul(a.pair(), df_recip(b.pair()))); }
// a b - c d (SUB) or a b + c d with one normalisation: the two TwoProds of
// the high parts, their TwoSum, the low parts and the four cross terms summed
// in FP32 (the error of the normalised products and sum taken together, about
// 2^-47 relative; 19 FP32 operations against 25 for two products and a sum).
template <bool SUB>
PPE_HD dd dd_dot2(dd a, dd b, dd c, dd d) {
  const float ch = SUB ? -c.hi : c.hi, cl = SUB ? -c.lo : c.lo;
  const df p = two_prod(a.hi, b.hi);
  const df q = two_prod(ch, d.hi);
  const df t = two_sum(p.hi, q.hi);
  float lo = (p.lo + q.lo) + t.lo;
  lo = fmaf(a.hi, b.lo, lo);
  lo = fmaf(a.lo, b.hi, lo);
  lo = fmaf(ch, d.lo, lo);
  lo = fmaf(cl, d.hi, lo);
  return dd(fast_two_sum(t.hi, lo));
}
// a + b without the final renormalisation (the lazy add above, as a dd): the
// high parts' TwoSum is exact, the low parts are summed in FP32; the result's
// low part may exceed half an ulp of its high part by a few ulps, which the
// next normalisation (dd_norm, a product, an add) absorbs.
PPE_HD dd dd_add_lazy(dd a, dd b) {
  const df s = two_sum(a.hi, b.hi);
  return dd(s.hi, s.lo + (a.lo + b.lo));
}
PPE_HD dd dd_sub_lazy(dd a, dd b) { return dd_add_lazy(a, dd(-b.hi, -b.lo)); }
PPE_HD dd dd_norm(dd a) { return dd(fast_two_sum(a.hi, a.lo)); }
PPE_HD dd& operator+=(dd& a, dd b) { return a = a + b; }
PPE_HD dd& operator-=(dd& a, dd b) { return a = a - b; }
PPE_HD dd& operator*=(dd& a, dd b) { return a = a * b; }

}  // namespace ppe
