// df32.cuh -- double-float arithmetic on the float32 pipe (every value the
// unevaluated sum hi + lo of two float32 numbers, about 48 significant bits):
// TwoSum (Knuth), FastTwoSum (Dekker), the FMA-based TwoProd (Ogita, Rump and
// Oishi, SISC 2005), a Newton reciprocal square root, and float64 <-> float
// pair conversions by integer operations (float64 arithmetic, conversions
// included, runs at ~1/64 of the float32 rate on this part).  The _rn
// intrinsics keep the compiler from contracting sums into multiply-adds.
#pragma once

#include "common.cuh"

namespace sks {
namespace {

struct F2 {
  float h, l;
};

SKS_DEV F2 f2_fast_two_sum(float a, float b) {  // exact when |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
SKS_DEV F2 f2_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
SKS_DEV F2 f2_mul(F2 x, F2 y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return f2_fast_two_sum(p, e);
}
// (h, l) += s * x * y with s = +1 or -1; the low part is accumulated without
// renormalising (TwoSum of the high parts, the product's TwoProd error and
// cross terms added to the low part).
template <bool SUB>
SKS_DEV void f2_acc(float& h, float& l, F2 x, F2 y) {
  const float p0 = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p0);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  const float p = SUB ? -p0 : p0;
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float t = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  l = SUB ? __fadd_rn(l, __fsub_rn(t, e)) : __fadd_rn(l, __fadd_rn(t, e));
}
// 1 / sqrt(p), p > 0: float32 seed (relative error <= 2^-22) and one Newton
// step r + r (1 - p r^2) / 2 in double-float (error ~1.5 * 2^-44).
SKS_DEV F2 f2_rsqrt(F2 p) {
  const float r0 = rsqrtf(p.h);
  const F2 q = f2_mul(f2_mul(p, {r0, 0.f}), {r0, 0.f});
  const float t = __fsub_rn(__fsub_rn(1.f, q.h), q.l);  // 1 - q.h is exact (Sterbenz)
  return f2_fast_two_sum(r0, __fmul_rn(__fmul_rn(r0, t), 0.5f));
}

// float64 -> hi + lo with integer operations only: hi keeps the top 24
// significant bits, lo the next 24 (the last 5 bits are dropped: relative
// error <= 2^-47).  Where lo would fall below float32's normal range
// (|x| < ~2^-100) only hi is kept, and values below that range become 0, so
// the caller scales the matrix by a power of two first; non-finite values
// stay non-finite in hi.
SKS_DEV F2 split_f64(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int E = (int)((u >> 52) & 0x7ff);
  const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  if (E == 0x7ff) return {__uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u)), 0.f};
  const int fe = E - 896;  // float32 biased exponent of hi
  if (fe <= 0) return {0.f, 0.f};
  if (fe >= 255) return {__uint_as_float(sign | 0x7f800000u), 0.f};
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(mant >> 29));
  const unsigned r = (unsigned)(mant & 0x1FFFFFFFull);  // lo = r * 2^(E - 1075)
  if (r == 0) return {hi, 0.f};
  const int sh = __clz(r) - 8;                         // moves the leading one to bit 23
  const unsigned m24 = sh >= 0 ? (r << sh) : (r >> (-sh));
  const int le = E - 925 - sh;                          // float32 biased exponent of lo
  if (le <= 0) return {hi, 0.f};
  return {hi, __uint_as_float(sign | ((unsigned)le << 23) | (m24 & 0x7FFFFFu))};
}
// float32 -> float64 exactly, integer operations only (subnormals become 0).
SKS_DEV double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xff;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (e == 0) return __longlong_as_double((long long)s);
  if (e == 255) return __longlong_as_double((long long)(s | 0x7FF0000000000000ull | m));
  return __longlong_as_double((long long)(s | ((unsigned long long)(e + 896) << 52) | m));
}

// 2^s v by exponent arithmetic (no float64 operation) while the result stays
// normal; ldexp otherwise.
SKS_DEV double scale_pow2(double v, int s) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  if (s == 0 || E == 0x7ff || (b << 1) == 0) return v;  // unscaled, non-finite or zero
  if (E == 0 || E + s <= 0 || E + s >= 0x7ff) return ldexp(v, s);  // subnormal or out of range
  return __longlong_as_double(b + ((long long)s << 52));
}


}  // namespace
}  // namespace sks
