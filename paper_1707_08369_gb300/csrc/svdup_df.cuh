// svdup_df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi), about 47 significant bits (Dekker 1971, "A
// floating-point technique for extending the available precision"; Knuth's TwoSum).
// The FP32 pipe issues about 80 times as many operations per clock as the FP64 pipe on
// this GPU, so sums whose terms need more than 24 but not 53 bits run here.
//
// Conversions from FP64 use the IEEE-754 bit fields (integer operations only): the
// FP64 pipe then sees none of the per-term work but the exact pole differences.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace svdup {

struct Df {
  float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ Df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return Df{s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker's Fast2Sum).
__device__ __forceinline__ Df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return Df{s, b - (s - a)};
}

__device__ __forceinline__ Df df_add(Df a, Df b) {
  Df s = df_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ Df df_neg(Df a) { return Df{-a.hi, -a.lo}; }

__device__ __forceinline__ Df df_mul(Df a, Df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a * a
__device__ __forceinline__ Df df_sqr(Df a) {
  const float p = a.hi * a.hi;
  float e = fmaf(a.hi, a.hi, -p);
  e = fmaf(2.0f * a.hi, a.lo, e);
  return df_fast_two_sum(p, e);
}

// 1 / a: r0 = an FP32 reciprocal of hi (MUFU, about one ulp), the residual
// e = 1 - a r0 from one FMA and one product, then r0 (1 + e + e^2) as a pair: the
// truncation after e^2 is below 2^-69 and the pair carries about 2^-46 relative error.
__device__ __forceinline__ Df df_rcp(Df a) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(a.hi));
  const float t = fmaf(-a.hi, r0, 1.0f);
  const float e = fmaf(-a.lo, r0, t);
  return df_fast_two_sum(r0, r0 * fmaf(e, e, e));
}

// Exact power of two 2^s as an FP32 number, -126 <= s <= 127.
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((s + 127) << 23); }

// Exact power of two 2^s as an FP64 number, -1022 <= s <= 1023.
__device__ __forceinline__ double pow2d(int s) {
  return __longlong_as_double((long long)(s + 1023) << 52);
}

// Unbiased binary exponent of a finite FP64 value (floor(log2 |x|)); -1100 for zero and
// subnormals (they are below every scale used here).
__device__ __forceinline__ int exp2_of(double x) {
  const int b = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return b == 0 ? -1100 : b - 1023;
}

// x * 2^-s as a pair, by the bit fields: hi keeps the top 24 significand bits
// (truncated), lo the next 23 (truncated), so |x 2^-s - (hi + lo)| < 2^-46 |x 2^-s|.
// The scaled value must lie below 2^127 in magnitude; below 2^-126 it becomes zero.
__device__ __forceinline__ Df df_from_f64(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int eb = (int)((b >> 52) & 0x7ff) - 1023 - s;  // unbiased exponent after scaling
  if (eb < -126) return Df{0.0f, 0.0f};
  const unsigned long long man = b & 0xfffffffffffffull;  // 52 fraction bits
  const float hi = __int_as_float((int)(sign | ((unsigned)(eb + 127) << 23) |
                                        (unsigned)(man >> 29)));
  // the next 23 fraction bits as an integer n < 2^23, worth n 2^(eb - 46)
  const unsigned n = (unsigned)(man >> 6) & 0x7fffffu;
  float lo = __int_as_float(0x4b000000 | (int)n) - 8388608.0f;  // exact: n < 2^23
  // 2^(eb - 46) in two exact steps (eb - 46 may fall below the normal range)
  lo = (lo * pow2f(max(eb - 46, -126) + 0)) * pow2f(min(0, eb - 46 + 126));
  return Df{hi, sign ? -lo : lo};
}

// The FP64 value of a pair scaled by 2^s: hi and lo widened exactly by their bit fields
// (FP32 subnormals become zero) and summed in FP64, then the power of two applied.
__device__ __forceinline__ double df_to_f64(Df a, int s) {
  auto widen = [](float x) -> double {
    const uint32_t u = __float_as_uint(x);
    const uint32_t mag = u & 0x7fffffffu;
    unsigned long long d = (unsigned long long)(u & 0x80000000u) << 32;
    if (mag >= 0x00800000u && mag < 0x7f800000u) d |= ((unsigned long long)mag << 29) + (896ull << 52);
    else if (mag >= 0x7f800000u) d |= 0x7ff8000000000000ull;
    return __longlong_as_double((long long)d);
  };
  return (widen(a.hi) + widen(a.lo)) * pow2d(s);
}

// x 2^s in FP64 by the bit fields, for x a normal FP32 number or a zero and a result in
// the FP64 normal range (ok is cleared otherwise): no FP64 operation.
__device__ __forceinline__ double widen_scaled(float x, int s, bool& ok) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t mag = u & 0x7fffffffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (mag == 0u) return __longlong_as_double((long long)sign);
  const int e = (int)(mag >> 23) + 896 + s;  // FP32 bias 127 -> FP64 bias 1023
  if (mag < 0x00800000u || mag >= 0x7f800000u || e < 1 || e > 2046) {
    ok = false;
    return 0.0;
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)e << 52) | ((unsigned long long)(mag & 0x7fffffu) << 29)));
}

// A pair times 2^s in FP64: both parts scaled by their exponent fields and added (one
// FP64 operation; the same value as df_to_f64(a, 0) 2^s whenever no part leaves the
// normal ranges, which then takes the multiplications).
__device__ __forceinline__ double df_to_f64_scaled(Df a, int s) {
  bool ok = true;
  const double h = widen_scaled(a.hi, s, ok), l = widen_scaled(a.lo, s, ok);
  if (ok) return h + l;
  const int q = s / 2;
  return df_to_f64(a, 0) * pow2d(max(-1022, min(1023, q))) * pow2d(max(-1022, min(1023, s - q)));
}

// FP64 finiteness by the exponent field (an integer test, no FP64 operation).
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ Df df_shfl_xor(Df a, int o) {
  return Df{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ Df df_warp_sum(Df a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return a;
}

// FP64 -> FP32 rounded to nearest (ties away from zero) by the bit fields: the top 24
// significant bits plus the next one as a carry, which the exponent field absorbs when
// it overflows the fraction.  Values below the FP32 normal range become signed zeros.
__device__ __forceinline__ float narrow_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex <= 896) return __uint_as_float(sign);
  if (ex >= 1151) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  const unsigned u = (unsigned)((mag >> 29) - (896ull << 23)) + (unsigned)((b >> 28) & 1ull);
  return __uint_as_float(sign | u);
}

// Exact FP32 -> FP64 widening through the IEEE-754 bit fields: the exponent is re-biased
// (1023 - 127 = 896) and the 23 fraction bits move up by 29.  FP32 subnormals (below
// 1.2e-38) become signed zeros; Inf and NaN keep their class.  Integer work only, so the
// conversion of an output tile stays off the FP64 pipe.
__device__ __forceinline__ double widen_f32(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t mag = u & 0x7fffffffu;
  unsigned long long d = (unsigned long long)(u & 0x80000000u) << 32;
  if (mag >= 0x7f800000u)
    d |= 0x7ff0000000000000ull | ((unsigned long long)(mag & 0x007fffffu) << 29);
  else if (mag >= 0x00800000u)
    d |= ((unsigned long long)mag << 29) + (896ull << 52);
  return __longlong_as_double((long long)d);
}

}  // namespace svdup
