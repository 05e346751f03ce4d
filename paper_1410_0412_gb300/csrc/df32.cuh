// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from
// error-free transformations on the FP32 pipe:
//   two-sum (Knuth):        s = a + b, e = (a - (s - v)) + (b - v), v = s - a
//   fast two-sum (Dekker):  s = a + b, e = b - (s - a)        when |a| >= |b|
//   two-product with FMA:   p = a * b, e = fma(a, b, -p)
// GB300 runs FP32 FMAs 63x faster than FP64 ones, so the FP64-storage step can
// do its collision arithmetic here and keep IEEE doubles in memory.
// Conversions between double and df use integer bit operations only, so they
// stay off the FP64 pipe as well.
#pragma once

#include <cuda_runtime.h>

namespace lbm {
namespace dev {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit df(float h) : hi(h), lo(0.0f) {}
  __host__ __device__ constexpr explicit df(int h) : hi(float(h)), lo(0.0f) {}
  // Host-side split of a double constant: hi rounded to nearest, lo the rest.
  __host__ explicit df(double x) : hi(float(x)), lo(float(x - double(float(x)))) {}
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return df(s, (a - (s - v)) + (b - v));
}

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const float e = s.lo + (a.lo + b.lo);
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// df times a float (constants that are exact in float, e.g. -1.5, 6)
__device__ __forceinline__ df operator*(float f, df a) {
  const float p = f * a.hi;
  float e = __fmaf_rn(f, a.hi, -p);
  e = __fmaf_rn(f, a.lo, e);
  return fast_two_sum(p, e);
}

// exact halving (both parts scale by a power of two)
__device__ __forceinline__ df half(df a) { return df(0.5f * a.hi, 0.5f * a.lo); }
__device__ __forceinline__ double half(double a) { return 0.5 * a; }
__device__ __forceinline__ float half(float a) { return 0.5f * a; }

__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

// a * b + c with one rounding of the product's error folded into the sum.
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, s.lo + (e + c.lo));
}

// 1 / a: a correctly rounded float reciprocal refined by one Newton step in df.
__device__ __forceinline__ df recip(df a) {
  const float y = __frcp_rn(a.hi);
  const df ay = a * df(y);                 // a * y ~ 1
  const df r = df(1.0f) - ay;              // residual, |r| <~ 2^-23
  const float corr = y * (r.hi + r.lo);    // y * r needs only float accuracy
  return fast_two_sum(y, corr);
}
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }

// ---- IEEE double <-> df by integer bit manipulation ----------------------------
// double -> df: hi keeps the top 24 significand bits (truncated), lo the next 29
// bits rounded to 24 (relative error <= 2^-48).  Magnitudes below 2^-126 (far
// below any PDF value) are flushed to zero.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hw = static_cast<unsigned>(b >> 32), lw = static_cast<unsigned>(b);
  const int e = static_cast<int>((hw >> 20) & 0x7ffu);
  const int fe = e - 896;  // float biased exponent
  if (fe < 1) return df(0.0f, 0.0f);
  if (fe > 254) return df(__int_as_float(0x7fc00000), 0.0f);  // overflow, Inf, NaN -> NaN
  const unsigned sign = hw & 0x80000000u;
  const unsigned hb = sign | (static_cast<unsigned>(fe) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  const float hi = __uint_as_float(hb);
  const unsigned rem = lw & 0x1fffffffu;  // weight 2^(e - 1075)
  const int se = e - 948;                 // float biased exponent of 2^(e - 1075)
  float lo = 0.0f;
  if (se >= 1) lo = __uint2float_rn(rem) * __uint_as_float(static_cast<unsigned>(se) << 23);
  return df(hi, sign ? -lo : lo);
}

// float -> double bit pattern (exact; denormal floats flush to zero).
__device__ __forceinline__ double double_from_float_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0) return 0.0;
  const unsigned hw = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lw = (u & 0x7u) << 29;
  return __hiloint2double(static_cast<int>(hw), static_cast<int>(lw));
}

// df -> double: both parts exactly, then one FP64 add.
__device__ __forceinline__ double double_from_df(df a) {
  return double_from_float_bits(a.hi) + double_from_float_bits(a.lo);
}

// 1 / a for doubles: a float reciprocal of a's leading bits (integer ops and one
// MUFU, no FP64 conversion) refined by two Newton steps e = 1 - a y, y += y e
// (each roughly doubles the correct bits: 23 -> 46 -> 53), four FP64 FMAs in
// place of the ~10 FP64 instructions of an IEEE division.  Outside the float
// exponent range it falls back to the division.
__device__ __forceinline__ double recip(double a) {
  const unsigned hw = static_cast<unsigned>(__double_as_longlong(a) >> 32);
  const int fe = static_cast<int>((hw >> 20) & 0x7ffu) - 896;
  if (fe < 2 || fe > 252) return 1.0 / a;
  const float af = __uint_as_float((hw & 0x80000000u) | (static_cast<unsigned>(fe) << 23) | ((hw & 0xfffffu) << 3));
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(af));
  double y = double_from_float_bits(yf);
  double e = ::fma(-a, y, 1.0);
  y = ::fma(y, e, y);
  e = ::fma(-a, y, 1.0);
  return ::fma(y, e, y);
}
}  // namespace dev
}  // namespace lbm
