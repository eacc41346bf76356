// lc_df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
// Built from the error-free transformations TwoSum (Knuth) and TwoProd
// (with fma), so every operation runs on the FP32 pipe; GB300's FP64 pipe is
// about 70x slower than its FP32 pipe.  Exponent range is FP32's: values are
// brought into range by power-of-two scaling where needed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct __align__(8) lc_df {
  float hi, lo;
  __host__ __device__ lc_df() {}
  __host__ __device__ constexpr lc_df(float h, float l) : hi(h), lo(l) {}
  // exact for |v| < 2^48
  __device__ explicit lc_df(int64_t v) {
    hi = __ll2float_rn(v);
    lo = __ll2float_rn(v - __float2ll_rn(hi));
  }
  __device__ explicit lc_df(int v) : hi(float(v)), lo(0.0f) {}
};

__device__ __forceinline__ lc_df lc_df_fast2(float a, float b) {
  const float s = a + b;
  return lc_df(s, b - (s - a));
}
__device__ __forceinline__ lc_df lc_df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return lc_df(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ lc_df operator+(const lc_df& a, const lc_df& b) {
  lc_df s = lc_df_two_sum(a.hi, b.hi);
  return lc_df_fast2(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ lc_df operator-(const lc_df& a) { return lc_df(-a.hi, -a.lo); }
__device__ __forceinline__ lc_df operator-(const lc_df& a, const lc_df& b) { return a + (-b); }
__device__ __forceinline__ lc_df operator*(const lc_df& a, const lc_df& b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return lc_df_fast2(p, e);
}
__device__ __forceinline__ lc_df& operator+=(lc_df& a, const lc_df& b) { return a = a + b; }
__device__ __forceinline__ lc_df& operator*=(lc_df& a, const lc_df& b) { return a = a * b; }
// a*b + c with one rounding of the product's error terms
__device__ __forceinline__ lc_df fma(const lc_df& a, const lc_df& b, const lc_df& c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  lc_df s = lc_df_two_sum(p, c.hi);
  return lc_df_fast2(s.hi, s.lo + (e + c.lo));
}

// x * 2^-e as a double-float, from the bit pattern (no FP64 instruction on
// the common path).  The caller picks e per vector (the exponent of its
// largest entry), so the scaled values lie below 2 and everything FP32's
// range cannot hold is below 2^-126 of the vector's largest entry: those
// values flush to zero, which changes a normwise result by less than 1e-38.
// Subnormal FP64 inputs are normalised first; infinities and NaNs pass
// through unscaled.
__device__ __forceinline__ lc_df lc_df_from_double_s(double x, int e) {
  const uint64_t u = __double_as_longlong(x);
  int E = int((u >> 52) & 0x7ff);
  uint64_t m = u & ((uint64_t(1) << 52) - 1);
  if (E == 2047) return lc_df(float(x), 0.0f);
  if (E == 0) {  // zero or subnormal: m * 2^-1074
    if (m == 0) return lc_df(0.0f, 0.0f);
    const int sh = __clzll(m) - 11;  // bring the leading bit to position 52
    m <<= sh;
    E = 1 - sh;
  } else {
    m |= uint64_t(1) << 52;
  }
  E -= e;
  const int eh = E - 1023 + 127;
  if (eh < 1) return lc_df(0.0f, 0.0f);
  const uint32_t sgn = uint32_t(u >> 63) << 31;
  if (eh > 254) return lc_df(__uint_as_float(sgn | 0x7f800000u), 0.0f);
  const float hi = __uint_as_float(sgn | (uint32_t(eh) << 23) | (uint32_t(m >> 29) & 0x7fffffu));
  // remaining 29 bits: value (m & (2^29-1)) * 2^(E-1075)
  const int k = E - 1075;
  float lo = __uint2float_rn(uint32_t(m & 0x1fffffffu));
  lo = (k + 127 >= 1) ? lo * __uint_as_float(uint32_t(k + 127) << 23) : ldexpf(lo, k);
  return lc_df(hi, sgn ? -lo : lo);
}
__device__ __forceinline__ lc_df lc_df_from_double(double x) { return lc_df_from_double_s(x, 0); }
// f * 2^e as a double: exact (from the bit pattern) when the result is a
// normal FP64 number, else by a correctly rounded FP64 scaling.
__device__ __forceinline__ double lc_f2d_s(float f, int e) {
  const uint32_t u = __float_as_uint(f);
  const int ef = int((u >> 23) & 0xff);
  const uint64_t sgn = uint64_t(u >> 31) << 63;
  if (ef == 0) return __longlong_as_double(sgn);  // FP32 subnormals are not produced by the kernels
  if (ef == 255) return __longlong_as_double(sgn | (uint64_t(2047) << 52) | (uint64_t(u & 0x7fffffu) << 29));
  const int ed = ef - 127 + 1023 + e;
  if (ed >= 1 && ed <= 2046)
    return __longlong_as_double(sgn | (uint64_t(ed) << 52) | (uint64_t(u & 0x7fffffu) << 29));
  return ldexp(double(f), e);
}
__device__ __forceinline__ double lc_f2d(float f) { return lc_f2d_s(f, 0); }
// (hi + lo) * 2^e in FP64 (one FP64 add; exact when no scaled word leaves FP64's normal range).
__device__ __forceinline__ double lc_df_to_double_s(const lc_df& v, int e) { return lc_f2d_s(v.hi, e) + lc_f2d_s(v.lo, e); }
__device__ __forceinline__ double lc_df_to_double(const lc_df& v) { return lc_df_to_double_s(v, 0); }
