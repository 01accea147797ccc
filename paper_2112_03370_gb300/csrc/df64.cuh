// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, which carries a 48-bit significand.  GB300 runs FP32 at 64 times its
// FP64 rate, so an FFT written in df64 on the FP32 pipes delivers FP64-class accuracy
// (normwise relative error ~1e-14 per transform) several times faster than native FP64.
//
// The primitives are the classical error-free transformations (Knuth's TwoSum, Dekker's
// FastTwoSum, and the FMA form of TwoProduct).  Every FP32 operation that belongs to an
// error-free transformation uses an explicit round-to-nearest intrinsic: the compiler never
// fuses those into an FMA, which would break the exactness the transformations rely on.
//
// Additions are the "sloppy" variant: the error is bounded by a small multiple of
// 2^-48 (|a| + |b|), not of |a + b|.  That is the bound an FFT's normwise error analysis uses,
// and it is what FP64 itself guarantees for a sum up to the constant.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_smem.cuh"

namespace mm {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l, int) : hi(h), lo(l) {}
  // rounding split of a double: hi = fl32(d), lo = fl32(d - hi)
  __host__ __device__ constexpr explicit df(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__device__ __forceinline__ df df_make(float h, float l) { return df(h, l, 0); }

// s + e = a + b exactly (no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, given |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator+(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);            // exact error of the leading product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }

// Exact FP32 -> FP64 widening by moving the fields of the IEEE-754 encodings (sign, exponent
// re-biased by 1023 - 127, significand shifted by 52 - 23) with integer instructions: on GB300 the
// conversion instruction runs on the FP64 pipe, 1/64 of the FP32 rate.  Zeros and subnormals map
// to a signed zero (a df64 low part is subnormal only when |hi| < 2^-102); infinities and NaNs
// keep their class.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sign);
  const uint64_t ed = (e == 0xffu) ? 0x7ffull : (uint64_t)(e + 896u);
  const uint64_t man = (uint64_t)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | (ed << 52) | man));
}

// exact widening of each part, then one FP64 rounding of their sum
__device__ __forceinline__ double df_to_double(df a) { return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo); }

struct __align__(16) dfc {
  df x, y;
};
template <> struct V2<df> { using t = dfc; };
template <> struct GenericProduct<dfc> { static constexpr bool value = false; };

// a b + c d with one renormalisation: both leading products and their exact errors, one TwoSum,
// and the low-order cross terms folded into the error word (19 FP32 operations instead of 25
// for two products and a sum)
__device__ __forceinline__ df df_prod_sum(df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float p2 = __fmul_rn(c.hi, d.hi);
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s, e;
  two_sum(p1, p2, s, e);
  float t = __fadd_rn(e1, e2);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fmaf_rn(c.hi, d.lo, t);
  t = __fmaf_rn(c.lo, d.hi, t);
  return fast_two_sum(s, __fadd_rn(e, t));
}

__device__ __forceinline__ dfc c_mul(dfc a, dfc b) {
  return dfc{df_prod_sum(a.x, b.x, -a.y, b.y), df_prod_sum(a.x, b.y, a.y, b.x)};
}
// a * conj(b)
__device__ __forceinline__ dfc c_mulc(dfc a, dfc b) {
  return dfc{df_prod_sum(a.x, b.x, a.y, b.y), df_prod_sum(a.y, b.x, -a.x, b.y)};
}

// 16-byte read-only load of a df64 complex value
template <>
__device__ __forceinline__ dfc ldg_c<dfc>(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfc{df_make(v.x, v.y), df_make(v.z, v.w)};
}

}  // namespace mm
