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

// exact widening of each part, then one FP64 rounding of their sum
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

struct __align__(16) dfc {
  df x, y;
};
template <> struct V2<df> { using t = dfc; };

// 16-byte read-only load of a df64 complex value
template <>
__device__ __forceinline__ dfc ldg_c<dfc>(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfc{df_make(v.x, v.y), df_make(v.z, v.w)};
}

}  // namespace mm
