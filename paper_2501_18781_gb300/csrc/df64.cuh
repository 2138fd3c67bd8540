// Double-float ("df64") arithmetic: a value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, giving a 48-bit significand.  Products use the FMA error-free product
// (Dekker / Karp-Markstein: p = a*b, e = fma(a, b, -p) is exact), sums use Knuth's two-sum
// with the low parts added in ("sloppy" double-float addition, whose error is bounded by a few
// units of 2^-47 relative to |a| + |b|).  Bailey's double-double library and Joldes, Muller and
// Popescu (ACM TOMS 2017) describe and bound these algorithms.  GB300 runs fp32 at about 62x its
// fp64 rate, so fp64-accurate contractions are cheaper on the fp32 pipes this way.
// Range: the fp32 exponent (values far below 1e-30 lose low-part bits, above 1e38 overflow).
#pragma once

#include <cuda_runtime.h>

namespace mf {

struct df64 {
  float hi, lo;
  __device__ __forceinline__ df64() {}
  __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - double(hi));
  }
  __device__ __forceinline__ explicit df64(int x) : hi(float(x)), lo(0.f) {}
  __device__ __forceinline__ double to_double() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ df64 df_quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df64(s, e);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s = __fadd_rn(a.hi, b.hi);
  float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_quick_two_sum(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// storage precision of a compute type: df64 values live in fp64 memory
template <typename T> struct Store { using type = T; };
template <> struct Store<df64> { using type = double; };

template <typename T> __device__ __forceinline__ T from_store(typename Store<T>::type v) { return T(v); }
template <typename T> __device__ __forceinline__ typename Store<T>::type to_store(T v) { return v; }
template <> __device__ __forceinline__ double to_store<df64>(df64 v) { return v.to_double(); }

}  // namespace mf
