// Double-word ("float-float") arithmetic for the FP64-class residuals of the mixed-precision
// solver.  A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about
// 48 significant bits, computed on the FP32 pipes (GB300 runs FP32 at 64 times its FP64 rate).
//
// Building blocks (error-free transformations): Knuth's TwoSum, Dekker's FastTwoSum (|a| >= |b|)
// and the FMA-based exact product.  The sum is the plain double-word addition (absolute error a
// few units of 2^-47 (|x| + |y|), no relative bound under cancellation, which is the bound an
// FP64 sum of the same terms has up to the unit); the products follow the double-word times
// double-word and double-word times float algorithms of Joldes, Muller and Popescu (ACM TOMS 44,
// 2017).  The *_rn intrinsics are used so that no product is contracted into an FMA.
#pragma once

#include <cuda_runtime.h>

namespace xfft {

struct dw {
  float hi, lo;
  dw() = default;
  __device__ __forceinline__ dw(float x) : hi(x), lo(0.0f) {}
  __device__ __forceinline__ dw(int x) : hi((float)x), lo(0.0f) {}
  __device__ __forceinline__ explicit dw(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  dw r;
  r.hi = s;
  r.lo = e;
  return r;
}
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  dw r;
  r.hi = s;
  r.lo = __fsub_rn(b, __fsub_rn(s, a));
  return r;
}

__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = dw_two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  return dw_fast_two_sum(s.hi, __fadd_rn(s.lo, v));
}
__device__ __forceinline__ dw operator-(dw x) {
  x.hi = -x.hi;
  x.lo = -x.lo;
  return x;
}
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float ph = __fmul_rn(x.hi, y.hi);
  float pl = __fmaf_rn(x.hi, y.hi, -ph);
  pl = __fmaf_rn(x.hi, y.lo, pl);
  pl = __fmaf_rn(x.lo, y.hi, pl);
  return dw_fast_two_sum(ph, pl);
}
__device__ __forceinline__ dw& operator+=(dw& x, dw y) { return x = x + y; }
__device__ __forceinline__ dw& operator-=(dw& x, dw y) { return x = x - y; }
__device__ __forceinline__ dw& operator*=(dw& x, dw y) { return x = x * y; }
__device__ __forceinline__ float absval(float x) { return fabsf(x); }
__device__ __forceinline__ double absval(double x) { return ::fabs(x); }
__device__ __forceinline__ dw absval(dw x) { return x.hi < 0.0f ? -x : x; }

// Storage type of each compute type: double-word values live in FP64 arrays.
template <typename T>
struct Store {
  typedef T type;
};
template <>
struct Store<dw> {
  typedef double type;
};

// storage -> compute and compute -> storage conversions
template <typename T, typename S>
__device__ __forceinline__ T from_store(S x) {
  return (T)x;
}
template <>
__device__ __forceinline__ dw from_store<dw, double>(double x) {
  return dw(x);
}
template <>
__device__ __forceinline__ dw from_store<dw, float>(float x) {
  return dw(x);
}
__device__ __forceinline__ float to_store(float x) { return x; }
__device__ __forceinline__ double to_store(double x) { return x; }
__device__ __forceinline__ double to_store(dw x) { return (double)x; }

// value type of warp reductions: the arithmetic type, FP64 for double-word values
__device__ __forceinline__ float red_val(float x) { return x; }
__device__ __forceinline__ double red_val(double x) { return x; }
__device__ __forceinline__ double red_val(dw x) { return (double)x; }

__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(dw x) { return (double)x; }

template <typename T>
__device__ __forceinline__ T shfl_up_t(unsigned mask, T v, int delta, int width) {
  return __shfl_up_sync(mask, v, delta, width);
}
template <>
__device__ __forceinline__ dw shfl_up_t<dw>(unsigned mask, dw v, int delta, int width) {
  dw r;
  r.hi = __shfl_up_sync(mask, v.hi, delta, width);
  r.lo = __shfl_up_sync(mask, v.lo, delta, width);
  return r;
}

}  // namespace xfft
