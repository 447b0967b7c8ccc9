// Double-float ("float-float") arithmetic on the FP32 pipe.
//
// A value is hi + lo with two floats, |lo| <= ulp(hi)/2: about 48 significant
// bits.  On GB300 the FP32 pipe issues 64 times more FMAs than the FP64 pipe,
// so a double-float FMA (about 15 FP32 instructions) costs roughly a quarter
// of a native FP64 FMA while keeping a relative precision near 1e-14.  The
// operations are built from the error-free transformations two-sum (Knuth)
// and two-product through fmaf, renormalised with quick-two-sum.
#pragma once
#include <cuda_runtime.h>

namespace adft {

struct df {
  float hi, lo;
  __host__ __device__ df() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// compile-time constant from a double literal
__host__ __device__ constexpr df dfc(double x) { return df((float)x, (float)(x - (double)(float)x)); }

// run-time conversion from double (two double-to-float roundings)
__device__ __forceinline__ df to_df(double v) {
  const float h = __double2float_rn(v);
  return df(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df(s, (a - (s - bb)) + (b - bb));
}

// accurate addition: both the high and the low parts are added error-free
__device__ __forceinline__ df operator+(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  const df t = two_sum(x.lo, y.lo);
  s = quick_two_sum(s.hi, s.lo + t.hi);
  return quick_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& x, df y) { return x = x + y; }
__device__ __forceinline__ df& operator*=(df& x, df y) { return x = x * y; }

// 1/sqrt(x): single-precision estimate refined by two Newton steps in
// double-float, r' = r + r (1 - x r^2) / 2.
__device__ __forceinline__ df rsqrt_df(df x) {
  df r(rsqrtf(x.hi), 0.f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df e = dfc(1.0) - x * (r * r);
    r = r + r * (e * dfc(0.5));
  }
  return r;
}

// 1/x: single-precision estimate refined by two Newton steps, r' = r + r (1 - x r).
__device__ __forceinline__ df rcp_df(df x) {
  df r(1.0f / x.hi, 0.f);
#pragma unroll
  for (int it = 0; it < 2; ++it) r = r + r * (dfc(1.0) - x * r);
  return r;
}

using ::__ldg;
__device__ __forceinline__ df __ldg(const df* p) {
  const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}

}  // namespace adft
