// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats (|lo| <= ulp(hi)/2), about 48 significant bits.  The building
// blocks are the error-free transformations of floating-point sums and
// products: Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|), and the
// exact product a*b = p + e with e = fma(a, b, -p).  On GB300 the float pipe
// issues 61 times as many operations per clock as the double pipe, so the
// FP64-class element arithmetic runs on it in this form.
#pragma once
#include <cuda_runtime.h>

namespace mcw {

struct dflt {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ dflt df_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ dflt df_of(float x) { return {x, 0.0f}; }
__device__ __forceinline__ double to_double(dflt a) { return (double)a.hi + (double)a.lo; }

// Sum with error at most about 2^-48 (|a| + |b|): the high parts are added
// exactly (two-sum), the low parts in float, then renormalized.
__device__ __forceinline__ dflt operator+(dflt a, dflt b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  fast_two_sum(s, e, s, e);
  return {s, e};
}
__device__ __forceinline__ dflt operator-(dflt a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dflt operator-(dflt a, dflt b) { return a + (-b); }

__device__ __forceinline__ dflt operator*(dflt a, dflt b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return {s, t};
}

// product with an exactly representable float constant (0.5, 0.125, +-1, ...)
__device__ __forceinline__ dflt operator*(dflt a, float c) {
  const float p = a.hi * c;
  float e = fmaf(a.hi, c, -p);
  e = fmaf(a.lo, c, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return {s, t};
}

// 1/a: a float estimate refined by one Newton step, r + r (1 - a r)
__device__ __forceinline__ dflt reciprocal(dflt a) {
  const float r = 1.0f / a.hi;
  const dflt rr = {r, 0.0f};
  const dflt res = dflt{1.0f, 0.0f} - a * rr;
  return rr + rr * res;
}

__device__ __forceinline__ bool positive(dflt a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }

}  // namespace mcw
