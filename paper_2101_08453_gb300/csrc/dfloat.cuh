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

// The same split of a double taken apart in integer arithmetic, without the
// double pipe: hi = the leading 24 significand bits rounded to nearest
// (halfway cases away from zero), lo = the remaining 29 bits, signed, rounded
// to a float and scaled by the exponent.  hi + lo = x to within
// 2^-48 |x|, |lo| <= ulp(hi)/2.  Values outside [2^-70, 2^100] in
// magnitude, zero, infinities and NaN take the conversion path of df_of.
__host__ __device__ inline float2 split_bits(double x) {
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &x, 8);
#endif
  const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
  const int e = (int)((h32 >> 20) & 0x7FFu);
  if (e < 1023 - 70 || e > 1023 + 100) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
  }
  const unsigned sign = h32 & 0x80000000u;
  // magnitude bits of the truncated float: exponent rebased, top 23 fraction bits
  unsigned hb = ((unsigned)(e - 1023 + 127) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
  int r = (int)(l32 & 0x1FFFFFFFu);  // the 29 bits below, units 2^(e - 1075)
  if (r >= (1 << 28)) {              // round the head up: a carry rolls into the exponent
    hb += 1u;
    r -= 1 << 29;
  }
  // 2^(e - 1075) as a float: biased exponent e - 948 is in [5, 175] here
  const unsigned sb = (unsigned)(e - 948) << 23;
#ifdef __CUDA_ARCH__
  const float scale = __uint_as_float(sb);
  const float lo = __int2float_rn(r) * scale;
  const float hi = __uint_as_float(hb | sign);
#else
  float scale, hi;
  __builtin_memcpy(&scale, &sb, 4);
  const unsigned hs = hb | sign;
  __builtin_memcpy(&hi, &hs, 4);
  const float lo = (float)r * scale;
#endif
  return make_float2(hi, sign ? -lo : lo);
}
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
