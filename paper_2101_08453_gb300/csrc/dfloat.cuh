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

// The rare cases of the integer conversions below go through the double
// pipe in functions of their own: a call is a real branch, so the compiler
// cannot turn the rare path into predicated instructions that every call
// would issue.
static __host__ __device__ __noinline__ float2 split_by_conversion(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
static __host__ __device__ __noinline__ double pair_sum_by_conversion(float hi, float lo) {
  return (double)hi + (double)lo;
}
static __host__ __device__ __noinline__ float float_by_conversion(double x) { return (float)x; }

// (float)r for |r| < 2^29, rounded to nearest even, on the float pipe (on
// GB300 ncu counts the int-to-float conversion instruction as double-pipe
// work): the two halves h = r >> 14 and l = r & 0x3FFF are read exactly off
// the 1.5 * 2^23 bias, and h * 2^14 + l is rounded once by the FMA.
__host__ __device__ inline float float_of_i29(int r) {
  const int h = r >> 14, l = r & 0x3FFF;
#ifdef __CUDA_ARCH__
  const float fh = __int_as_float(0x4B400000 + h) - 12582912.0f;
  const float fl = __int_as_float(0x4B400000 + l) - 12582912.0f;
  return __fmaf_rn(fh, 16384.0f, fl);
#else
  const int bh = 0x4B400000 + h, bl = 0x4B400000 + l;
  float fh, fl;
  __builtin_memcpy(&fh, &bh, 4);
  __builtin_memcpy(&fl, &bl, 4);
  return __builtin_fmaf(fh - 12582912.0f, 16384.0f, fl - 12582912.0f);
#endif
}

// The same split of a double taken apart in integer arithmetic, without the
// double pipe: hi = the leading 24 significand bits rounded to nearest
// (halfway cases away from zero), lo = the remaining 29 bits, signed, rounded
// to a float and scaled by the exponent.  hi + lo = x to within
// 2^-48 |x|, |lo| <= ulp(hi)/2.  Zero gives (+-0, 0); other values outside
// [2^-70, 2^100] in magnitude, infinities and NaN take the conversion path
// of df_of.
__host__ __device__ inline float2 split_bits(double x) {
#ifdef __CUDA_ARCH__
  const unsigned h32 = (unsigned)__double2hiint(x), l32 = (unsigned)__double2loint(x);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &x, 8);
  const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
#endif
  const int e = (int)((h32 >> 20) & 0x7FFu);
  // zero test on the two 32-bit words
  if (((h32 << 1) | l32) == 0u) {
#ifdef __CUDA_ARCH__
    return make_float2(__uint_as_float(h32), 0.0f);
#else
    float z;
    __builtin_memcpy(&z, &h32, 4);
    return make_float2(z, 0.0f);
#endif
  }
  if (e < 1023 - 70 || e > 1023 + 100) return split_by_conversion(x);
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
  const float lo = float_of_i29(r) * scale;
  const float hi = __uint_as_float(hb | sign);
#else
  float scale, hi;
  __builtin_memcpy(&scale, &sb, 4);
  const unsigned hs = hb | sign;
  __builtin_memcpy(&hi, &hs, 4);
  const float lo = float_of_i29(r) * scale;
#endif
  return make_float2(hi, sign ? -lo : lo);
}
__device__ __forceinline__ double to_double(dflt a) { return (double)a.hi + (double)a.lo; }

// hi + lo rounded to the nearest double (ties to even), the value to_double
// gives, formed in integer arithmetic and one float-to-integer conversion
// (GB300 issues that on the double pipe; there is no double arithmetic).
// The pair must be normalized (|lo| <= ulp(hi)/2, as every sum and product
// below leaves it).  |hi| as a double is its bit pattern
// with the exponent rebased and the 23 fraction bits moved up by 29; lo is
// then a whole number k of units of the double's last place in hi's binade
// (|k| <= 2^28), added to the magnitude's bit pattern.  That addition never
// carries into the exponent; it borrows from it only when hi is a power of
// two and lo lowers the magnitude, and then k is taken in the units of the
// binade below.  Zeros give the sum's zero; hi outside [2^-74, 2^128),
// infinities and NaN take the double-pipe path.
__host__ __device__ inline double pair_to_double(float hi, float lo) {
#ifdef __CUDA_ARCH__
  const unsigned uh = __float_as_uint(hi);
#else
  unsigned uh;
  __builtin_memcpy(&uh, &hi, 4);
#endif
  const int eh = (int)((uh >> 23) & 0xFFu);
  if ((uh << 1) == 0u && lo == 0.0f) {  // zero, negative only if both parts are -0
#ifdef __CUDA_ARCH__
    const unsigned ul = __float_as_uint(lo);
    return __longlong_as_double((long long)((unsigned long long)(uh & ul) << 32));
#else
    unsigned ul;
    __builtin_memcpy(&ul, &lo, 4);
    const unsigned long long zb = (unsigned long long)(uh & ul) << 32;
    double z;
    __builtin_memcpy(&z, &zb, 8);
    return z;
#endif
  }
  if (eh < 53 || eh > 254) return pair_sum_by_conversion(hi, lo);
  const unsigned sign = uh & 0x80000000u, mh = uh & 0x7FFFFFu;
  unsigned long long mag = ((unsigned long long)(((unsigned)(eh + 896) << 20) | (mh >> 3)) << 32) |
                           ((unsigned long long)(mh & 7u) << 29);
  const float l = sign ? -lo : lo;  // lo's share of the magnitude
  // 2^(52 - E) (or 2^(53 - E) for the binade below), E = eh - 127
  const unsigned sb = (unsigned)((mh == 0u && l < 0.0f) ? 307 - eh : 306 - eh) << 23;
#ifdef __CUDA_ARCH__
  const int k = __float2int_rn(l * __uint_as_float(sb));
  return __longlong_as_double((long long)((mag + (unsigned long long)(long long)k) |
                                          ((unsigned long long)sign << 32)));
#else
  float scale;
  __builtin_memcpy(&scale, &sb, 4);
  const int k = (int)__builtin_nearbyintf(l * scale);
  const unsigned long long bits = (mag + (unsigned long long)(long long)k) | ((unsigned long long)sign << 32);
  double out;
  __builtin_memcpy(&out, &bits, 8);
  return out;
#endif
}
__host__ __device__ inline double pair_to_double(float2 v) { return pair_to_double(v.x, v.y); }

// (float)x, rounded to nearest with ties to even as the conversion does, in
// integer arithmetic: the 23 fraction bits kept are rounded on the 29 below
// them (a carry may roll into the exponent, up to infinity).  Zero keeps
// its sign; results that would be subnormal or overflow before rounding,
// infinities and NaN take the conversion.
__host__ __device__ inline float float_of_bits(double x) {
#ifdef __CUDA_ARCH__
  const unsigned h32 = (unsigned)__double2hiint(x), l32 = (unsigned)__double2loint(x);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &x, 8);
  const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
#endif
  const unsigned sign = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7FFu);
  unsigned fb;
  if (e == 0 && (h32 & 0xFFFFFu) == 0u && l32 == 0u) {
    fb = sign;
  } else if (e < 1023 - 126 || e > 1023 + 127) {
    return float_by_conversion(x);
  } else {
    const unsigned top = ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);  // 23 fraction bits
    const unsigned rem = l32 & 0x1FFFFFFFu;
    fb = ((unsigned)(e - 1023 + 127) << 23) | top;
    if (rem > 0x10000000u || (rem == 0x10000000u && (top & 1u))) fb += 1u;
    fb |= sign;
  }
#ifdef __CUDA_ARCH__
  return __uint_as_float(fb);
#else
  float out;
  __builtin_memcpy(&out, &fb, 4);
  return out;
#endif
}

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
