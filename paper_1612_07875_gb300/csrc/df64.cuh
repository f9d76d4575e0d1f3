// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two float32 numbers with |lo| <= ulp(hi)/2, giving about 48 significant
// bits. GB300 executes FP32 at 64x the FP64 rate, so the O(p^3) parts of the
// small eigen-solvers run on these operations instead of FP64.
//
// Building blocks (error-free transformations, exact in IEEE float32 with
// round-to-nearest and a fused multiply-add):
//   two_sum(a, b)       = (s, e) with s + e == a + b          (Knuth)
//   quick_two_sum(a, b) = (s, e) with s + e == a + b, |a|>=|b| (Dekker)
//   two_prod(a, b)      = (p, e) with p + e == a * b          (FMA)
// The compound operations renormalise their result; relative errors are a
// few units of 2^-48 (division and square root one Newton-type correction
// each; the reciprocal one Newton step). No operation relies on reassociation, so the code must be built
// without fast-math flags (it is: see build.py).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace sdmd {

struct alignas(8) dd {   // 8-byte aligned: one 64-bit load or store per value
  float hi, lo;
};

DF_HD dd two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  const float e = (a - (s - bp)) + (b - bp);
  return {s, e};
}

DF_HD dd quick_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}

DF_HD dd two_prod(float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  return {p, e};
}

DF_HD dd dd_make(float x) { return {x, 0.f}; }
DF_HD dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

DF_HD dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}

DF_HD dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

DF_HD dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, p.lo);
  p.lo = fmaf(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

DF_HD dd dd_mul_f(dd a, float b) {
  dd p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// a * b + c with one rounding of the product's tail folded into the sum
DF_HD dd dd_fma(dd a, dd b, dd c) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, p.lo);
  p.lo = fmaf(a.lo, b.hi, p.lo);
  return dd_add(p, c);
}

DF_HD dd dd_div(dd a, dd b) {
  const float q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_f(b, q1));
  const float q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_f(b, q2));
  const float q3 = r.hi / b.hi;
  const dd q = quick_two_sum(q1, q2);
  return dd_add(q, dd_make(q3));
}

// 1 / b: the FP32 reciprocal r0 refined by one Newton step r0 + r0 (1 - b r0),
// with the residual formed exactly (two_prod; 1 - p is exact for p near 1).
// r0 is correctly rounded, so the step leaves about 2^-47 relative error.
DF_HD dd dd_recip(dd b) {
  const float r0 = 1.f / b.hi;
  const dd pr = two_prod(b.hi, r0);
  const float res = fmaf(-b.lo, r0, (1.f - pr.hi) - pr.lo);
  return quick_two_sum(r0, r0 * res);
}

DF_HD dd dd_sqrt(dd a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float x = sqrtf(a.hi);
  const dd r = dd_sub(a, two_prod(x, x));
  return quick_two_sum(x, r.hi / (2.f * x));
}

DF_HD dd dd_scale(dd a, float pow2) { return {a.hi * pow2, a.lo * pow2}; }  // pow2 = exact power of two
DF_HD dd dd_abs(dd a) { return (a.hi < 0.f) ? dd_neg(a) : a; }
DF_HD bool dd_lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
DF_HD double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// Split a double into hi + lo floats using integer operations only (the
// 53-bit significand's top 24 bits, then the next 29 rounded to 24). Values
// must be normal and inside float range; zero maps to zero.
DF_HD dd dd_from_double(double x) {
  union {
    double d;
    unsigned long long u;
  } v;
  v.d = x;
  const unsigned long long b = v.u;
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return {0.f, 0.f};
  const bool neg = (b >> 63) != 0;
  const unsigned long long m = (b & 0xfffffffffffffULL) | (1ULL << 52);
  const int e2 = ex - 1075;                              // x = m * 2^e2
  const float fh = (float)(unsigned)(m >> 29);           // exact, < 2^24
  const float fl = (float)(unsigned)(m & 0x1fffffffULL); // rounds 29 -> 24 bits
  float hi = ldexpf(fh, e2 + 29);
  float lo = ldexpf(fl, e2);
  if (neg) {
    hi = -hi;
    lo = -lo;
  }
  return quick_two_sum(hi, lo);
}

// Same for an int64 (exact integers up to 2^48, rounded beyond).
DF_HD dd dd_from_ll(long long x) {
  const float hi = (float)x;
  const long long rem = x - (long long)hi;
  return quick_two_sum(hi, (float)rem);
}

// complex df64
struct zd {
  dd re, im;
};
DF_HD zd zd_add(zd a, zd b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
DF_HD zd zd_sub(zd a, zd b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
DF_HD zd zd_mul(zd a, zd b) {
  return {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
DF_HD zd zd_conj(zd a) { return {a.re, dd_neg(a.im)}; }
DF_HD dd zd_abs2(zd a) { return dd_add(dd_mul(a.re, a.re), dd_mul(a.im, a.im)); }
DF_HD zd zd_div(zd a, zd b) {
  const dd den = zd_abs2(b);
  const zd num = zd_mul(a, zd_conj(b));
  return {dd_div(num.re, den), dd_div(num.im, den)};
}

}  // namespace sdmd
