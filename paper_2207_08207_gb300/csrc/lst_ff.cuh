// Double-float arithmetic on the float32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2: about 48
// significant bits, the float exponent range. GB300 runs float64 at a small fraction of its float32
// rate, so the decision kernels (T3, T5, pT3, pT5) evaluate the cut definitions in this format:
// each operation costs a few float32 instructions, against dozens of float32-equivalent issue
// slots for one float64 operation. Its rounding (~1e-14 relative per operation) is far inside the
// 1e-5 borderline band of the selections, so the decisions equal float64 ones outside that band.
//
// Building blocks are the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
// TwoProd by fused multiply-add; addition, multiplication, division and square root follow the
// double-length algorithms of Dekker (Numer. Math. 18 (1971) 224), as in the double-double library
// of Hida, Li and Bailey (ARITH-15, 2001). asin and sin are written below from their Taylor series and a Newton step.
// Non-finite intermediate results are returned with lo = 0 so that inf propagates like in float64.
#pragma once
#include <cuda_runtime.h>

namespace lst {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ff(float h) : hi(h), lo(0.0f) {}
  __host__ __device__ constexpr ff(int i) : hi((float)i), lo(0.0f) {}
  // from a double (host-side constants, literals): the nearest float and the rounded remainder
  __host__ __device__ constexpr ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

// Rounded float operations that the compiler may not fuse with their neighbours: the error-free
// transformations below assume that each product and sum is rounded on its own, and a product
// contracted into a following addition (an FMA) would count its rounding error twice. On the device
// the _rn intrinsics are never contracted; host builds of this header must disable contraction.
__host__ __device__ __forceinline__ float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

__host__ __device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float bb = f_sub(s, a);
  return ff(s, f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb)));
}
__host__ __device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = f_add(a, b);
  return ff(s, f_sub(b, f_sub(s, a)));
}
__host__ __device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = f_mul(a, b);
  return ff(p, fmaf(a, b, -p));
}

__host__ __device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }

__host__ __device__ __forceinline__ ff operator+(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  if (!isfinite(s.hi)) return ff(s.hi, 0.0f);
  s.lo += a.lo + b.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__host__ __device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__host__ __device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }

__host__ __device__ __forceinline__ ff operator*(ff a, ff b) {
  ff p = ff_two_prod(a.hi, b.hi);
  if (!isfinite(p.hi)) return ff(p.hi, 0.0f);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return ff_fast_two_sum(p.hi, p.lo);
}

__host__ __device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

// quotient: two float quotient digits, the second from the remainder of the first (Dekker);
// the float reciprocal needs to be good to a few ulp only
__host__ __device__ __forceinline__ ff operator/(ff a, ff b) {
#ifdef __CUDA_ARCH__
  const float ab = fabsf(b.hi);
  const float inv = (ab > 1e-30f && ab < 1e30f) ? __fdividef(1.0f, b.hi) : 1.0f / b.hi;
#else
  const float inv = 1.0f / b.hi;
#endif
  const float q1 = f_mul(a.hi, inv);
  if (!isfinite(q1) || b.hi == 0.0f) return ff(a.hi / b.hi, 0.0f);
  const ff p = ff_two_prod(b.hi, q1);
  const float r = (((a.hi - p.hi) - p.lo) + a.lo) - b.lo * q1;
  return ff_fast_two_sum(q1, f_mul(r, inv));
}

// comparisons (exact for normalised pairs)
__host__ __device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__host__ __device__ __forceinline__ bool operator>(ff a, ff b) { return b < a; }
__host__ __device__ __forceinline__ bool operator<=(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__host__ __device__ __forceinline__ bool operator>=(ff a, ff b) { return b <= a; }
__host__ __device__ __forceinline__ bool operator==(ff a, ff b) { return a.hi == b.hi && a.lo == b.lo; }
__host__ __device__ __forceinline__ bool operator!=(ff a, ff b) { return !(a == b); }

__host__ __device__ __forceinline__ ff m_abs(ff a) { return a.hi < 0.0f ? -a : a; }
__host__ __device__ __forceinline__ ff m_min(ff a, ff b) { return b < a ? b : a; }
__host__ __device__ __forceinline__ ff m_max(ff a, ff b) { return a < b ? b : a; }

// square root: float root s, then s + (a - s^2) / (2 s) with s^2 exact by TwoProd
__host__ __device__ __forceinline__ ff m_sqrt(ff a) {
  if (!(a.hi > 0.0f) || !isfinite(a.hi)) return ff(sqrtf(a.hi), 0.0f);
  const float s = sqrtf(a.hi);
  const ff p = ff_two_prod(s, s);
  const float e = ((a.hi - p.hi) - p.lo) + a.lo;
  return ff_fast_two_sum(s, e / f_mul(2.0f, s));
}

// a*d - b*c
__host__ __device__ __forceinline__ ff diff_prod(ff a, ff d, ff b, ff c) { return a * d - b * c; }

// sin y for |y| <= 0.8 by its Taylor series through y^15 (the next term is below 1e-16
// relative): the terms through y^7 in double-float, the rest (below 5e-7 relative) in float
__host__ __device__ __forceinline__ ff ff_sin_small(ff y) {
  const ff y2 = y * y;
  const float t2 = y2.hi;
  float tail = 1.0f / 1307674368000.0f;                 // 1/15!
  tail = fmaf(tail, -t2, 1.0f / 6227020800.0f);         // 1/13!
  tail = fmaf(tail, -t2, 1.0f / 39916800.0f);           // 1/11!
  tail = fmaf(tail, -t2, 1.0f / 362880.0f);             // 1/9!
  ff p = ff(1.0 / 5040.0) - ff(tail * t2);              // 1/7! - ...
  p = ff(1.0 / 120.0) - y2 * p;
  p = ff(1.0 / 6.0) - y2 * p;
  p = ff(1.0f) - y2 * p;
  return y * p;
}

// cos y for |y| <= 0.8 by its Taylor series through y^16 (the next term is below 2e-17)
__host__ __device__ __forceinline__ ff ff_cos_small(ff y) {
  const ff y2 = y * y;
  const float t2 = y2.hi;
  float tail = 1.0f / 20922789888000.0f;                // 1/16!
  tail = fmaf(tail, -t2, 1.0f / 87178291200.0f);        // 1/14!
  tail = fmaf(tail, -t2, 1.0f / 479001600.0f);          // 1/12!
  tail = fmaf(tail, -t2, 1.0f / 3628800.0f);            // 1/10!
  ff p = ff(1.0 / 40320.0) - ff(tail * t2);             // 1/8! - ...
  p = ff(1.0 / 720.0) - y2 * p;
  p = ff(1.0 / 24.0) - y2 * p;
  p = ff(0.5f) - y2 * p;
  return ff(1.0f) - y2 * p;
}

// sin and cos of a float angle |phi| <= 4: phi - k pi/2 (k the nearest integer; phi - k hi(pi/2)
// is exact for these k by Sterbenz's lemma), the quadrant's Taylor series, and the quadrant swap
__host__ __device__ __forceinline__ void ff_sincos(float phi, ff& sn, ff& cs) {
  const ff half_pi = ff(1.5707963267948966);
  const float k = rintf(phi * 0.63661977236758134f);
  const ff r = ff(fmaf(-k, half_pi.hi, phi)) - ff(k) * ff(half_pi.lo);
  const ff s = ff_sin_small(r), c = ff_cos_small(r);
  const int q = ((int)k) & 3;
  sn = q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
  cs = q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}

// exp x for |x| <= 0.35 by its Taylor series through x^13 (the next term is below 1e-16)
__host__ __device__ __forceinline__ ff ff_exp_small(ff x) {
  const float t = x.hi;
  float tail = 1.0f / 6227020800.0f;                    // 1/13!
  tail = fmaf(tail, t, 1.0f / 479001600.0f);            // 1/12!
  tail = fmaf(tail, t, 1.0f / 39916800.0f);             // 1/11!
  tail = fmaf(tail, t, 1.0f / 3628800.0f);              // 1/10!
  tail = fmaf(tail, t, 1.0f / 362880.0f);               // 1/9!
  ff p = ff(1.0 / 40320.0) + ff(tail * t);              // 1/8! + ...
  p = ff(1.0 / 5040.0) + x * p;
  p = ff(1.0 / 720.0) + x * p;
  p = ff(1.0 / 120.0) + x * p;
  p = ff(1.0 / 24.0) + x * p;
  p = ff(1.0 / 6.0) + x * p;
  p = ff(0.5f) + x * p;
  p = ff(1.0f) + x * p;
  return ff(1.0f) + x * p;
}

// sinh of a float |x| <= 40: the odd Taylor series for |x| < 0.5 (through x^15), else
// (e^x - e^-x) / 2 with e^x = 2^k e^(x - k ln 2)
__host__ __device__ __forceinline__ ff ff_sinh(float x) {
  const ff X(x);
  if (fabsf(x) < 0.5f) {
    const ff x2 = X * X;
    const float t2 = x2.hi;
    float tail = 1.0f / 1307674368000.0f;               // 1/15!
    tail = fmaf(tail, t2, 1.0f / 6227020800.0f);        // 1/13!
    tail = fmaf(tail, t2, 1.0f / 39916800.0f);          // 1/11!
    tail = fmaf(tail, t2, 1.0f / 362880.0f);            // 1/9!
    ff p = ff(1.0 / 5040.0) + ff(tail * t2);
    p = ff(1.0 / 120.0) + x2 * p;
    p = ff(1.0 / 6.0) + x2 * p;
    p = ff(1.0f) + x2 * p;
    return X * p;
  }
  const ff ln2 = ff(0.69314718055994531);
  const float k = rintf(x * 1.4426950408889634f);
  const ff r = ff(fmaf(-k, ln2.hi, x)) - ff(k) * ff(ln2.lo);
  const ff e = ff_exp_small(r);
  const float sc = ldexpf(1.0f, (int)k);
  const ff ep = ff(e.hi * sc, e.lo * sc);
  return (ep - ff(1.0f) / ep) * ff(0.5f);
}

// asin x for |x| <= 0.7 by one Newton step on sin from the float32 arcsine:
// y = y0 + (x - sin y0) / cos y0; the step's error is about tan(y0) e0^2 / 2 with e0 ~ 2e-7.
__host__ __device__ __forceinline__ ff ff_asin_small(ff x) {
  const float y0 = asinf(x.hi);
  const ff r = x - ff_sin_small(ff(y0));
  return ff_two_sum(y0, r.hi / cosf(y0));
}

// asin on [-1, 1]: near |x| = 1 through asin x = pi/2 - 2 asin sqrt((1 - x) / 2)
__host__ __device__ __forceinline__ ff m_asin(ff x) {
  const bool neg = x.hi < 0.0f;
  const ff ax = neg ? -x : x;
  ff y;
  if (ax.hi <= 0.7f) {
    y = ff_asin_small(ax);
  } else {
    const ff t = m_sqrt((ff(1.0f) - ax) * ff(0.5f));
    y = ff(1.5707963267948966) - ff(2.0f) * ff_asin_small(t);
  }
  return neg ? -y : y;
}

}  // namespace lst
