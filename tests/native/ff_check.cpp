// Host-side check of the double-float primitives of the CUDA library (csrc/lst_ff.cuh).
//
// TEST INFRASTRUCTURE. The header's functions are __host__ __device__, so a host build runs the
// same source. Each entry point evaluates one primitive on arrays of inputs and returns, per input,
// the error of the double-float result (hi + lo) against the same function evaluated in long
// double by the C library: relative for + - * / sqrt asin sinh, absolute for sin and cos.
#include <cmath>
#include <cstdint>

namespace lst { using std::isfinite; }   // the header calls the CUDA device-side name unqualified
#include "lst_ff.cuh"

using lst::ff;

namespace {
long double val(ff a) { return (long double)a.hi + (long double)a.lo; }
double rel(long double got, long double ref) {
  long double d = got - ref;
  if (d < 0) d = -d;
  long double s = ref < 0 ? -ref : ref;
  return s > 0 ? (double)(d / s) : (double)d;
}
double absdiff(long double got, long double ref) {
  long double d = got - ref;
  return (double)(d < 0 ? -d : d);
}
}  // namespace

extern "C" {

// op: 0 add, 1 sub, 2 mul, 3 div, 4 sqrt (of a), 5 asin (of a), 6 diff_prod(a, b, b, a) = a^2 - b^2
int ffc_binary(int op, int64_t n, const float* ahi, const float* alo, const float* bhi, const float* blo,
               double* err) {
  for (int64_t i = 0; i < n; ++i) {
    const ff a(ahi[i], alo[i]), b(bhi[i], blo[i]);
    const long double A = val(a), B = val(b);
    switch (op) {
      case 0: err[i] = absdiff(val(a + b), A + B) / (double)(fabsl(A) + fabsl(B)); break;
      case 1: err[i] = absdiff(val(a - b), A - B) / (double)(fabsl(A) + fabsl(B)); break;
      case 2: err[i] = rel(val(a * b), A * B); break;
      case 3: err[i] = rel(val(a / b), A / B); break;
      case 4: err[i] = rel(val(lst::m_sqrt(a)), sqrtl(A)); break;
      case 5: err[i] = rel(val(lst::m_asin(a)), asinl(A)); break;
      case 6: err[i] = absdiff(val(lst::diff_prod(a, a, b, b)), A * A - B * B) / (double)(A * A + B * B); break;
      default: return -1;
    }
  }
  return 0;
}

// sin and cos of float angles (absolute errors), sinh of floats (relative error)
int ffc_unary(int op, int64_t n, const float* x, double* err) {
  for (int64_t i = 0; i < n; ++i) {
    const long double X = (long double)x[i];
    if (op == 0 || op == 1) {
      ff s, c;
      lst::ff_sincos(x[i], s, c);
      err[i] = op == 0 ? absdiff(val(s), sinl(X)) : absdiff(val(c), cosl(X));
    } else if (op == 2) {
      err[i] = rel(val(lst::ff_sinh(x[i])), sinhl(X));
    } else {
      return -1;
    }
  }
  return 0;
}

// 1 when every result is a normalised pair (|lo| <= ulp(hi) / 2), else 0
int ffc_normalised(int op, int64_t n, const float* ahi, const float* alo, const float* bhi, const float* blo) {
  for (int64_t i = 0; i < n; ++i) {
    const ff a(ahi[i], alo[i]), b(bhi[i], blo[i]);
    ff r = op == 0 ? a + b : op == 1 ? a * b : op == 2 ? a / b : lst::m_sqrt(a);
    if (r.hi == 0.0f) continue;
    const float up = nextafterf(fabsf(r.hi), INFINITY) - fabsf(r.hi);
    if (!(fabsf(r.lo) <= 0.5f * up)) return 0;
  }
  return 1;
}
}
