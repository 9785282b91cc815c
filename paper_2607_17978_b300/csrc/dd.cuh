// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, about 48 significant bits (relative 2^-44 per operation).  The
// error-free transformations are the classical ones: Knuth's two-sum (s = a + b exactly as
// s + e), Dekker's fast two-sum for |a| >= |b|, and the FMA form of the exact product
// (p = a b exactly as p + fma(a, b, -p)); Dekker (1971), Knuth TAOCP vol. 2 4.2.2.  The
// FFT passes of the mixed-precision final check run in this type on the FP32 pipes: on
// this GPU FP32 issues ~60x faster than FP64, and a double-float operation costs 8-11
// FP32 instructions.  Sums take the "sloppy" form (one two-sum of the high parts, the low
// parts added plainly): its error is below 2^-44 of the larger operand, which is what a
// linear transform needs (its errors are measured against the norm of the data).
#pragma once

#include <cmath>

#ifdef __CUDA_ARCH__
#define QEQ_DD_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define QEQ_DD_FMA(a, b, c) std::fmaf(a, b, c)
#endif

struct dd {
  float hi, lo;
  dd() = default;  // trivial: shared-memory arrays of dd need no constructor
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // from double: the nearest FP32 and the FP32 of the remainder (constant-folded for
  // literals; one FP64 subtraction otherwise)
  __host__ __device__ constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) ddc {
  dd x, y;
};

__host__ __device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}
__host__ __device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return dd(s, b - (s - a));
}
__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  return dd_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = QEQ_DD_FMA(a.hi, b.hi, -p);
  e = QEQ_DD_FMA(a.hi, b.lo, QEQ_DD_FMA(a.lo, b.hi, e));
  return dd_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__host__ __device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }
__host__ __device__ __forceinline__ bool operator>(dd a, dd b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__host__ __device__ __forceinline__ bool operator<=(dd a, dd b) { return !(a > b); }
