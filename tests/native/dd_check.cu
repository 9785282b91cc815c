// Host check of the double-float arithmetic (csrc/dd.cuh) used by the FFT passes of the
// final checks: conversion, sum, difference and product of seeded random values against
// FP64, and a 64-point DFT evaluated in double-float against the same DFT in FP64, with
// the bounds the kernels rely on.  Prints one line per quantity and exits non-zero on a
// violated bound.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>

#include "../../paper_2607_17978_b300/csrc/dd.cuh"

static double rel(double got, double ref, double scale) { return std::fabs(got - ref) / scale; }

int main() {
  std::mt19937_64 gen(20260);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-20, 20);
  const double eps44 = std::ldexp(1.0, -44);
  int bad = 0;
  double m_conv = 0, m_add = 0, m_mul = 0;
  for (int i = 0; i < 200000; ++i) {
    const double a = std::ldexp(u(gen), ex(gen)), b = std::ldexp(u(gen), ex(gen));
    const dd A(a), B(b);
    m_conv = std::fmax(m_conv, rel((double)A, a, std::fabs(a)));
    const double s_scale = std::fmax(std::fabs(a), std::fabs(b));
    m_add = std::fmax(m_add, rel((double)(A + B), (double)A + (double)B, s_scale));
    m_add = std::fmax(m_add, rel((double)(A - B), (double)A - (double)B, s_scale));
    m_mul = std::fmax(m_mul, rel((double)(A * B), (double)A * (double)B, std::fabs(a * b)));
  }
  std::printf("conversion max rel %.3e (bound 2^-47 = %.3e)\n", m_conv, std::ldexp(1.0, -47));
  std::printf("sum/difference max err / max|operand| %.3e (bound 2^-44 = %.3e)\n", m_add, eps44);
  std::printf("product max rel %.3e (bound 2^-44 = %.3e)\n", m_mul, eps44);
  bad |= m_conv > std::ldexp(1.0, -47);
  bad |= m_add > eps44;
  bad |= m_mul > eps44;
  // 64-point DFT, direct sum with double-float twiddles, against FP64
  const int n = 64;
  double xr[n], xi[n];
  dd Xr[n], Xi[n];
  for (int k = 0; k < n; ++k) {
    xr[k] = u(gen);
    xi[k] = u(gen);
    Xr[k] = dd(xr[k]);
    Xi[k] = dd(xi[k]);
  }
  double err = 0.0, norm = 0.0;
  const double kTwoPi = 6.28318530717958647692;
  for (int f = 0; f < n; ++f) {
    double sr = 0, si = 0;
    dd Sr(0.0), Si(0.0);
    for (int k = 0; k < n; ++k) {
      const int m = (f * k) % n;
      const double c = std::cos(kTwoPi * m / n), s = -std::sin(kTwoPi * m / n);
      sr += xr[k] * c - xi[k] * s;
      si += xr[k] * s + xi[k] * c;
      const dd C(c), S(s);
      Sr += Xr[k] * C - Xi[k] * S;
      Si += Xr[k] * S + Xi[k] * C;
    }
    err = std::fmax(err, std::fmax(std::fabs((double)Sr - sr), std::fabs((double)Si - si)));
    norm = std::fmax(norm, std::fmax(std::fabs(sr), std::fabs(si)));
  }
  std::printf("64-point DFT max err / max|X| %.3e (bound 1e-11)\n", err / norm);
  bad |= !(err / norm < 1e-11);
  return bad ? 1 : 0;
}
