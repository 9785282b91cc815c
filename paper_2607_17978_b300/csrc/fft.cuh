// FFT machinery of the plane-wave matvec: register DFT butterflies (radices 2-16),
// mixed-radix in-place stages on lines staged in shared memory by TMA bulk copies, and
// the transposing passes of the 3D FFT with the reciprocal multiply of eq. (matvec)
// fused into the x pass.  Included by matvec.cu only (its kernels live in that unit).
#pragma once

// threads per CTA of the FP32 FFT kernels and the resident CTAs per SM they are compiled
// for (register budget 65536 / (threads n)); FP64 kernels: 256 threads, one CTA per SM
#ifndef QEQ_FFT_THREADS32
#define QEQ_FFT_THREADS32 256
#endif
#ifndef QEQ_FFT_MIN_BLOCKS32
#define QEQ_FFT_MIN_BLOCKS32 2
#endif
#include <math.h>

#include <type_traits>
#include <utility>

#include "dd.cuh"
#include "qeq_internal.cuh"

namespace {

// complex element of a mesh of real type T: FP32, FP64, or double-float (the final check
// of mixed-precision solves; dd.cuh)
template <typename T>
struct C2;
template <>
struct C2<float> {
  using t = float2;
};
template <>
struct C2<double> {
  using t = double2;
};
template <>
struct C2<dd> {
  using t = ddc;
};
// resident CTAs per SM the FFT kernels of type T are compiled for: FP64 one (its stages
// need ~150 registers), double-float two (128 registers, a few spilled, ran the final
// check's passes 1.3x faster than one CTA with 200 registers)
template <typename T>
__host__ __device__ constexpr int fft_min_blocks() {
  return std::is_same<T, float>::value ? QEQ_FFT_MIN_BLOCKS32 : (std::is_same<T, dd>::value ? 2 : 1);
}
// which of a length's three FFT plans a pass of type T uses: FP32 stages (radices up to
// 24), FP64 stages (up to 16) with FP64 twiddles, the same stages with double-float twiddles
template <typename T>
__host__ __device__ constexpr int fft_plan_variant() {
  return std::is_same<T, float>::value ? 0 : (std::is_same<T, double>::value ? 1 : 2);
}

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename V>
__device__ __forceinline__ V csub(V a, V b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by i*sgn
template <typename V, typename T>
__device__ __forceinline__ V cmul_i(V a, T sgn) {
  return {-sgn * a.y, sgn * a.x};
}
template <typename V, typename T>
__device__ __forceinline__ V cscale(V a, T s) {
  return {a.x * s, a.y * s};
}

template <typename T>
__device__ __forceinline__ const typename C2<T>::t* twiddles(const double2* tw64, const float2* tw32);
template <>
__device__ __forceinline__ const float2* twiddles<float>(const double2*, const float2* tw32) {
  return tw32;
}
template <>
__device__ __forceinline__ const double2* twiddles<double>(const double2* tw64, const float2*) {
  return tw64;
}
template <>
__device__ __forceinline__ const ddc* twiddles<dd>(const double2* tw64, const float2*) {
  return reinterpret_cast<const ddc*>(tw64);  // the double-float tables share the FP64 array (16 bytes each)
}

// ------------------------------------------------------------------ small DFTs
// y_a = sum_b v_b exp(sgn * 2 pi i a b / R), sgn = -1 forward, +1 inverse
template <typename T, typename V>
__device__ __forceinline__ void dft2(V* v) {
  V a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <typename T, typename V>
__device__ __forceinline__ void dft3(V* v, T sgn) {
  const T s3 = (T)0.86602540378443864676;  // sin(2 pi/3)
  V t1 = cadd(v[1], v[2]);
  V t2 = {v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y};
  V t3 = cmul_i<V, T>(csub(v[1], v[2]), sgn * s3);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, t3);
  v[2] = csub(t2, t3);
}
template <typename T, typename V>
__device__ __forceinline__ void dft4(V* v, T sgn) {
  V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  V c = cadd(v[1], v[3]), d = cmul_i<V, T>(csub(v[1], v[3]), sgn);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}
template <typename T, typename V>
__device__ __forceinline__ void dft5(V* v, T sgn) {
  const T c1 = (T)0.30901699437494742410;   // cos(2 pi/5)
  const T c2 = (T)-0.80901699437494742410;  // cos(4 pi/5)
  const T s1 = (T)0.95105651629515357212;   // sin(2 pi/5)
  const T s2 = (T)0.58778525229247312917;   // sin(4 pi/5)
  V a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
  V a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
  V x0 = v[0];
  V r1 = {x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y};
  V r2 = {x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y};
  V i1 = cmul_i<V, T>(V{s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y}, sgn);
  V i2 = cmul_i<V, T>(V{s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y}, sgn);
  v[0] = {x0.x + a1.x + a2.x, x0.y + a1.y + a2.y};
  v[1] = cadd(r1, i1);
  v[4] = csub(r1, i1);
  v[2] = cadd(r2, i2);
  v[3] = csub(r2, i2);
}

// ------------------------------------------------------------------ composite register butterflies
// cos and sin of 2 pi m / R at compile time (quadrant reduction, Taylor series
// on [0, pi/2]), for the internal twiddles of the composite radices.
__host__ __device__ constexpr double cx_poly_cos(double x) {
  double x2 = x * x, t = 1.0, s = 1.0;
  for (int k = 1; k < 14; ++k) {
    t *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double cx_poly_sin(double x) {
  double x2 = x * x, t = x, s = x;
  for (int k = 1; k < 14; ++k) {
    t *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
__host__ __device__ constexpr double cx_cos2pi(int m, int R) {
  const int q = (4 * m) / R, rem = 4 * m - q * R;  // 2 pi m / R = q pi/2 + phi
  const double phi = 1.57079632679489661923 * rem / R;
  const double c = cx_poly_cos(phi), s = cx_poly_sin(phi);
  return q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}
__host__ __device__ constexpr double cx_sin2pi(int m, int R) {
  const int q = (4 * m) / R, rem = 4 * m - q * R;
  const double phi = 1.57079632679489661923 * rem / R;
  const double c = cx_poly_cos(phi), s = cx_poly_sin(phi);
  return q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
}

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// a * exp(sgn * 2 pi i M / R) with the constant folded in
template <typename T, typename V, int M, int R>
__device__ __forceinline__ V tw_const(V a, T sgn) {
  constexpr int m = M % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (4 * m == R) {
    return cmul_i<V, T>(a, sgn);
  } else if constexpr (2 * m == R) {
    return V{-a.x, -a.y};
  } else if constexpr (4 * m == 3 * R) {
    return cmul_i<V, T>(a, -sgn);
  } else {
    constexpr double c = cx_cos2pi(m, R), sn = cx_sin2pi(m, R);
    const T ss = sgn * (T)sn;
    return V{a.x * (T)c - a.y * ss, a.x * ss + a.y * (T)c};
  }
}

template <typename T, typename V, int R>
struct DftR;
template <typename T, typename V>
struct DftR<T, V, 2> {
  static __device__ __forceinline__ void run(V* v, T) { dft2<T, V>(v); }
};
template <typename T, typename V>
struct DftR<T, V, 3> {
  static __device__ __forceinline__ void run(V* v, T sgn) { dft3<T, V>(v, sgn); }
};
template <typename T, typename V>
struct DftR<T, V, 4> {
  static __device__ __forceinline__ void run(V* v, T sgn) { dft4<T, V>(v, sgn); }
};
template <typename T, typename V>
struct DftR<T, V, 5> {
  static __device__ __forceinline__ void run(V* v, T sgn) { dft5<T, V>(v, sgn); }
};

// R = A*B point DFT in registers (Cooley-Tukey): inputs n = B n1 + n2, outputs
// k = k1 + A k2; A-point DFTs over n1, internal twiddles W_R^(n2 k1), B-point
// DFTs over n2.
template <typename T, typename V, int A, int B>
__device__ __forceinline__ void dft_ab(V* v, T sgn) {
  constexpr int R = A * B;
  V y[R];
  static_for<B>([&](auto n2c) {
    constexpr int n2 = decltype(n2c)::value;
    V t[A];
    static_for<A>([&](auto n1c) { t[decltype(n1c)::value] = v[B * decltype(n1c)::value + n2]; });
    DftR<T, V, A>::run(t, sgn);
    static_for<A>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      y[n2 * A + k1] = tw_const<T, V, n2 * k1, R>(t[k1], sgn);
    });
  });
  static_for<A>([&](auto k1c) {
    constexpr int k1 = decltype(k1c)::value;
    V u[B];
    static_for<B>([&](auto n2c) { u[decltype(n2c)::value] = y[decltype(n2c)::value * A + k1]; });
    DftR<T, V, B>::run(u, sgn);
    static_for<B>([&](auto k2c) { v[k1 + A * decltype(k2c)::value] = u[decltype(k2c)::value]; });
  });
}
#define QEQ_COMPOSITE_DFT(R, A, B)                                                        \
  template <typename T, typename V>                                                       \
  struct DftR<T, V, R> {                                                                  \
    static __device__ __forceinline__ void run(V* v, T sgn) { dft_ab<T, V, A, B>(v, sgn); } \
  };
QEQ_COMPOSITE_DFT(6, 2, 3)
QEQ_COMPOSITE_DFT(8, 2, 4)
QEQ_COMPOSITE_DFT(9, 3, 3)
QEQ_COMPOSITE_DFT(10, 2, 5)
QEQ_COMPOSITE_DFT(12, 3, 4)
QEQ_COMPOSITE_DFT(15, 3, 5)
QEQ_COMPOSITE_DFT(16, 4, 4)
QEQ_COMPOSITE_DFT(18, 2, 9)
QEQ_COMPOSITE_DFT(20, 4, 5)
QEQ_COMPOSITE_DFT(24, 3, 8)
#undef QEQ_COMPOSITE_DFT


// ------------------------------------------------------------------ TMA bulk copies, mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy (TMA engine), completion counted on the mbarrier; both
// addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// orders this CTA's earlier generic-proxy shared-memory accesses before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Every wait for a bulk copy is bounded by the global nanosecond timer: a wait that has
// not completed after kBulkWaitNs sets ERRBIT_TIMEOUT (the host call then returns
// QEQ_ERR_TIMEOUT) and the CTA gives up.
constexpr uint64_t kBulkWaitNs = 500000000ull;  // 0.5 s
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > kBulkWaitNs) return false;
  }
}

// ------------------------------------------------------------------ mixed-radix stages in shared memory
// A line of K = R_0 ... R_{m-1} points is transformed in place, stage after stage
// (decimation in time over blocks): stage s works on Q_s = R_0...R_{s-1} blocks of
// L_s = K / Q_s points; inside a block, point n + S_s r (S_s = L_s / R_s, n < S_s,
// r < R_s) takes part in butterfly n; an R_s-point DFT over r is followed by the twiddle
// W_{L_s}^{n k} and the outputs go back to n + S_s k.  After the last stage (S = 1) the
// point at position sum_s S_s k_s holds frequency sum_s Q_s k_s ("block order"; the
// host tables blk / freq / pos translate between the two).  Twiddles come from the
// K-point table exp(-2 pi i m / K): W_{L_s}^{n k} = tw[n k Q_s] (n k Q_s < K).
//
// Work assignment: with exactly 8 lines, and in a stage with S_s = 1 and even R_s, the
// lanes run over the lines first, else over n first (elements adjacent in a line).
// Lines are ld = 2 mod 4 elements apart, so 8 lines fill 8 distinct bank pairs and the
// butterflies of two neighbouring n the other 8: the accesses of a half-warp hit
// distinct banks, and its lanes read two twiddles.  The blocks of one line in a stage
// with S_s = 1 start R_s elements apart, which for even R_s would put a warp running
// over them on a few banks.

__device__ __forceinline__ int ceil_log2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <typename T, typename V>
__device__ __forceinline__ V twiddle(const V* __restrict__ tw, int idx, T sgn) {
  V t = tw[idx];
  t.y *= -sgn;  // table holds exp(-2 pi i m/K); sgn = -1 keeps it, +1 conjugates
  return t;
}

// forward-order stage s (DFT of sign sgn, then twiddles), in place on nl lines
template <typename T, int R>
__device__ __forceinline__ void stage_fwd(typename C2<T>::t* tile, int nl, int ld, const FftPlanDev& fp, int s,
                                          const typename C2<T>::t* __restrict__ tw, T sgn) {
  using V = typename C2<T>::t;
  const int S = fp.S[s], L = fp.L[s], Q = fp.Q[s];
  const int nb = fp.K / R;
  const bool lf = (nl == 8) || (R % 2 == 0 && S == 1);  // lanes over lines first (see above)
  const int lsh = ceil_log2(nl);
  const int total = lf ? (nb << lsh) : nl * nb;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int l, j;
    if (lf) {
      l = w & ((1 << lsh) - 1);
      j = w >> lsh;
      if (l >= nl) continue;
    } else {
      l = (int)fdiv((uint32_t)w, fp.fnb[s]);
      j = w - l * nb;
    }
    const int beta = (int)fdiv((uint32_t)j, fp.fS[s]);
    const int n = j - beta * S;
    V* b = tile + l * ld + beta * L + n;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[r * S];
    DftR<T, V, R>::run(v, sgn);
    if (n != 0) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twiddle<T, V>(tw, n * k * Q, sgn));
    }
#pragma unroll
    for (int k = 0; k < R; ++k) b[k * S] = v[k];
  }
}

// the exact inverse of forward stage s (sign -1): conjugate twiddles, then the DFT of
// sign +1 (unnormalised), in place
template <typename T, int R>
__device__ __forceinline__ void stage_inv(typename C2<T>::t* tile, int nl, int ld, const FftPlanDev& fp, int s,
                                          const typename C2<T>::t* __restrict__ tw) {
  using V = typename C2<T>::t;
  const int S = fp.S[s], L = fp.L[s], Q = fp.Q[s];
  const int nb = fp.K / R;
  const bool lf = (nl == 8) || (R % 2 == 0 && S == 1);  // lanes over lines first (see above)
  const int lsh = ceil_log2(nl);
  const int total = lf ? (nb << lsh) : nl * nb;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int l, j;
    if (lf) {
      l = w & ((1 << lsh) - 1);
      j = w >> lsh;
      if (l >= nl) continue;
    } else {
      l = (int)fdiv((uint32_t)w, fp.fnb[s]);
      j = w - l * nb;
    }
    const int beta = (int)fdiv((uint32_t)j, fp.fS[s]);
    const int n = j - beta * S;
    V* b = tile + l * ld + beta * L + n;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[r * S];
    if (n != 0) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twiddle<T, V>(tw, n * k * Q, (T)1));
    }
    DftR<T, V, R>::run(v, (T)1);
#pragma unroll
    for (int k = 0; k < R; ++k) b[k * S] = v[k];
  }
}

// Last forward-order stage (S = 1), straight to global memory in natural order: the
// block whose outputs start at natural index u sits at blk[u]; output k of it is
// frequency u + (K/R) k.  LF: lanes run over lines first (transposed stores, lines
// adjacent in memory); otherwise over u (contiguous stores).  nlp: nl rounded up to a
// power of two, 1 << lsh.
template <typename T, int R, bool LF, class Store>
__device__ __forceinline__ void stage_last(const typename C2<T>::t* tile, int nl, int lsh, int ld,
                                           const FftPlanDev& fp, const int* __restrict__ blk, T sgn, Store store) {
  using V = typename C2<T>::t;
  const int nu = fp.K / R;
  const int m = fp.nst - 1;
  const int total = LF ? (nu << lsh) : nl * nu;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int l, u;
    if (LF) {
      l = w & ((1 << lsh) - 1);
      u = w >> lsh;
      if (l >= nl) continue;
    } else {
      l = (int)fdiv((uint32_t)w, fp.fnb[m]);
      u = w - l * nu;
    }
    const V* b = tile + l * ld + blk[u];
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[r];
    DftR<T, V, R>::run(v, sgn);
#pragma unroll
    for (int k = 0; k < R; ++k) store(l, u + nu * k, v[k]);
  }
}

// The last step of the inverse transform of block-ordered data: the inverse of forward
// stage 0, straight to global memory in natural order (point n + S_0 r).  Lines are
// grouped: line g * nl + l, l < nl; lanes run over l first.
template <typename T, int R, class Store>
__device__ __forceinline__ void stage_inv0_out(const typename C2<T>::t* tile, int ngroups, int nl, int lsh, int ld,
                                               const FftPlanDev& fp, const typename C2<T>::t* __restrict__ tw,
                                               Store store) {
  using V = typename C2<T>::t;
  const int S = fp.S[0];
  const int total = (ngroups * S) << lsh;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int l = w & ((1 << lsh) - 1);
    if (l >= nl) continue;
    const int rest = w >> lsh;
    const int g = (int)fdiv((uint32_t)rest, fp.fS[0]);
    const int n = rest - g * S;
    const int line = g * nl + l;
    const V* b = tile + line * ld + n;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[r * S];
    if (n != 0) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twiddle<T, V>(tw, n * k, (T)1));
    }
    DftR<T, V, R>::run(v, (T)1);
#pragma unroll
    for (int r = 0; r < R; ++r) store(line, n + S * r, v[r]);
  }
}

// dispatch on a stage's radix; radices above 16 exist for FP32 stages only (T is the
// enclosing template's mesh precision)
#define QEQ_RADIX_SWITCH(R, CALL)                  \
  switch (R) {                                     \
    case 2: CALL(2); break;                        \
    case 3: CALL(3); break;                        \
    case 4: CALL(4); break;                        \
    case 5: CALL(5); break;                        \
    case 6: CALL(6); break;                        \
    case 8: CALL(8); break;                        \
    case 9: CALL(9); break;                        \
    case 10: CALL(10); break;                      \
    case 12: CALL(12); break;                      \
    case 15: CALL(15); break;                      \
    case 16: CALL(16); break;                      \
    default:                                       \
      if constexpr (sizeof(T) == 4) {              \
        switch (R) {                               \
          case 18: CALL(18); break;                \
          case 20: CALL(20); break;                \
          case 24: CALL(24); break;                \
          default: break;                          \
        }                                          \
      }                                            \
      break;                                       \
  }

// all stages but the last, in forward order
template <typename T>
__device__ __forceinline__ void stages_fwd_inplace(typename C2<T>::t* tile, int nl, int ld, const FftPlanDev& fp,
                                                   int nstages, const typename C2<T>::t* __restrict__ tw, T sgn) {
  for (int s = 0; s < nstages; ++s) {
#define QEQ_CALL(RR) stage_fwd<T, RR>(tile, nl, ld, fp, s, tw, sgn)
    QEQ_RADIX_SWITCH(fp.radix[s], QEQ_CALL)
#undef QEQ_CALL
    __syncthreads();
  }
}

// ------------------------------------------------------------------ transposing FFT passes
// Mesh layouts (complex elements; one complex mesh after another, Mp elements each; the
// innermost line of every layout is padded to an even length P_d = K_d + (K_d & 1) so
// that every line starts on a 16-byte boundary for the bulk copies):
//   L0 [x][y][z]   spreading writes it, gathering reads it, the inverse z pass works in place
//   L1 [x][z][y]
//   L2 [z][y][x]
//   L3 [z][x][y]
// Every pass reads whole contiguous lines (bulk copies into shared memory), transforms
// them there, and writes either transposed (a tile's lines are adjacent in the output, so
// a warp stores runs of TL elements) or in place:
//   ZF: L0 -> L1 (FFT z)   YF: L1 -> L2 (FFT y)   X: L2 -> L3 (FFT x, multiply, inverse x)
//   YI: L3 -> L0 (inverse FFT y)   ZI: L0 in place (inverse FFT z)
enum { PASS_ZF = 0, PASS_YF = 1, PASS_YI = 2, PASS_ZI = 3 };

// shared-memory line stride: even (16-byte aligned FP32 lines) and 2 mod 4 (transposed
// accesses of lines spread over the banks); FP64: odd
template <typename T>
__host__ __device__ __forceinline__ int fft_smem_ld(int K) {
  if (sizeof(T) == 8) return K | 1;
  int ld = K + (K & 1);
  return (ld & 3) ? ld : ld + 2;
}
// elements of a line copied from global memory (FP32 lines padded to an even length)
template <typename T>
__host__ __device__ __forceinline__ int fft_copy_elems(int K) {
  return sizeof(T) == 4 ? K + (K & 1) : K;
}

// Issue the bulk copies of one work unit into buffer B (one warp): when `tables`, the
// unit's FFT plan, its twiddles and ntab of its int tables (from table t0); then nl mesh
// lines.  extra_tx > 0 (a test hook, see QEQ_FLAG_TEST_STALL) announces more bytes than
// the copies deliver.
template <typename T, class LineSrc>
__device__ __forceinline__ void issue_unit(unsigned char* B, const FftBuf& L, uint64_t* bar,
                                           const FftPlanDev* __restrict__ fsrc, const typename C2<T>::t* twg,
                                           const int* __restrict__ tabs, int t0, int ntab, int nl, int ld,
                                           LineSrc line, int extra_tx, bool tables) {
  using V = typename C2<T>::t;
  const int lane = threadIdx.x & 31;
  const int K = fsrc->K;
  const int twn = sizeof(T) == 4 ? K + (K & 1) : K;
  const int K4 = (K + 3) & ~3;
  const int elems = fft_copy_elems<T>(K);
  const size_t tab_bytes = tables ? sizeof(FftPlanDev) + twn * sizeof(V) + ntab * K4 * 4 : 0;
  if (lane == 0) {
    fence_proxy_async();
    mbar_expect_tx(bar, (uint32_t)(tab_bytes + (size_t)nl * elems * sizeof(V) + extra_tx));
  }
  __syncwarp();
  if (tables) {  // skipped when the buffer already holds this plan's tables
    if (lane == 0) bulk_load(B, fsrc, sizeof(FftPlanDev), bar);
    if (lane == 1) bulk_load(B + L.tw, twg + fsrc->tw_off, (uint32_t)(twn * sizeof(V)), bar);
    if (lane == 2) bulk_load(B + L.tab, tabs + fsrc->tab_off + t0 * K4, (uint32_t)(ntab * K4 * 4), bar);
  }
  V* tile = reinterpret_cast<V*>(B + L.tile);
  for (int l = lane; l < nl; l += 32) bulk_load(tile + (size_t)l * ld, line(l), (uint32_t)(elems * sizeof(V)), bar);
}

// A failed bounded wait: flag it, wait (bounded) for the copies of both buffers, give up.
__device__ __forceinline__ void give_up(int* err, uint64_t* bar, const uint32_t* ph, bool next_issued, int b) {
  if (threadIdx.x == 0) atomicOr(err, ERRBIT_TIMEOUT);
  mbar_wait_bounded(&bar[b], ph[b]);
  if (next_issued) mbar_wait_bounded(&bar[b ^ 1], ph[b ^ 1]);
}

// units of a persistent CTA whose geometry is read once, before the first (static shared
// memory: a few KB); later units compute theirs when they are issued
#ifndef QEQ_FFT_GEO_CACHE
#define QEQ_FFT_GEO_CACHE 128
#endif
// Fill cache[k] = geo(blockIdx.x + k gridDim.x) for this CTA's first units (all threads);
// returns how many.
template <class G, class F>
__device__ __forceinline__ int geo_cache_fill(G* cache, int nunits, F geo) {
  const int G0 = (int)blockIdx.x, GS = (int)gridDim.x;
  const int nmine = (nunits > G0) ? (nunits - G0 + GS - 1) / GS : 0;
  const int n = min(nmine, QEQ_FFT_GEO_CACHE);
  for (int k = threadIdx.x; k < n; k += blockDim.x) cache[k] = geo(G0 + k * GS);
  __syncthreads();
  return n;
}

// The warp that issues a pass's bulk copies: the last one, which the stages leave idle
// whenever a unit has fewer butterflies than the CTA has threads (the copies of the next
// unit are issued once the current unit's data has arrived, while the stages run).
__device__ __forceinline__ bool fft_issuer_warp() { return (threadIdx.x >> 5) == (blockDim.x >> 5) - 1; }

// Persistent, two-slot pipeline: CTA b takes work units b, b + G, b + 2G, ... (a unit is a
// sub-tile of `sub` lines of an item); the bulk copies of the next unit are in flight while
// the current one is transformed.
template <typename T, int PASS>
__global__ void __launch_bounds__(sizeof(T) == 4 ? QEQ_FFT_THREADS32 : 256, fft_min_blocks<T>())
    k_fft_tile(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl, const int4* __restrict__ items,
               int nitems, int TL, int sub, int Kmax, int ldmax, const double2* __restrict__ tw64,
               const float2* __restrict__ tw32, const int* __restrict__ tabs, const PcgScalars* __restrict__ sc,
               int use_active, const typename C2<T>::t* src, typename C2<T>::t* dst, int* __restrict__ err) {
  // src and dst are the same buffer in the in-place inverse z pass (no __restrict__)
  using V = typename C2<T>::t;
  constexpr bool isZ = (PASS == PASS_ZF || PASS == PASS_ZI);
  constexpr bool fwd = (PASS == PASS_ZF || PASS == PASS_YF);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  const FftBuf L = fft_buf(Kmax, ldmax, sub, (int)sizeof(V), 1, 0);
  unsigned char* bufs = smem_raw + 128;
  __shared__ int buf_plan[2];  // FFT plan whose tables each buffer holds (read and written by the issuer)
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    buf_plan[0] = buf_plan[1] = -1;
  }
  __syncthreads();
  const int nsub = (TL + sub - 1) / sub;
  const int nunits = nitems * nsub;
  const V* twg = twiddles<T>(tw64, tw32);
  const T sgn = fwd ? (T)-1 : (T)1;
  // unit u: sub-tile (u mod nsub) of item u / nsub
  struct Geo {
    int ok, plan, K, nl;
    int64_t in0, out0;
    int ils, ols, oes, pad;
  };
  auto geo = [&](int u) {
    Geo g;
    g.ok = 0;
    if (u >= nunits) return g;
    const int i = u / nsub, part = u - i * nsub;
    const int4 it = items[i];  // ZF, ZI: {s, c, x, y0}; YF: {s, c, z, x0}; YI: {s, c, x, z0}
    if (use_active && !sc[it.x].active) return g;
    const StructDev& S = st[it.x];
    const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
    const int P0 = S.P[0], P1 = S.P[1], P2 = S.P[2];
    const int nitem = min(TL, (isZ ? K1 : (PASS == PASS_YF ? K0 : K2)) - it.w);
    g.nl = min(sub, nitem - part * sub);
    if (g.nl <= 0) return g;
    g.ok = 1;
    g.plan = S.fft_plan[isZ ? 2 : 1] + fft_plan_variant<T>();
    g.K = isZ ? K2 : K1;
    const int64_t mb = S.mesh_off + (int64_t)it.y * S.Mp;
    // line l starts at in0 + l ils; element e of line l goes to out0 + l ols + e oes
    int64_t ib, ob;
    if (PASS == PASS_ZF) {
      ib = ((int64_t)it.z * K1 + it.w) * P2; g.ils = P2;
      ob = (int64_t)it.z * K2 * P1 + it.w; g.ols = 1; g.oes = P1;
    } else if (PASS == PASS_ZI) {
      ib = ((int64_t)it.z * K1 + it.w) * P2; g.ils = P2;
      ob = ib; g.ols = P2; g.oes = 1;
    } else if (PASS == PASS_YF) {
      ib = ((int64_t)it.w * K2 + it.z) * P1; g.ils = K2 * P1;
      ob = (int64_t)it.z * K1 * P0 + it.w; g.ols = 1; g.oes = P0;
    } else {
      ib = ((int64_t)it.w * K0 + it.z) * P1; g.ils = K0 * P1;
      ob = (int64_t)it.z * K1 * P2 + it.w; g.ols = 1; g.oes = P2;
    }
    (void)P0;
    g.in0 = mb + ib + (int64_t)part * sub * g.ils;
    g.out0 = mb + ob + (int64_t)part * sub * g.ols;
    return g;
  };
  // the geometry of this CTA's first QEQ_FFT_GEO_CACHE units, read at once: the chain of
  // global loads behind it would otherwise delay every unit's copies and first barrier
  __shared__ Geo gcache[QEQ_FFT_GEO_CACHE];
  const int ncache = geo_cache_fill(gcache, nunits, geo);
  auto geo_k = [&](int k, int u) { return (k < ncache) ? gcache[k] : geo(u); };
  auto issue = [&](const Geo& g, int b) {  // the issuer warp
    issue_unit<T>(bufs + (size_t)b * L.bytes, L, &bar[b], fpl + g.plan, twg, tabs, 0, 1, g.nl,
                  fft_smem_ld<T>(g.K), [&](int l) { return src + g.in0 + (int64_t)l * g.ils; }, 0,
                  buf_plan[b] != g.plan);
    if ((threadIdx.x & 31) == 0) buf_plan[b] = g.plan;
  };
  uint32_t ph[2] = {0u, 0u};
  const bool issuer = fft_issuer_warp();
  int u = blockIdx.x, k = 0;
  if (issuer) {
    const Geo g0 = geo_k(0, u);
    if (g0.ok) issue(g0, 0);
  }
  for (; u < nunits; u += gridDim.x, ++k) {
    const int b = k & 1;
    const Geo cur = geo_k(k, u);
    if (cur.ok) {
      bool ok = __syncthreads_and(mbar_wait_bounded(&bar[b], ph[b]));
      if (!ok) {
        give_up(err, bar, ph, false, b);  // only this unit's copies are in flight
        return;
      }
      ph[b] ^= 1u;
    }
    if (issuer) {  // the next unit into buffer b^1 (released at the end of the last unit)
      const Geo nxt = geo_k(k + 1, u + gridDim.x);
      if (nxt.ok) issue(nxt, b ^ 1);
    }
    if (cur.ok) {
      unsigned char* B = bufs + (size_t)b * L.bytes;
      const FftPlanDev& fp = *reinterpret_cast<const FftPlanDev*>(B);
      const V* tw = reinterpret_cast<const V*>(B + L.tw);
      const int* blk = reinterpret_cast<const int*>(B + L.tab);
      V* tile = reinterpret_cast<V*>(B + L.tile);
      const int ld = fft_smem_ld<T>(cur.K), nl = cur.nl;
      stages_fwd_inplace<T>(tile, nl, ld, fp, fp.nst - 1, tw, sgn);
      int lsh = 0;
      while ((1 << lsh) < nl) ++lsh;
      V* o = dst + cur.out0;
      const int64_t ols = cur.ols, oes = cur.oes;  // 64-bit products below
      auto store = [&](int l, int e, V v) { o[l * ols + e * oes] = v; };
#define QEQ_CALL(RR)                                                                      \
  if (PASS == PASS_ZI)                                                                    \
    stage_last<T, RR, false>(tile, nl, lsh, ld, fp, blk, sgn, store);                     \
  else                                                                                    \
    stage_last<T, RR, true>(tile, nl, lsh, ld, fp, blk, sgn, store)
      QEQ_RADIX_SWITCH(fp.radix[fp.nst - 1], QEQ_CALL)
#undef QEQ_CALL
      __syncthreads();  // the buffer is free for the unit after next
    }
  }
}

// exp2 and 1/x in the mesh precision: the FP32 path uses the hardware
// approximations (ex2.approx: relative error ~2^-22 plus the argument's own
// rounding, which only matters where the Gaussian is already below ~1e-8 of its
// peak; rcp with round-to-nearest), the FP64 path the exact library calls.
template <typename T>
__device__ __forceinline__ T exp2_mesh(T x);
template <>
__device__ __forceinline__ float exp2_mesh<float>(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <>
__device__ __forceinline__ double exp2_mesh<double>(double x) {
  return exp2(x);
}
template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) {
  return __frcp_rn(x);
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return 1.0 / x;
}
// double-float: through FP64 (once per reciprocal-space point, not per butterfly)
template <>
__device__ __forceinline__ dd exp2_mesh<dd>(dd x) {
  return dd(exp2((double)x));
}
template <>
__device__ __forceinline__ dd recip<dd>(dd x) {
  return dd(1.0 / (double)x);
}

// largest x = s0 g0 of the smoothest preconditioner mode for which beta = 1 is used
// (112 on a 13.8k-atom rock-salt cell: 17 iterations against 25 with beta = 0.98;
// cells of x ~ 450 and more need beta < 1)
constexpr double kPreBetaOneX = 150.0;

// ------------------------------------------------------------------ x: FFT, reciprocal multiply, inverse FFT
// An item holds np lines (z, y0..y0+np-1) of layout L2 and their mirror lines (-z, -y):
// the reciprocal multiply needs Z(m) and Z(-m) of every complex mesh to separate its two
// species.  Items cover z <= K2/2 (and y <= K1/2 on the planes z = 0, K2/2, which are
// their own mirrors), so every line is written once.  The forward x FFT leaves each line
// in block order, the multiply works there (tables freq / pos), and the inverse FFT runs
// the stages backwards and writes layout L3 [z][x][y] (np adjacent y per x).
// MAXS: most species of any structure of the plan (2: one complex mesh, the common case;
// 8: any).
// VIR: instead of the multiply and the inverse FFT, the strain derivative of the
// reciprocal energy Q(x) = sum_m sum_st conj(x_s(m)) g_st(m) x_t(m) of the charges on
// the mesh (the quadratic form behind the matvec): g_st = (4 pi/V) b(m) exp(-G^2 w_st^2/2)/G^2
// changes with a homogeneous strain through dG^2/d eps_ab = -2 G_a G_b and dV = V tr(eps),
//   dQ/d eps_ab = sum_m sum_st E_st(m) [-delta_ab + G_a G_b (w_st^2 + 2/G^2)].
// Each unit writes its 7 sums {sum E, (sum E_st (w_st^2 + 2/G^2)) G_a G_b for ab = xx, yy,
// zz, xy, xz, yz} to vir[8 u ..] (dst reinterpreted), in a fixed order: a line that is
// not its own mirror stands for itself and its mirror (weight 2).
template <typename T, bool PRE, int MAXS, bool VIR = false>
__global__ void __launch_bounds__(sizeof(T) == 4 ? QEQ_FFT_THREADS32 : 256, fft_min_blocks<T>())
    k_fft_x_green(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl,
                  const int4* __restrict__ items, int nitems, int TLX, int sub, int Kmax, int ldmax,
                  const T* __restrict__ bmod, const double2* __restrict__ tw64, const float2* __restrict__ tw32,
                  const int* __restrict__ tabs, const PcgScalars* __restrict__ sc, int use_active,
                  const typename C2<T>::t* __restrict__ src, typename C2<T>::t* __restrict__ dst,
                  int* __restrict__ err, int stall) {
  using V = typename C2<T>::t;
  constexpr int HX = MAXS / 2;  // most complex meshes
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  const FftBuf L = fft_buf(Kmax, ldmax, 2 * HX * sub, (int)sizeof(V), 2, fft_x_extra(sub, HX, (int)sizeof(T)));
  unsigned char* bufs = smem_raw + 128;
  __shared__ T hw2[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];
  __shared__ int hw2_s;
  __shared__ int buf_plan[2];  // FFT plan whose tables each buffer holds (read and written by the issuer)
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    hw2_s = -1;
    buf_plan[0] = buf_plan[1] = -1;
  }
  __syncthreads();
  const int nsub = (TLX + sub - 1) / sub;
  const int nunits = nitems * nsub;
  const V* twg = twiddles<T>(tw64, tw32);
  // unit u: pairs [j0, j0 + np) of item u / nsub, j0 = (u mod nsub) sub
  struct Geo {
    int ok, s, z, y0, np;
  };
  auto geo = [&](int u) {
    Geo g;
    g.ok = 0;
    if (u >= nunits) return g;
    const int i = u / nsub, part = u - i * nsub;
    const int4 it = items[i];  // {struct, z, y0, number of lines}
    if (use_active && !sc[it.x].active) return g;
    g.np = min(sub, it.w - part * sub);
    if (g.np <= 0) return g;
    g.ok = 1;
    g.s = it.x;
    g.z = it.y;
    g.y0 = it.z + part * sub;
    return g;
  };
  __shared__ Geo gcache[QEQ_FFT_GEO_CACHE];  // this CTA's first units (see geo_cache_fill)
  const int ncache = geo_cache_fill(gcache, nunits, geo);
  auto geo_k = [&](int k, int u) { return (k < ncache) ? gcache[k] : geo(u); };
  // the issuer warp: slot tables and line constants of the unit in buffer b, then its copies
  auto issue = [&](const Geo& g, int b, int extra) {
    const StructDev& S = st[g.s];
    const int K = S.K[0], K1 = S.K[1], K2 = S.K[2], P0 = S.P[0], P1 = S.P[1], ncm = S.ncm;
    unsigned char* B = bufs + (size_t)b * L.bytes;
    int64_t* slot_in = reinterpret_cast<int64_t*>(B + L.extra);
    int64_t* slot_out = slot_in + 2 * HX * sub;
    T(*lineg)[4] = reinterpret_cast<T(*)[4]>(slot_out + 2 * HX * sub);
    const int np = g.np, nsl = 2 * ncm * np, z = g.z, mz = (K2 - z) % K2;
    const int lane = threadIdx.x & 31;
    for (int sl = lane; sl < nsl; sl += 32) {  // slot (ab * ncm + c) * np + l
      const int l = sl % np, gc = sl / np, c = gc % ncm, ab = gc / ncm;
      const int y = g.y0 + l;
      const int yy = ab ? (K1 - y) % K1 : y, zz = ab ? mz : z;
      const int64_t mb = S.mesh_off + (int64_t)c * S.Mp;
      slot_in[sl] = mb + ((int64_t)zz * K1 + yy) * P0;
      slot_out[sl] = (ab && zz == z && yy == y) ? -1 : mb + (int64_t)zz * K * P1 + yy;  // self-paired copy
    }
    const T* bm1 = bmod + S.bmod_off[1];
    const T* bm2 = bmod + S.bmod_off[2];
    const int c2 = (z <= K2 / 2) ? z : z - K2;
    for (int l = lane; l < np; l += 32) {
      const int my = g.y0 + l;
      const int c1 = (my <= K1 / 2) ? my : my - K1;
      lineg[l][0] = (T)(c1 * S.B[3] + c2 * S.B[6]);
      lineg[l][1] = (T)(c1 * S.B[4] + c2 * S.B[7]);
      lineg[l][2] = (T)(c1 * S.B[5] + c2 * S.B[8]);
      lineg[l][3] = (T)S.green_pref * bm1[my] * bm2[z];
    }
    __syncwarp();
    const int plan = S.fft_plan[0] + fft_plan_variant<T>();
    issue_unit<T>(B, L, &bar[b], fpl + plan, twg, tabs, 1, 2, nsl, fft_smem_ld<T>(K),
                  [&](int sl) { return src + slot_in[sl]; }, extra, buf_plan[b] != plan);
    if (lane == 0) buf_plan[b] = plan;
  };
  uint32_t ph[2] = {0u, 0u};
  const bool issuer = fft_issuer_warp();
  int u = blockIdx.x, k = 0;
  if (issuer) {
    const Geo g0 = geo_k(0, u);
    if (g0.ok) issue(g0, 0, (stall && blockIdx.x == 0) ? 16 : 0);
  }
  for (; u < nunits; u += gridDim.x, ++k) {
    const int b = k & 1;
    const Geo cur = geo_k(k, u);
    if (cur.ok) {
      bool ok = __syncthreads_and(mbar_wait_bounded(&bar[b], ph[b]));
      if (!ok) {
        give_up(err, bar, ph, false, b);  // only this unit's copies are in flight
        return;
      }
      ph[b] ^= 1u;
    }
    if (issuer) {  // the next unit into buffer b^1 (released at the end of the last unit)
      const Geo nxt = geo_k(k + 1, u + gridDim.x);
      if (nxt.ok) issue(nxt, b ^ 1, 0);
    }
    if (!cur.ok) {
      if constexpr (VIR) {
        if (threadIdx.x < 8) reinterpret_cast<double*>(dst)[8 * (int64_t)u + threadIdx.x] = 0.0;
      }
      continue;
    }
    const StructDev& S = st[cur.s];
    const int K = S.K[0], P1 = S.P[1], ncm = S.ncm, np = cur.np, nsl = 2 * ncm * np;
    const int ld = fft_smem_ld<T>(K);
    unsigned char* B = bufs + (size_t)b * L.bytes;
    const FftPlanDev& fp = *reinterpret_cast<const FftPlanDev*>(B);
    const V* tw = reinterpret_cast<const V*>(B + L.tw);
    const int K4 = (K + 3) & ~3;
    const int* freq = reinterpret_cast<const int*>(B + L.tab);
    const int* pos = freq + K4;
    const int64_t* slot_out = reinterpret_cast<const int64_t*>(B + L.extra) + 2 * HX * sub;
    const T(*lineg)[4] = reinterpret_cast<const T(*)[4]>(slot_out + 2 * HX * sub);
    V* tile = reinterpret_cast<V*>(B + L.tile);
    if (hw2_s != cur.s) {  // exponent factors -w_st^2/2 log2(e) of this structure
      __syncthreads();
      for (int i = threadIdx.x; i < QEQ_MAX_SPECIES * QEQ_MAX_SPECIES; i += blockDim.x)
        hw2[i] = (T)(-0.5 * 1.44269504088896340736 * S.w2[i]);
      if (threadIdx.x == 0) hw2_s = cur.s;
      __syncthreads();
    }
    const T* bm0 = bmod + S.bmod_off[0];
    const T B0 = (T)S.B[0], B1 = (T)S.B[1], B2 = (T)S.B[2];
    const T gpref = (T)S.green_pref;
    // beta: 1 (the plain Woodbury factor) while the smoothest mode's x = s0 g0 stays small,
    // else the plan's safety factor (S.omega holds it for the preconditioner mesh); large
    // cells need it because the correction nearly cancels D^-1 for their smooth modes and
    // the circulant mean's error would then make M indefinite
    const T pre_beta = PRE ? ((sc[cur.s].s0 * S.pre_g0max <= kPreBetaOneX) ? (T)1 : (T)S.omega) : (T)0;
    const T pre_s0 = PRE ? (T)sc[cur.s].s0 : (T)0;
    const int nspec = S.S;
    // forward x FFT, every stage in place: block order
    stages_fwd_inplace<T>(tile, nsl, ld, fp, fp.nst, tw, (T)-1);
    if constexpr (VIR) {
      const int K1 = S.K[1], K2 = S.K[2];
      double acc[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int w = threadIdx.x; w < np * K; w += blockDim.x) {
        const int l = (int)fdiv((uint32_t)w, fp.fK), p = w - l * K;
        const int mx = freq[p];
        const int mmx = (mx == 0) ? 0 : K - mx;
        const int p2 = pos[mmx];
        const int c0 = (mx <= K / 2) ? mx : mx - K;
        const double Gx = (double)c0 * S.B[0] + (double)lineg[l][0];
        const double Gy = (double)c0 * S.B[1] + (double)lineg[l][1];
        const double Gz = (double)c0 * S.B[2] + (double)lineg[l][2];
        const double G2 = Gx * Gx + Gy * Gy + Gz * Gz;
        if (!(G2 > 0.0)) continue;  // G = 0 term dropped
        const double rG2 = 1.0 / G2;
        const int y = cur.y0 + l;
        const double wt = ((K1 - y) % K1 == y && (K2 - cur.z) % K2 == cur.z) ? 1.0 : 2.0;
        const double pref = wt * (double)lineg[l][3] * (double)bm0[mx] * rG2;
        V Qh[MAXS];
#pragma unroll
        for (int c = 0; c < HX; ++c) {
          if (c >= ncm) break;
          const V za = tile[(size_t)(c * np + l) * ld + p];
          const V zb = tile[(size_t)((ncm + c) * np + l) * ld + p2];
          Qh[2 * c] = {(T)0.5 * (za.x + zb.x), (T)0.5 * (za.y - zb.y)};
          Qh[2 * c + 1] = {(T)0.5 * (za.y + zb.y), (T)-0.5 * (za.x - zb.x)};
        }
        double e = 0.0, k = 0.0;
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
          if (s >= nspec) break;
#pragma unroll
          for (int t = 0; t < MAXS; ++t) {
            if (t >= nspec) break;
            const int st_ = s * QEQ_MAX_SPECIES + t;
            const double E = pref * exp2_mesh<double>(G2 * (double)hw2[st_]) *
                             ((double)Qh[s].x * Qh[t].x + (double)Qh[s].y * Qh[t].y);
            e += E;
            k += E * (S.w2[st_] + 2.0 * rG2);
          }
        }
        acc[0] += e;
        acc[1] += k * Gx * Gx;
        acc[2] += k * Gy * Gy;
        acc[3] += k * Gz * Gz;
        acc[4] += k * Gx * Gy;
        acc[5] += k * Gx * Gz;
        acc[6] += k * Gy * Gz;
      }
      // fixed-order block sums: shuffle tree per warp, then warps in order
      __shared__ double vred[7][8];  // VIR: FP64 kernels, 256 threads
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        double a = acc[i];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) vred[i][threadIdx.x >> 5] = a;
      }
      __syncthreads();
      if (threadIdx.x < 8) {
        double a = 0.0;
        if (threadIdx.x < 7)
          for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += vred[threadIdx.x][i];
        reinterpret_cast<double*>(dst)[8 * (int64_t)u + threadIdx.x] = a;
      }
      __syncthreads();  // the buffer is free for the unit after next
    } else {
    // reciprocal multiply; each Gaussian is one exp2
    for (int w = threadIdx.x; w < np * K; w += blockDim.x) {
      const int l = (int)fdiv((uint32_t)w, fp.fK), p = w - l * K;
      const int mx = freq[p];
      const int mmx = (mx == 0) ? 0 : K - mx;
      const int p2 = pos[mmx];
      const int c0 = (mx <= K / 2) ? mx : mx - K;
      const T Gx = (T)c0 * B0 + lineg[l][0];
      const T Gy = (T)c0 * B1 + lineg[l][1];
      const T Gz = (T)c0 * B2 + lineg[l][2];
      const T G2 = Gx * Gx + Gy * Gy + Gz * Gz;
      const T rG2 = (G2 > (T)0) ? recip<T>(G2) : (T)0;
      const T pref = lineg[l][3] * bm0[mx] * rG2;  // G = 0 term dropped
      V Qh[MAXS];
#pragma unroll
      for (int c = 0; c < HX; ++c) {
        if (c >= ncm) break;
        const V za = tile[(size_t)(c * np + l) * ld + p];
        const V zb = tile[(size_t)((ncm + c) * np + l) * ld + p2];
        // F[Q_2c] = (Z(m) + conj Z(-m))/2,  F[Q_2c+1] = (Z(m) - conj Z(-m))/(2i)
        Qh[2 * c] = {(T)0.5 * (za.x + zb.x), (T)0.5 * (za.y - zb.y)};
        Qh[2 * c + 1] = {(T)0.5 * (za.y + zb.y), (T)-0.5 * (za.x - zb.x)};
      }
#pragma unroll
      for (int c = 0; c < HX; ++c) {
        if (c >= ncm) break;
        V p0 = {(T)0, (T)0}, p1 = {(T)0, (T)0};
        if (PRE) {
          // Fourier preconditioner: h(m) = beta |b(m)|^2 g0 / (1 + s0 g0),
          // g0 = k_e (4 pi/V) exp(-G^2 w^2/2)/G^2 (see pre_beta)
          const T e = exp2_mesh<T>(G2 * hw2[0]);
          const T g0 = gpref * e * rG2;
          const T hm = pre_beta * pref * e * recip<T>((T)1 + pre_s0 * g0);
          p0.x = hm * Qh[0].x;
          p0.y = hm * Qh[0].y;
        } else if (MAXS == 2) {
          // g_st = g_ts: three Gaussians for the two species of the complex mesh
          const T g00 = pref * exp2_mesh<T>(G2 * hw2[0]);
          if (nspec > 1) {
            const T g01 = pref * exp2_mesh<T>(G2 * hw2[1]);
            const T g11 = pref * exp2_mesh<T>(G2 * hw2[QEQ_MAX_SPECIES + 1]);
            p0.x = g00 * Qh[0].x + g01 * Qh[1].x;
            p0.y = g00 * Qh[0].y + g01 * Qh[1].y;
            p1.x = g01 * Qh[0].x + g11 * Qh[1].x;
            p1.y = g01 * Qh[0].y + g11 * Qh[1].y;
          } else {
            p0.x = g00 * Qh[0].x;
            p0.y = g00 * Qh[0].y;
          }
        } else {
#pragma unroll
          for (int t = 0; t < MAXS; ++t) {
            if (t >= nspec) break;
            const T g0 = pref * exp2_mesh<T>(G2 * hw2[(2 * c) * QEQ_MAX_SPECIES + t]);
            p0.x += g0 * Qh[t].x;
            p0.y += g0 * Qh[t].y;
            if (2 * c + 1 < nspec) {
              const T g1 = pref * exp2_mesh<T>(G2 * hw2[(2 * c + 1) * QEQ_MAX_SPECIES + t]);
              p1.x += g1 * Qh[t].x;
              p1.y += g1 * Qh[t].y;
            }
          }
        }
        // W(m) = P_2c + i P_2c+1 ; W(-m) = conj(P_2c) + i conj(P_2c+1)
        tile[(size_t)(c * np + l) * ld + p] = {p0.x - p1.y, p0.y + p1.x};
        tile[(size_t)((ncm + c) * np + l) * ld + p2] = {p0.x + p1.y, -p0.y + p1.x};
      }
    }
    __syncthreads();
    // inverse x FFT: the forward stages undone in reverse order, the last one to layout L3
    for (int s = fp.nst - 1; s >= 1; --s) {
#define QEQ_CALL(RR) stage_inv<T, RR>(tile, nsl, ld, fp, s, tw)
      QEQ_RADIX_SWITCH(fp.radix[s], QEQ_CALL)
#undef QEQ_CALL
      __syncthreads();
    }
    int lsh = 0;
    while ((1 << lsh) < np) ++lsh;
    auto store = [&](int sl, int e, V v) {
      const int64_t bo = slot_out[sl];
      if (bo >= 0) dst[bo + (int64_t)e * P1] = v;
    };
#define QEQ_CALL(RR) stage_inv0_out<T, RR>(tile, 2 * ncm, np, lsh, ld, fp, tw, store)
    QEQ_RADIX_SWITCH(fp.radix[0], QEQ_CALL)
#undef QEQ_CALL
    __syncthreads();  // the buffer is free for the unit after next
    }  // VIR
  }
}

}  // namespace
