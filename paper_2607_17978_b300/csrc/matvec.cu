// The plane-wave matrix-vector product y = (E + diag J) x of eq. (matvec)
// (Sec. 2.4 "Electrostatics Solvers"), Ewald-split as in SI "Ewald Summation":
//
//   y_i = sum_k theta_i(k) phi_{s_i}[k]                       (mesh part)
//       + sum_{j,n} v_ij x_j                                  (real space, narrow pairs)
//       + (J_i + self_{s_i}) x_i - sum_t corr_{s_i t} X_t     (local terms)
//
//   Q_t[k]        = sum_{i in t} x_i theta_i(k)               B-spline spreading
//   phi_s         = F^-1[ sum_t g_st(m) F[Q_t](m) ]           FFT, reciprocal multiply, inverse FFT
//   g_st(m)       = k_e (4 pi/V) exp(-G^2 w_st^2/2) / G^2 |b(m)|^2,  g(0) = 0
//
// Two species share one complex mesh (species 2c in the real part, 2c+1 in
// the imaginary part), so every FFT is complex-to-complex; the reciprocal
// multiply separates them with Z(m) and conj(Z(-m)).  The x-direction FFT,
// the multiply and the inverse x-direction FFT run in one kernel over pairs of
// mesh lines (y,z) and (-y,-z).  Spreading and gathering work on 8^3 bricks
// whose atoms were sorted by prep.cu; spreading accumulates in per-warp shared
// copies of the brick (no atomics, fixed order) and writes each mesh point once.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "qeq_internal.cuh"

namespace {

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

// Asynchronous global -> shared copy of one complex element (cp.async): a thread
// issues all its copies back to back and waits once, so many loads are in flight.
__device__ __forceinline__ void cp_async_elem(float2* smem, const float2* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* smem, const double2* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

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
#undef QEQ_COMPOSITE_DFT

// One Stockham radix-R stage over all lines in shared memory (padded layout).
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const typename C2<T>::t* __restrict__ src,
                                               typename C2<T>::t* __restrict__ dst, int nlines, int K, int ld, int Ns,
                                               const typename C2<T>::t* __restrict__ tw, T sgn,
                                               const FastDiv& fnbf, const FastDiv& fns) {
  using V = typename C2<T>::t;
  const int nbf = K / R;
  const int tws = K / (Ns * R);
  const int total = nlines * nbf;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int line = (int)fdiv((uint32_t)w, fnbf);
    const int j = w - line * nbf;
    const int jq = (int)fdiv((uint32_t)j, fns);
    const int k = j - jq * Ns;
    const V* s = src + line * ld;
    V* d = dst + line * ld;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[fft_pidx(j + r * nbf)];
    if (Ns > 1) {  // the first stage has k = 0: all its twiddles are 1
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V t = tw[r * k * tws];
        t.y *= -sgn;  // table holds exp(-2 pi i m/K); sgn = -1 keeps it, +1 conjugates
        v[r] = cmul(v[r], t);
      }
    }
    DftR<T, V, R>::run(v, sgn);
    const int o = jq * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[fft_pidx(o + r * Ns)] = v[r];
  }
}

// Unnormalised FFT of nlines lines of length K held in a; returns the buffer with the result.
template <typename T>
__device__ typename C2<T>::t* fft_lines(typename C2<T>::t* a, typename C2<T>::t* b, int nlines, int K, int ld,
                                        const FftPlanDev& fp, const typename C2<T>::t* tw, T sgn) {
  int Ns = 1;
  for (int st = 0; st < fp.nst; ++st) {
    const int R = fp.radix[st];
    switch (R) {
#define QEQ_STAGE(RR) \
  case RR:            \
    stockham_stage<T, RR>(a, b, nlines, K, ld, Ns, tw, sgn, fp.nbf[st], fp.ns[st]); \
    break;
      QEQ_STAGE(2)
      QEQ_STAGE(3)
      QEQ_STAGE(4)
      QEQ_STAGE(5)
      QEQ_STAGE(6)
      QEQ_STAGE(8)
      QEQ_STAGE(9)
      QEQ_STAGE(10)
      QEQ_STAGE(12)
      QEQ_STAGE(15)
      QEQ_STAGE(16)
#undef QEQ_STAGE
      default:
        break;
    }
    __syncthreads();
    typename C2<T>::t* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

template <typename T>
__device__ __forceinline__ void load_twiddles(typename C2<T>::t* tw_s, const double2* tw64, const float2* tw32,
                                              const FftPlanDev& fp) {
  const typename C2<T>::t* g = twiddles<T>(tw64, tw32) + fp.tw_off;
  for (int m = threadIdx.x; m < fp.K; m += blockDim.x) cp_async_elem(tw_s + m, g + m);
}

// ------------------------------------------------------------------ transposing FFT passes
// Mesh layouts (complex elements, one complex mesh after another):
//   L0 [x][y][z]   spreading writes it, gathering reads it
//   L1 [x][z][y]
//   L2 [z][y][x]   the x pass (FFT, reciprocal multiply, inverse FFT) works on it in place
// Every pass reads whole contiguous lines or tiles of TL consecutive lines, and
// writes the other way round, so global loads and stores are full segments:
//   ZF: L0 -> L1 (FFT z)   YF: L1 -> L2 (FFT y)   X: L2 in place
//   YI: L2 -> L1 (inverse FFT y)                  ZI: L1 -> L0 (inverse FFT z)
enum { PASS_ZF = 0, PASS_YF = 1, PASS_YI = 2, PASS_ZI = 3 };

template <typename T, int PASS>
__global__ void __launch_bounds__(256) k_fft_pass(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl,
                                                  const int4* __restrict__ items, const double2* __restrict__ tw64,
                                                  const float2* __restrict__ tw32, const PcgScalars* __restrict__ sc,
                                                  int use_active, const typename C2<T>::t* __restrict__ src,
                                                  typename C2<T>::t* __restrict__ dst, int TL) {
  using V = typename C2<T>::t;
  constexpr bool isZ = (PASS == PASS_ZF || PASS == PASS_ZI);
  constexpr bool fwd = (PASS == PASS_ZF || PASS == PASS_YF);
  const int4 it = items[blockIdx.x];  // Z passes: {s, c, x, y0};  Y passes: {s, c, z, x0}
  const StructDev& S = st[it.x];
  if (use_active && !sc[it.x].active) return;
  const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
  const FftPlanDev& fp = fpl[S.fft_plan[isZ ? 2 : 1]];
  const int K = isZ ? K2 : K1;
  const int nl = min(TL, (isZ ? K1 : K0) - it.w);
  const int64_t mb = S.mesh_off + (int64_t)it.y * S.M;
  // element e of line l is at base + l * ls + e * es
  int64_t ib, ob, ils, ies, ols, oes;
  if (PASS == PASS_ZF) {        // L0 (x, y0+l, e) -> L1 (x, e, y0+l)
    ib = ((int64_t)it.z * K1 + it.w) * K2; ils = K2; ies = 1;
    ob = (int64_t)it.z * K2 * K1 + it.w; ols = 1; oes = K1;
  } else if (PASS == PASS_ZI) { // L1 -> L0
    ib = (int64_t)it.z * K2 * K1 + it.w; ils = 1; ies = K1;
    ob = ((int64_t)it.z * K1 + it.w) * K2; ols = K2; oes = 1;
  } else if (PASS == PASS_YF) { // L1 (x0+l, z, e) -> L2 (z, e, x0+l)
    ib = ((int64_t)it.w * K2 + it.z) * K1; ils = (int64_t)K2 * K1; ies = 1;
    ob = (int64_t)it.z * K1 * K0 + it.w; ols = 1; oes = K0;
  } else {                      // L2 -> L1
    ib = (int64_t)it.z * K1 * K0 + it.w; ils = 1; ies = K0;
    ob = ((int64_t)it.w * K2 + it.z) * K1; ols = (int64_t)K2 * K1; oes = 1;
  }
  const int ld = fft_ld(K);  // padded shared lines: transposed accesses spread over the banks
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + K;
  V* b = a + nl * ld;
  load_twiddles<T>(tw_s, tw64, tw32, fp);
  const FastDiv fnl = make_fastdiv(nl);
  const V* g = src + mb + ib;
  if (ies == 1) {
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
      int l = (int)fdiv((uint32_t)idx, fp.k), e = idx - l * K;
      cp_async_elem(a + l * ld + fft_pidx(e), g + l * ils + e);
    }
  } else {
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
      int e = (int)fdiv((uint32_t)idx, fnl), l = idx - e * nl;
      cp_async_elem(a + l * ld + fft_pidx(e), g + e * ies + l);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  V* res = fft_lines<T>(a, b, nl, K, ld, fp, tw_s, fwd ? (T)-1 : (T)1);
  V* o = dst + mb + ob;
  if (oes == 1) {
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
      int l = (int)fdiv((uint32_t)idx, fp.k), e = idx - l * K;
      o[l * ols + e] = res[l * ld + fft_pidx(e)];
    }
  } else {
    for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
      int e = (int)fdiv((uint32_t)idx, fnl), l = idx - e * nl;
      o[e * oes + l] = res[l * ld + fft_pidx(e)];
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

// largest x = s0 g0 of the smoothest preconditioner mode for which beta = 1 is used
// (112 on a 13.8k-atom rock-salt cell: 17 iterations against 25 with beta = 0.98;
// cells of x ~ 450 and more need beta < 1)
constexpr double kPreBetaOneX = 150.0;

// ------------------------------------------------------------------ x: FFT, reciprocal multiply, inverse FFT
// Works in place on layout L2 [z][y][x], where every x line is contiguous.
// An item holds pairs of lines (z, y) and (-z, -y): the reciprocal multiply
// needs Z(m) and Z(-m) of every complex mesh to separate its two species.
// MAXS: most species of any structure of the plan (2: one complex mesh, the
// common case, with small register use; 8: any).
template <typename T, bool PRE, int MAXS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_x_green(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl,
                              const int4* __restrict__ items, const int2* __restrict__ xpairs,
                              const T* __restrict__ bmod, const double2* __restrict__ tw64,
                              const float2* __restrict__ tw32, const PcgScalars* __restrict__ sc,
                              int use_active, typename C2<T>::t* __restrict__ mesh) {
  using V = typename C2<T>::t;
  int4 it = items[blockIdx.x];  // {struct, first pair (global), npairs, -}
  const StructDev& S = st[it.x];
  if (use_active && !sc[it.x].active) return;
  const FftPlanDev& fp = fpl[S.fft_plan[0]];
  const int K = S.K[0], K1 = S.K[1], K2 = S.K[2];
  const int ncm = S.ncm, np = it.z;
  const int nslot = 2 * np * ncm;
  const int ld = fft_ld(K);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + K;
  V* b = a + nslot * ld;
  load_twiddles<T>(tw_s, tw64, tw32, fp);
  // slot = (j*2 + ab)*ncm + c; line l = z*K1 + y starts at l*K (layout L2)
  const FastDiv fncm = make_fastdiv(ncm), fK1 = make_fastdiv(K1);
  for (int idx = threadIdx.x; idx < nslot * K; idx += blockDim.x) {
    int slot = (int)fdiv((uint32_t)idx, fp.k), e = idx - slot * K;
    int jab = (int)fdiv((uint32_t)slot, fncm), c = slot - jab * ncm;
    int2 pr = xpairs[it.y + (jab >> 1)];
    int l = (jab & 1) ? pr.y : pr.x;
    cp_async_elem(a + slot * ld + fft_pidx(e), mesh + S.mesh_off + (int64_t)c * S.M + (int64_t)l * K + e);
  }
  cp_async_wait_all();
  __syncthreads();
  V* R = fft_lines<T>(a, b, nslot, K, ld, fp, tw_s, (T)-1);
  V* other = (R == a) ? b : a;
  // reciprocal multiply.  Per pair of lines the constant parts (the G(m) share of
  // m1 b1 + m2 b2, and k_e 4 pi/V |b1(m1) b2(m2)|^2) are staged in shared memory;
  // exponent factors are -w_st^2/2 log2(e), so each Gaussian is one exp2.
  const T* bm0 = bmod + S.bmod_off[0];
  const T* bm1 = bmod + S.bmod_off[1];
  const T* bm2 = bmod + S.bmod_off[2];
  const T B0 = (T)S.B[0], B1 = (T)S.B[1], B2 = (T)S.B[2];
  const T gpref = (T)S.green_pref;
  __shared__ T hw2[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];
  __shared__ T lineg[QEQ_XPAIRS_MAX][4];
  for (int i = threadIdx.x; i < QEQ_MAX_SPECIES * QEQ_MAX_SPECIES; i += blockDim.x)
    hw2[i] = (T)(-0.5 * 1.44269504088896340736 * S.w2[i]);
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    const int2 pr = xpairs[it.y + j];
    const int mz = (int)fdiv((uint32_t)pr.x, fK1), my = pr.x - mz * K1;
    const int c1 = (my <= K1 / 2) ? my : my - K1;
    const int c2 = (mz <= K2 / 2) ? mz : mz - K2;
    lineg[j][0] = (T)(c1 * S.B[3] + c2 * S.B[6]);
    lineg[j][1] = (T)(c1 * S.B[4] + c2 * S.B[7]);
    lineg[j][2] = (T)(c1 * S.B[5] + c2 * S.B[8]);
    lineg[j][3] = gpref * bm1[my] * bm2[mz];
  }
  // beta: 1 (the plain Woodbury factor) while the smoothest mode's x = s0 g0 stays small,
  // else the plan's safety factor (S.omega holds it for the preconditioner mesh); large
  // cells need it because the correction nearly cancels D^-1 for their smooth modes and
  // the circulant mean's error would then make M indefinite
  const T pre_beta = PRE ? ((sc[it.x].s0 * S.pre_g0max <= kPreBetaOneX) ? (T)1 : (T)S.omega) : (T)0;
  const T pre_s0 = PRE ? (T)sc[it.x].s0 : (T)0;
  const int nspec = S.S;
  __syncthreads();
  for (int idx = threadIdx.x; idx < np * K; idx += blockDim.x) {
    const int j = (int)fdiv((uint32_t)idx, fp.k), mx = idx - j * K;
    const int mmx = (mx == 0) ? 0 : K - mx;
    const int c0 = (mx <= K / 2) ? mx : mx - K;
    const T Gx = (T)c0 * B0 + lineg[j][0];
    const T Gy = (T)c0 * B1 + lineg[j][1];
    const T Gz = (T)c0 * B2 + lineg[j][2];
    const T G2 = Gx * Gx + Gy * Gy + Gz * Gz;
    const T rG2 = (G2 > (T)0) ? recip<T>(G2) : (T)0;
    const T pref = lineg[j][3] * bm0[mx] * rG2;  // G = 0 term dropped
    V Qh[MAXS];
#pragma unroll
    for (int c = 0; c < MAXS / 2; ++c) {
      if (c >= ncm) break;
      V za = R[((j * 2 + 0) * ncm + c) * ld + fft_pidx(mx)];
      V zb = R[((j * 2 + 1) * ncm + c) * ld + fft_pidx(mmx)];
      // F[Q_2c] = (Z(m) + conj Z(-m))/2,  F[Q_2c+1] = (Z(m) - conj Z(-m))/(2i)
      Qh[2 * c] = {(T)0.5 * (za.x + zb.x), (T)0.5 * (za.y - zb.y)};
      Qh[2 * c + 1] = {(T)0.5 * (za.y + zb.y), (T)-0.5 * (za.x - zb.x)};
    }
#pragma unroll
    for (int c = 0; c < MAXS / 2; ++c) {
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
      R[((j * 2 + 0) * ncm + c) * ld + fft_pidx(mx)] = {p0.x - p1.y, p0.y + p1.x};
      R[((j * 2 + 1) * ncm + c) * ld + fft_pidx(mmx)] = {p0.x + p1.y, -p0.y + p1.x};
    }
  }
  __syncthreads();
  V* res = fft_lines<T>(R, other, nslot, K, ld, fp, tw_s, (T)1);
  for (int idx = threadIdx.x; idx < nslot * K; idx += blockDim.x) {
    int slot = (int)fdiv((uint32_t)idx, fp.k), e = idx - slot * K;
    int jab = (int)fdiv((uint32_t)slot, fncm), c = slot - jab * ncm;
    int2 pr = xpairs[it.y + (jab >> 1)];
    if ((jab & 1) && pr.y == pr.x) continue;  // self-paired line: written from its A copy
    int l = (jab & 1) ? pr.y : pr.x;
    mesh[S.mesh_off + (int64_t)c * S.M + (int64_t)l * K + e] = res[slot * ld + fft_pidx(e)];
  }
}

// ------------------------------------------------------------------ brick geometry
struct Brick {
  int x0[3], ext[3];
};

__device__ __forceinline__ Brick brick_of(const StructDev& S, int g) {
  Brick B;
  int gl = g - S.brick_off;
  int bc2 = gl % S.nbr[2];
  int bc1 = (gl / S.nbr[2]) % S.nbr[1];
  int bc0 = gl / (S.nbr[2] * S.nbr[1]);
  int bc[3] = {bc0, bc1, bc2};
  for (int d = 0; d < 3; ++d) {
    B.x0[d] = bc[d] * QEQ_BRICK;
    B.ext[d] = min(QEQ_BRICK, S.K[d] - B.x0[d]);
  }
  return B;
}

// the matvec input in the mesh precision: the FP32 copy in mixed precision
template <typename T>
__device__ __forceinline__ T xval(const double* __restrict__ x, const float* __restrict__ x32, int64_t i);
template <>
__device__ __forceinline__ float xval<float>(const double*, const float* __restrict__ x32, int64_t i) {
  return x32[i];
}
template <>
__device__ __forceinline__ double xval<double>(const double* __restrict__ x, const float*, int64_t i) {
  return x[i];
}

// ------------------------------------------------------------------ spreading
// One CTA per 16^3 brick and complex mesh, no atomics: thread (lx, ly) owns the
// brick's z-row at (x0 + lx, y0 + ly) and keeps its 16 points (both species
// parts) in registers.  The candidate atoms (those of the bins whose stencils
// can reach the brick) are staged in batches of QEQ_SPB as compact records in
// shared memory: stencil offsets relative to the brick, 16-bit masks of the
// brick rows the stencil covers in x and y, the x / y weights (x pre-multiplied
// by the charge) and the z weights at the brick's 16 z positions.  Every thread
// then adds, atom after atom in a fixed order, its row's contribution: the
// spread is deterministic and each mesh point is written to global memory once.
#define QEQ_SPB 256  // candidate records per batch (one per thread)

// Bits l in [0, ext) of brick rows covered by a stencil of P rows that starts
// o rows into the brick (o in [0, K), periodic with period K >= P).
template <int P>
__device__ __forceinline__ unsigned stencil_rows(int o, int K, int ext) {
  const unsigned win = (1u << P) - 1u;
  unsigned m = 0;
  if (o < 16) m |= win << o;                     // the stencil itself
  if (K - o < P) m |= win >> (K - o);            // its image one period down
  if (o + K < 16) m |= win << (o + K);           // ... and one period up (K < 16)
  if (2 * K - o < P) m |= win >> (2 * K - o);    // two periods down (K < P + 16)
  return m & ((1u << ext) - 1u);
}

template <typename T, int P>
struct SpreadRecs {
  T wz[QEQ_SPB][QEQ_BRICK];  // z weights at the brick's z positions (0 outside the stencil)
  T wx[QEQ_SPB][P];          // q * x weights, by stencil index
  T wy[QEQ_SPB][P];
  unsigned mask[QEQ_SPB];    // x rows (bits 0-15) and y rows (bits 16-31) the stencil covers
  int off[QEQ_SPB];          // ox | oy << 10 | species part << 20
};

template <typename T, int P>
__global__ void __launch_bounds__(256) k_spread(const StructDev* __restrict__ st, const int* __restrict__ brick_struct,
                         const int* __restrict__ bin_start, const int* __restrict__ base,
                         const T* __restrict__ wts, const int* __restrict__ spec, const double* __restrict__ x,
                         const float* __restrict__ x32, const PcgScalars* __restrict__ sc, int use_active,
                         typename C2<T>::t* __restrict__ mesh) {
  using V = typename C2<T>::t;
  const int g = blockIdx.x;
  const int s = brick_struct[g];
  const StructDev& S = st[s];
  if (use_active && !sc[s].active) return;
  const int tid = threadIdx.x, lx = tid >> 4, ly = tid & 15;
  const Brick B = brick_of(S, g);
  const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
  __shared__ int cand[3][8], ncand[3];
  __shared__ int bin_beg[512], bin_pre[513];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SpreadRecs<T, P>& R = *reinterpret_cast<SpreadRecs<T, P>*>(smem_raw);
  if (tid < 3) {
    int d = tid, nc = 0;
    int span = min(B.ext[d] + P - 1, S.K[d]);
    for (int k = 0; k < span; ++k) {
      int bn = ((B.x0[d] + k) % S.K[d]) / QEQ_BIN;
      bool seen = false;
      for (int q = 0; q < nc; ++q) seen |= (cand[d][q] == bn);
      if (!seen && nc < 8) cand[d][nc++] = bn;
    }
    ncand[d] = nc;
  }
  __syncthreads();
  // candidate bins (at most 8 x 8 x 8) in (i0, i1, i2) order and the prefix of their sizes
  const int nc1 = ncand[1], nc2 = ncand[2], nbins = ncand[0] * nc1 * nc2;
  for (int k = tid; k < nbins; k += blockDim.x) {
    const int i2 = k % nc2, i1 = (k / nc2) % nc1, i0 = k / (nc2 * nc1);
    const int gb = S.bin_off + (cand[0][i0] * S.nb[1] + cand[1][i1]) * S.nb[2] + cand[2][i2];
    bin_beg[k] = bin_start[gb];
    bin_pre[k + 1] = bin_start[gb + 1] - bin_start[gb];
  }
  __syncthreads();
  if (tid < 32) {  // inclusive scan of the sizes in chunks of 32
    int carry = 0;
    for (int k0 = 0; k0 < nbins; k0 += 32) {
      int v = (k0 + tid < nbins) ? bin_pre[k0 + tid + 1] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (tid >= o) v += u;
      }
      if (k0 + tid < nbins) bin_pre[k0 + tid + 1] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (tid == 0) bin_pre[0] = 0;
  }
  __syncthreads();
  const int total = bin_pre[nbins];
  for (int cm = 0; cm < S.ncm; ++cm) {
    T re[QEQ_BRICK], im[QEQ_BRICK];
#pragma unroll
    for (int z = 0; z < QEQ_BRICK; ++z) re[z] = im[z] = (T)0;
    for (int c0 = 0; c0 < total; c0 += QEQ_SPB) {
      const int nbat = min(QEQ_SPB, total - c0);
      if (c0 > 0) __syncthreads();  // the previous batch is consumed
      if (tid < nbat) {
        const int c = c0 + tid;
        int lo = 0, hi = nbins - 1;  // last bin whose first candidate is <= c
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (bin_pre[mid] <= c) lo = mid;
          else hi = mid - 1;
        }
        const int t = bin_beg[lo] + (c - bin_pre[lo]);
        const int sp = spec[t];
        unsigned mask = 0;
        if ((sp >> 1) == cm) {
          const int bs = base[t];
          const int f[3] = {bs & 1023, (bs >> 10) & 1023, (bs >> 20) & 1023};
          int o[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {  // stencil start relative to the brick, in [0, K)
            int v = f[d] - (P - 1) - B.x0[d];
            if (v < 0) v += S.K[d];
            if (v < 0) v += S.K[d];
            o[d] = v;
          }
          const T* wt = wts + (size_t)t * 3 * QEQ_MAXP;
          const unsigned xm = stencil_rows<P>(o[0], K0, B.ext[0]);
          const unsigned ym = stencil_rows<P>(o[1], K1, B.ext[1]);
          const unsigned zm = stencil_rows<P>(o[2], K2, B.ext[2]);
#pragma unroll
          for (int l = 0; l < QEQ_BRICK; ++l) {
            int j = l - o[2];
            if (j < 0) j += K2;
            if (j >= K2) j -= K2;
            R.wz[tid][l] = ((zm >> l) & 1u) ? wt[2 * QEQ_MAXP + P - 1 - j] : (T)0;
          }
          const T q = xval<T>(x, x32, t);
#pragma unroll
          for (int j = 0; j < P; ++j) {
            R.wx[tid][j] = q * wt[P - 1 - j];
            R.wy[tid][j] = wt[QEQ_MAXP + P - 1 - j];
          }
          if (zm) mask = xm | (ym << 16);
          R.off[tid] = o[0] | (o[1] << 10) | ((sp & 1) << 20);
        }
        R.mask[tid] = mask;
      }
      __syncthreads();
      // every thread adds its row's share, atom after atom.  A warp owns the rows
      // lx = 2w, 2w+1: it ballots the records whose stencil covers one of them
      // (32 records per ballot) and visits only those, in record order.
      const unsigned wsel = 3u << (2 * (tid >> 5));
      const int lane = tid & 31;
      for (int i0 = 0; i0 < nbat; i0 += 32) {
        const int ii = i0 + lane;
        unsigned bal = __ballot_sync(0xffffffffu, ii < nbat && (R.mask[ii] & wsel) != 0u);
        while (bal) {
          const int k = i0 + __ffs(bal) - 1;
          bal &= bal - 1u;
          const unsigned m = R.mask[k];
          if (!((m >> lx) & 1u) || !((m >> (16 + ly)) & 1u)) continue;
          const int off = R.off[k];
          int jx = lx - (off & 1023);
          if (jx < 0) jx += K0;
          int jy = ly - ((off >> 10) & 1023);
          if (jy < 0) jy += K1;
          const T r = R.wx[k][jx] * R.wy[k][jy];
          const T* wz = R.wz[k];
          if ((off >> 20) & 1) {
#pragma unroll
            for (int z = 0; z < QEQ_BRICK; ++z) im[z] += r * wz[z];
          } else {
#pragma unroll
            for (int z = 0; z < QEQ_BRICK; ++z) re[z] += r * wz[z];
          }
        }
      }
      __syncthreads();
    }
    if (lx < B.ext[0] && ly < B.ext[1]) {
      V* mg = mesh + S.mesh_off + (int64_t)cm * S.M +
              ((int64_t)(B.x0[0] + lx) * K1 + (B.x0[1] + ly)) * K2 + B.x0[2];
#pragma unroll
      for (int z = 0; z < QEQ_BRICK; ++z)
        if (z < B.ext[2]) mg[z] = V{re[z], im[z]};
    }
  }
}

// ------------------------------------------------------------------ gathering + local + real space
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ const T* pair_vals(const double* v64, const float* v32);
template <>
__device__ __forceinline__ const float* pair_vals<float>(const double*, const float* v32) {
  return v32;
}
template <>
__device__ __forceinline__ const double* pair_vals<double>(const double* v64, const float*) {
  return v64;
}

// Gathering without shared-memory staging: a warp takes one atom (atoms in sorted
// order, so neighbouring warps touch the same mesh rows through L1), lanes own 4
// stencil rows x 8 z points and read the potential straight from the mesh; the
// same warp adds the real-space pair row and the local terms.  CTAs are atom
// chunks of one structure, so x.y is reduced per structure deterministically.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_gather_direct(
    const Chunk* __restrict__ chunks, const StructDev* __restrict__ st, const int* __restrict__ base,
    const T* __restrict__ wts, const int* __restrict__ spec, const double* __restrict__ J,
    const double* __restrict__ x, const float* __restrict__ x32, const int64_t* __restrict__ row,
    const int* __restrict__ col,
    const double* __restrict__ v64, const float* __restrict__ v32, int with_J, int with_pairs,
    PcgScalars* __restrict__ sc, int use_active, int fuse_pAp, double* __restrict__ part, int* __restrict__ counter,
    const typename C2<T>::t* __restrict__ mesh, double* __restrict__ y, int split) {
  using V = typename C2<T>::t;
  const Chunk ch = chunks[blockIdx.x / split];
  const int sub = blockIdx.x - (blockIdx.x / split) * split;
  if (use_active && !sc[ch.s].active) return;
  const StructDev& S = st[ch.s];
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jz = lane & 7, rsub = lane >> 3;
  const T* vals = pair_vals<T>(v64, v32);
  double blk = 0.0;
  // this CTA's share of the chunk: a contiguous run of atoms, so that the CTAs in
  // flight (launched in order) read a compact part of the mesh and the stencil
  // halos shared by neighbouring runs are still in L2
  const int64_t len = (ch.end - ch.begin + split - 1) / split;
  const int64_t lo = ch.begin + (int64_t)sub * len, hi = min(ch.end, lo + len);
  // a warp takes G <= 8 consecutive atoms: their stencils one after another (all
  // lanes), each atom's sum parked in lane g, then the FP64 local terms for the G
  // atoms on lanes 0..G-1 at once (FP64 issue slots are scarce)
  const int G = (int)max((int64_t)1, min((int64_t)8, (len + nw - 1) / nw));
  for (int64_t tb = lo + (int64_t)G * w; tb < hi; tb += (int64_t)G * nw) {
    T mine = (T)0;
    for (int g = 0; g < G; ++g) {
      const int64_t t = tb + g;
      if (t >= hi) break;
      const int sp = spec[t];
      const int part_ = sp & 1;
      const V* mg = mesh + S.mesh_off + (int64_t)(sp >> 1) * S.M;
      const int bs = base[t];
      const int f0 = bs & 1023, f1 = (bs >> 10) & 1023, f2 = (bs >> 20) & 1023;
      const T* wt = wts + (size_t)t * 3 * QEQ_MAXP;
      T acc = (T)0;
      if (jz < P) {
        int kz = f2 - (P - 1) + jz;
        if (kz < 0) kz += S.K[2];
        const T wzj = wt[2 * QEQ_MAXP + P - 1 - jz];
        T racc = (T)0;
#pragma unroll
        for (int r = rsub; r < P * P; r += 4) {
          const int jx = r / P, jy = r - (r / P) * P;
          int kx = f0 - (P - 1) + jx;
          if (kx < 0) kx += S.K[0];
          int ky = f1 - (P - 1) + jy;
          if (ky < 0) ky += S.K[1];
          const V v = __ldg(mg + ((int64_t)kx * S.K[1] + ky) * S.K[2] + kz);
          racc += wt[P - 1 - jx] * wt[QEQ_MAXP + P - 1 - jy] * (part_ ? v.y : v.x);
        }
        acc = racc * wzj;
      }
      if (with_pairs) {
        int64_t r0 = row[t], r1 = row[t + 1];
        for (int64_t k = r0 + lane; k < r1; k += 32) acc += vals[k] * xval<T>(x, x32, col[k]);
      }
      acc = warp_sum<T>(acc);
      if (lane == g) mine = acc;
    }
    const int64_t t = tb + lane;
    if (lane < G && t < hi) {
      const int sp = spec[t];
      const double xi = x[t];
      double loc = S.self_s[sp] * xi;
      if (with_J) loc += J[t] * xi;
      const PcgScalars& c = sc[ch.s];
      for (int tt = 0; tt < S.S; ++tt) loc -= S.corr[sp * QEQ_MAX_SPECIES + tt] * c.xsum[tt];
      const double yi = (double)mine + loc;
      y[t] = yi;
      blk += xi * yi;
    }
  }
  if (fuse_pAp) {
    __shared__ double wsum[32];
    __shared__ double red[256];
    __shared__ bool last;
    blk = warp_sum<double>(blk);  // lanes 0..G-1 hold the warp's atoms (fixed order)
    if (lane == 0) wsum[w] = blk;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int i = 0; i < nw; ++i) b += wsum[i];
      part[blockIdx.x] = b;
      __threadfence();
      last = (atomicAdd(&counter[ch.s], 1) == ch.count * split - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double tot = ordered_block_sum(part, ch.first * split, ch.count * split, 1, 0, red);
      if (threadIdx.x == 0) {
        PcgScalars& c = sc[ch.s];
        c.pAp = tot;
        c.alpha = (tot != 0.0) ? c.rz / tot : 0.0;
        counter[ch.s] = 0;
      }
    }
  }
}

// ------------------------------------------------------------------ per-species sums of x
__global__ void k_species_sums(const Chunk* __restrict__ chunks, const StructDev* __restrict__ st,
                               const int* __restrict__ spec, const double* __restrict__ x,
                               PcgScalars* __restrict__ sc, int use_active, double* __restrict__ part,
                               int* __restrict__ counter, float* __restrict__ x32) {
  const Chunk ch = chunks[blockIdx.x];
  if (use_active && !sc[ch.s].active) return;
  __shared__ double red[QEQ_MAX_SPECIES][33];
  double loc[QEQ_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < QEQ_MAX_SPECIES; ++k) loc[k] = 0.0;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const int sp = spec[a];
    const double xa = x[a];
    if (x32) x32[a] = (float)xa;
#pragma unroll
    for (int k = 0; k < QEQ_MAX_SPECIES; ++k) loc[k] += (sp == k) ? xa : 0.0;
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < QEQ_MAX_SPECIES; ++k) {
    double v = warp_sum<double>(loc[k]);
    if (lane == 0) red[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < QEQ_MAX_SPECIES) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[threadIdx.x][i];
    part[(size_t)blockIdx.x * QEQ_MAX_SPECIES + threadIdx.x] = v;
    __threadfence();  // each writer publishes its partial before the block is counted
  }
  __shared__ bool last;
  __shared__ double red2[256];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int prev = atomicAdd(&counter[ch.s], 1);
    last = (prev == ch.count - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int k = 0; k < QEQ_MAX_SPECIES; ++k) {
      double tot = ordered_block_sum(part, ch.first, ch.count, QEQ_MAX_SPECIES, k, red2);
      if (threadIdx.x == 0) sc[ch.s].xsum[k] = tot;
    }
    if (threadIdx.x == 0) counter[ch.s] = 0;
  }
}

// ------------------------------------------------------------------ Fourier preconditioner
// Power-of-two scale of the fixed-point coarse spread: max |D^-1 r| is at most
// max|r| max D^-1 (max D^-1 alone for the ones vector), mapped to 2^48; a mesh
// point sums the B-spline weights (each at most 2/3 per direction) of the atoms
// around it, far below the 2^15 headroom of a signed 64-bit integer.
__device__ __forceinline__ double pre_fixed_scale(const PcgScalars& c, int ones_input) {
  double b = c.dinv_max * (ones_input ? 1.0 : fmax(fabs(c.r_max), fabs(c.r_min)));
  if (!(b > 0.0) || !isfinite(b)) b = 1.0;
  int e;
  frexp(b, &e);                    // b < 2^e
  return ldexp(1.0, 48 - e);
}

// Cubic B-spline (order 4) weights of every atom on its structure's coarse mesh,
// once per solve: M_4(w + j), j = 0..3, for stencil points f - j.
__global__ void k_pre_weights(const StructDev* __restrict__ stp, const int* __restrict__ sorted_struct,
                              const double* __restrict__ posc, int64_t n, int* __restrict__ pbase,
                              float* __restrict__ pw) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const StructDev& S = stp[sorted_struct[a]];
  int f[3];
  for (int d = 0; d < 3; ++d) {
    double u = posc[3 * a] * S.hinv[d] + posc[3 * a + 1] * S.hinv[3 + d] + posc[3 * a + 2] * S.hinv[6 + d];
    u -= floor(u);
    double x = u * S.K[d];
    int fi = (int)floor(x);
    if (fi >= S.K[d]) fi = S.K[d] - 1;
    if (fi < 0) fi = 0;
    double w = x - fi;
    f[d] = fi;
    double w2 = w * w, w3 = w2 * w;
    pw[a * 12 + d * 4 + 0] = (float)(w3 / 6.0);
    pw[a * 12 + d * 4 + 1] = (float)((-3.0 * w3 + 3.0 * w2 + 3.0 * w + 1.0) / 6.0);
    pw[a * 12 + d * 4 + 2] = (float)((3.0 * w3 - 6.0 * w2 + 4.0) / 6.0);
    pw[a * 12 + d * 4 + 3] = (float)((1.0 - w) * (1.0 - w) * (1.0 - w) / 6.0);
  }
  pbase[a] = f[0] | (f[1] << 10) | (f[2] << 20);
}

// v = D^-1 r spread on the coarse mesh in 64-bit fixed point: every contribution
// is rounded to an integer multiple of 2^-e (e per structure, from a bound on
// max |v|) and added with an integer atomic.  Integer addition does not depend
// on the order of the atomics, so the coarse mesh, and with it every
// preconditioned solve, is bitwise reproducible.  k_pre_fixed_to_float turns the
// sums back into the FP32 mesh.
__global__ void k_pre_spread(const StructDev* __restrict__ stp, const int* __restrict__ sorted_struct,
                             const int* __restrict__ pbase, const float* __restrict__ pw,
                             const double* __restrict__ dinv, const double* __restrict__ r, int64_t n,
                             const PcgScalars* __restrict__ sc, int use_active, int ones_input,
                             unsigned long long* __restrict__ imesh) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int s = sorted_struct[a];
  if (use_active && !sc[s].active) return;
  const StructDev& S = stp[s];
  const int bs = pbase[a];
  const int f[3] = {bs & 1023, (bs >> 10) & 1023, (bs >> 20) & 1023};
  const float* w = pw + a * 12;
  const float v = (float)(dinv[a] * r[a]);
  const double scale = pre_fixed_scale(sc[s], ones_input);
  unsigned long long* m = imesh + S.mesh_off;
  for (int jx = 0; jx < 4; ++jx) {
    int kx = f[0] - jx;
    if (kx < 0) kx += S.K[0];
    for (int jy = 0; jy < 4; ++jy) {
      int ky = f[1] - jy;
      if (ky < 0) ky += S.K[1];
      const float wxy = v * w[jx] * w[4 + jy];
      unsigned long long* row = m + ((int64_t)kx * S.K[1] + ky) * S.K[2];
      for (int jz = 0; jz < 4; ++jz) {
        int kz = f[2] - jz;
        if (kz < 0) kz += S.K[2];
        const long long c = __double2ll_rn((double)(wxy * w[8 + jz]) * scale);
        atomicAdd(&row[kz], (unsigned long long)c);
      }
    }
  }
}

// fixed-point coarse mesh -> FP32 complex mesh (real part), structure found by bisection
__global__ void k_pre_fixed_to_float(const StructDev* __restrict__ stp, int ns, int64_t total,
                                     const PcgScalars* __restrict__ sc, int ones_input,
                                     const unsigned long long* __restrict__ imesh, float2* __restrict__ mesh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (stp[mid].mesh_off <= i) lo = mid;
      else hi = mid - 1;
    }
    const double inv = 1.0 / pre_fixed_scale(sc[lo], ones_input);
    mesh[i] = make_float2((float)((double)(long long)imesh[i] * inv), 0.f);
  }
}

// u = D^-1 (r - phi), phi the interpolated coarse potential; per-structure sum of u
__global__ void k_pre_gather(const Chunk* __restrict__ chunks, const StructDev* __restrict__ stp,
                             const int* __restrict__ pbase, const float* __restrict__ pw,
                             const double* __restrict__ dinv, const double* __restrict__ r,
                             const float2* __restrict__ mesh, PcgScalars* __restrict__ sc, int use_active,
                             int slot, double* __restrict__ u, double* __restrict__ part, int* __restrict__ counter) {
  const Chunk ch = chunks[blockIdx.x];
  if (use_active && !sc[ch.s].active) return;
  const StructDev& S = stp[ch.s];
  const float2* m = mesh + S.mesh_off;
  double acc = 0.0;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const int bs = pbase[a];
    const int f[3] = {bs & 1023, (bs >> 10) & 1023, (bs >> 20) & 1023};
    const float* w = pw + a * 12;
    float phi = 0.f;
    for (int jx = 0; jx < 4; ++jx) {
      int kx = f[0] - jx;
      if (kx < 0) kx += S.K[0];
      for (int jy = 0; jy < 4; ++jy) {
        int ky = f[1] - jy;
        if (ky < 0) ky += S.K[1];
        const float2* row = m + ((int64_t)kx * S.K[1] + ky) * S.K[2];
        float rs = 0.f;
        for (int jz = 0; jz < 4; ++jz) {
          int kz = f[2] - jz;
          if (kz < 0) kz += S.K[2];
          rs += w[8 + jz] * row[kz].x;
        }
        phi += w[jx] * w[4 + jy] * rs;
      }
    }
    double ua = dinv[a] * (r[a] - (double)phi);
    u[a] = ua;
    acc += ua;
  }
  __shared__ double red[256];
  __shared__ bool last;
  acc = warp_sum<double>(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += red[i];
    part[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(&counter[ch.s], 1) == ch.count - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double tot = ordered_block_sum(part, ch.first, ch.count, 1, 0, red);
    if (threadIdx.x == 0) {
      if (slot == 0)
        sc[ch.s].usum = tot;
      else
        sc[ch.s].w1sum = tot;
      counter[ch.s] = 0;
    }
  }
}

// ------------------------------------------------------------------ host side
template <typename T, int P>
cudaError_t matvec_impl(qeq_plan_s* Pl, const double* x, double* y, int with_J, int use_active, int fuse_pAp,
                        cudaEvent_t* ev) {
  using V = typename C2<T>::t;
  constexpr bool F32 = std::is_same<T, float>::value;
  cudaStream_t s = Pl->stream;
  V* mesh = reinterpret_cast<V*>(Pl->d_mesh);
  const T* wts = F32 ? (const T*)(const void*)Pl->d_wts32 : (const T*)(const void*)Pl->d_wts;
  const T* bmod = F32 ? (const T*)(const void*)Pl->d_bmod32 : (const T*)(const void*)Pl->d_bmod;
  const size_t csz = sizeof(V);
  int rec = 0;
  auto mark = [&]() -> cudaError_t { return ev ? cudaEventRecord(ev[rec++], s) : cudaSuccess; };
  count_launch(Pl, 8);
  QEQ_CUDA_TRY(mark());
  // stage 0: per-species sums of x (width-correction terms)
  float* x32 = std::is_same<T, float>::value ? Pl->d_x32 : nullptr;
  k_species_sums<<<Pl->n_chunks, 256, 0, s>>>(Pl->d_chunks, Pl->d_st, Pl->d_spec, x, Pl->d_sc, use_active,
                                               Pl->d_part, Pl->d_counter, x32);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  // stage 1: spreading
  {
    k_spread<T, P><<<Pl->total_bricks, 256, sizeof(SpreadRecs<T, P>), s>>>(Pl->d_st, Pl->d_brick_struct, Pl->d_bin_start, Pl->d_base, wts,
                                                      Pl->d_spec, x, x32, Pl->d_sc, use_active, mesh);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  QEQ_CUDA_TRY(mark());
  const size_t smf = csz * (size_t)Pl->fft_smem_elems;
  V* mesh2 = reinterpret_cast<V*>(Pl->d_mesh2);
  // stages 2-6: FFT z (L0 -> L1), FFT y (L1 -> L2), x + reciprocal multiply + inverse x (L2),
  //             inverse y (L2 -> L1), inverse z (L1 -> L0)
  k_fft_pass<T, PASS_ZF><<<Pl->n_zitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_zitems, Pl->d_tw64, Pl->d_tw32,
                                                        Pl->d_sc, use_active, mesh, mesh2, Pl->tl);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_pass<T, PASS_YF><<<Pl->n_yitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_yitems, Pl->d_tw64, Pl->d_tw32,
                                                        Pl->d_sc, use_active, mesh2, mesh, Pl->tl);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  if (Pl->max_species <= 2)
    k_fft_x_green<T, false, 2><<<Pl->n_xitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_xitems, Pl->d_xpairs, bmod,
                                                   Pl->d_tw64, Pl->d_tw32, Pl->d_sc, use_active, mesh);
  else
    k_fft_x_green<T, false, QEQ_MAX_SPECIES><<<Pl->n_xitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_xitems, Pl->d_xpairs, bmod,
                                                   Pl->d_tw64, Pl->d_tw32, Pl->d_sc, use_active, mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_pass<T, PASS_YI><<<Pl->n_yitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_yitems, Pl->d_tw64, Pl->d_tw32,
                                                        Pl->d_sc, use_active, mesh, mesh2, Pl->tl);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_pass<T, PASS_ZI><<<Pl->n_zitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_zitems, Pl->d_tw64, Pl->d_tw32,
                                                        Pl->d_sc, use_active, mesh2, mesh, Pl->tl);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  // stage 7: gathering + real-space pairs + local terms (+ x.y per structure)
  {
    int with_pairs = Pl->pair_cap > 0;
    k_gather_direct<T, P><<<Pl->n_chunks * Pl->gather_split, 256, 0, s>>>(
        Pl->d_chunks, Pl->d_st, Pl->d_base, wts, Pl->d_spec, Pl->d_J, x, x32, Pl->d_row, Pl->d_col, Pl->d_val64,
        Pl->d_val32, with_J, with_pairs, Pl->d_sc, use_active, fuse_pAp,
        Pl->d_part + (size_t)Pl->n_chunks * QEQ_MAX_SPECIES, Pl->d_counter + Pl->n_struct, mesh, y, Pl->gather_split);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  QEQ_CUDA_TRY(mark());
  return cudaSuccess;
}

template <typename T, int P>
cudaError_t set_smem_attrs() {
  const int big = 200 * 1024;
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_spread<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(SpreadRecs<T, P>)));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T, PASS_ZF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T, PASS_YF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T, PASS_YI>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T, PASS_ZI>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<T, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<T, false, QEQ_MAX_SPECIES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<T, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return cudaSuccess;
}

}  // namespace

cudaError_t matvec_set_attributes() {
  QEQ_CUDA_TRY((set_smem_attrs<float, 4>()));
  QEQ_CUDA_TRY((set_smem_attrs<float, 6>()));
  QEQ_CUDA_TRY((set_smem_attrs<float, 8>()));
  QEQ_CUDA_TRY((set_smem_attrs<double, 4>()));
  QEQ_CUDA_TRY((set_smem_attrs<double, 6>()));
  QEQ_CUDA_TRY((set_smem_attrs<double, 8>()));
  return cudaSuccess;
}

cudaError_t launch_matvec(qeq_plan_s* P, int prec, const double* x, double* y, int with_J, int use_active,
                          int fuse_pAp, cudaEvent_t* ev) {
  int p = P->max_p;
  if (prec == QEQ_MIXED) {
    if (p == 4) return matvec_impl<float, 4>(P, x, y, with_J, use_active, fuse_pAp, ev);
    if (p == 6) return matvec_impl<float, 6>(P, x, y, with_J, use_active, fuse_pAp, ev);
    return matvec_impl<float, 8>(P, x, y, with_J, use_active, fuse_pAp, ev);
  }
  if (p == 4) return matvec_impl<double, 4>(P, x, y, with_J, use_active, fuse_pAp, ev);
  if (p == 6) return matvec_impl<double, 6>(P, x, y, with_J, use_active, fuse_pAp, ev);
  return matvec_impl<double, 8>(P, x, y, with_J, use_active, fuse_pAp, ev);
}

cudaError_t launch_precond_setup(qeq_plan_s* P) {
  count_launch(P);
  k_pre_weights<<<(int)((P->n_atoms + 255) / 256), 256, 0, P->stream>>>(P->d_stp, P->d_key, P->d_posc, P->n_atoms,
                                                                        P->d_pbase, P->d_pw);
  return cudaGetLastError();
}

cudaError_t launch_precond(qeq_plan_s* P, const double* r, double* u, int slot, int use_active) {
  cudaStream_t s = P->stream;
  const size_t smf = sizeof(float2) * (size_t)P->fft_smem_elems;
  const float* bmod = P->d_bmod32;
  count_launch(P, 8);
  // fixed-point sums in the second coarse buffer (8 bytes per point, like the float2 mesh)
  unsigned long long* imesh = reinterpret_cast<unsigned long long*>(P->d_pmesh2);
  QEQ_CUDA_TRY(cudaMemsetAsync(imesh, 0, sizeof(unsigned long long) * (size_t)P->total_pmesh, s));
  k_pre_spread<<<(int)((P->n_atoms + 255) / 256), 256, 0, s>>>(P->d_stp, P->d_key, P->d_pbase, P->d_pw, P->d_dinv, r,
                                                               P->n_atoms, P->d_sc, use_active, slot == 1, imesh);
  {
    const int nb = (int)std::min<int64_t>((P->total_pmesh + 255) / 256, 148 * 16);
    k_pre_fixed_to_float<<<nb, 256, 0, s>>>(P->d_stp, P->n_struct, P->total_pmesh, P->d_sc, slot == 1, imesh,
                                            P->d_pmesh);
  }
  k_fft_pass<float, PASS_ZF><<<P->n_pz, 256, smf, s>>>(P->d_stp, P->d_fft, P->d_pzitems, P->d_tw64, P->d_tw32, P->d_sc,
                                                       use_active, P->d_pmesh, P->d_pmesh2, P->tlp);
  k_fft_pass<float, PASS_YF><<<P->n_py, 256, smf, s>>>(P->d_stp, P->d_fft, P->d_pyitems, P->d_tw64, P->d_tw32, P->d_sc,
                                                       use_active, P->d_pmesh2, P->d_pmesh, P->tlp);
  k_fft_x_green<float, true, 2><<<P->n_px, 256, smf, s>>>(P->d_stp, P->d_fft, P->d_pxitems, P->d_xpairs, bmod, P->d_tw64,
                                                       P->d_tw32, P->d_sc, use_active, P->d_pmesh);
  k_fft_pass<float, PASS_YI><<<P->n_py, 256, smf, s>>>(P->d_stp, P->d_fft, P->d_pyitems, P->d_tw64, P->d_tw32, P->d_sc,
                                                       use_active, P->d_pmesh, P->d_pmesh2, P->tlp);
  k_fft_pass<float, PASS_ZI><<<P->n_pz, 256, smf, s>>>(P->d_stp, P->d_fft, P->d_pzitems, P->d_tw64, P->d_tw32, P->d_sc,
                                                       use_active, P->d_pmesh2, P->d_pmesh, P->tlp);
  k_pre_gather<<<P->n_chunks, 256, 0, s>>>(P->d_chunks, P->d_stp, P->d_pbase, P->d_pw, P->d_dinv, r, P->d_pmesh, P->d_sc,
                                           use_active, slot, u, P->d_part + (size_t)P->n_chunks * QEQ_MAX_SPECIES,
                                           P->d_counter + 3 * P->n_struct);
  return cudaGetLastError();
}
