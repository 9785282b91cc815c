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

// One Stockham radix-R stage over all lines in shared memory.
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const typename C2<T>::t* __restrict__ src,
                                               typename C2<T>::t* __restrict__ dst, int nlines, int K, int Ns,
                                               const typename C2<T>::t* __restrict__ tw, T sgn) {
  using V = typename C2<T>::t;
  int nbf = K / R;
  int tws = K / (Ns * R);
  int total = nlines * nbf;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int line = w / nbf;
    int j = w - line * nbf;
    int k = j % Ns;
    const V* s = src + line * K;
    V* d = dst + line * K;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nbf];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      V t = tw[r * k * tws];
      t.y *= -sgn;  // table holds exp(-2 pi i m/K); sgn = -1 keeps it, +1 conjugates
      v[r] = cmul(v[r], t);
    }
    if (R == 2) dft2<T, V>(v);
    if (R == 3) dft3<T, V>(v, sgn);
    if (R == 4) dft4<T, V>(v, sgn);
    if (R == 5) dft5<T, V>(v, sgn);
    int o = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[o + r * Ns] = v[r];
  }
}

// Unnormalised FFT of nlines lines of length K held in a; returns the buffer with the result.
template <typename T>
__device__ typename C2<T>::t* fft_lines(typename C2<T>::t* a, typename C2<T>::t* b, int nlines, int K,
                                        const FftPlanDev& fp, const typename C2<T>::t* tw, T sgn) {
  int Ns = 1;
  for (int st = 0; st < fp.nst; ++st) {
    int R = fp.radix[st];
    if (R == 4)
      stockham_stage<T, 4>(a, b, nlines, K, Ns, tw, sgn);
    else if (R == 2)
      stockham_stage<T, 2>(a, b, nlines, K, Ns, tw, sgn);
    else if (R == 3)
      stockham_stage<T, 3>(a, b, nlines, K, Ns, tw, sgn);
    else
      stockham_stage<T, 5>(a, b, nlines, K, Ns, tw, sgn);
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
  for (int m = threadIdx.x; m < fp.K; m += blockDim.x) tw_s[m] = g[m];
}

// ------------------------------------------------------------------ FFT along z (contiguous lines)
template <typename T>
__global__ void k_fft_z(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl,
                        const int4* __restrict__ items, const double2* __restrict__ tw64,
                        const float2* __restrict__ tw32, const PcgScalars* __restrict__ sc, int use_active,
                        typename C2<T>::t* __restrict__ mesh, T sgn) {
  using V = typename C2<T>::t;
  int4 it = items[blockIdx.x];
  const StructDev& S = st[it.x];
  if (use_active && !sc[it.x].active) return;
  const FftPlanDev fp = fpl[S.fft_plan[2]];
  int K = S.K[2], nl = it.w;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + K;
  V* b = a + nl * K;
  load_twiddles<T>(tw_s, tw64, tw32, fp);
  V* g = mesh + S.mesh_off + (int64_t)it.y * S.M + (int64_t)it.z * K;
  for (int e = threadIdx.x; e < nl * K; e += blockDim.x) a[e] = g[e];
  __syncthreads();
  V* res = fft_lines<T>(a, b, nl, K, fp, tw_s, sgn);
  for (int e = threadIdx.x; e < nl * K; e += blockDim.x) g[e] = res[e];
}

// ------------------------------------------------------------------ FFT along y (stride K2)
template <typename T>
__global__ void k_fft_y(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl,
                        const int4* __restrict__ items, const double2* __restrict__ tw64,
                        const float2* __restrict__ tw32, const PcgScalars* __restrict__ sc, int use_active,
                        typename C2<T>::t* __restrict__ mesh, T sgn, int lines_per_item) {
  using V = typename C2<T>::t;
  int4 it = items[blockIdx.x];  // {struct, cmesh, x, z0}
  const StructDev& S = st[it.x];
  if (use_active && !sc[it.x].active) return;
  const FftPlanDev fp = fpl[S.fft_plan[1]];
  int K = S.K[1], K2 = S.K[2];
  int nl = min(lines_per_item, K2 - it.w);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + K;
  V* b = a + nl * K;
  load_twiddles<T>(tw_s, tw64, tw32, fp);
  V* g = mesh + S.mesh_off + (int64_t)it.y * S.M + (int64_t)it.z * K * K2 + it.w;
  for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
    int l = idx % nl, e = idx / nl;
    a[l * K + e] = g[(int64_t)e * K2 + l];
  }
  __syncthreads();
  V* res = fft_lines<T>(a, b, nl, K, fp, tw_s, sgn);
  for (int idx = threadIdx.x; idx < nl * K; idx += blockDim.x) {
    int l = idx % nl, e = idx / nl;
    g[(int64_t)e * K2 + l] = res[l * K + e];
  }
}

// ------------------------------------------------------------------ x: FFT, reciprocal multiply, inverse FFT
template <typename T>
__global__ void k_fft_x_green(const StructDev* __restrict__ st, const FftPlanDev* __restrict__ fpl,
                              const int4* __restrict__ items, const int2* __restrict__ xpairs,
                              const T* __restrict__ bmod, const double2* __restrict__ tw64,
                              const float2* __restrict__ tw32, const PcgScalars* __restrict__ sc,
                              int use_active, typename C2<T>::t* __restrict__ mesh) {
  using V = typename C2<T>::t;
  int4 it = items[blockIdx.x];  // {struct, first pair (global), npairs, -}
  const StructDev& S = st[it.x];
  if (use_active && !sc[it.x].active) return;
  const FftPlanDev fp = fpl[S.fft_plan[0]];
  const int K = S.K[0], K1 = S.K[1], K2 = S.K[2];
  const int ncm = S.ncm, np = it.z;
  const int nslot = 2 * np * ncm;
  const int64_t estride = (int64_t)K1 * K2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + K;
  V* b = a + nslot * K;
  load_twiddles<T>(tw_s, tw64, tw32, fp);
  // slot = (j*2 + ab)*ncm + c
  for (int idx = threadIdx.x; idx < nslot * K; idx += blockDim.x) {
    int slot = idx % nslot, e = idx / nslot;
    int c = slot % ncm, jab = slot / ncm;
    int2 pr = xpairs[it.y + (jab >> 1)];
    int l = (jab & 1) ? pr.y : pr.x;
    a[slot * K + e] = mesh[S.mesh_off + (int64_t)c * S.M + l + (int64_t)e * estride];
  }
  __syncthreads();
  V* R = fft_lines<T>(a, b, nslot, K, fp, tw_s, (T)-1);
  V* other = (R == a) ? b : a;
  // reciprocal multiply
  const T* bm0 = bmod + S.bmod_off[0];
  const T* bm1 = bmod + S.bmod_off[1];
  const T* bm2 = bmod + S.bmod_off[2];
  const T B0 = (T)S.B[0], B1 = (T)S.B[1], B2 = (T)S.B[2], B3 = (T)S.B[3], B4 = (T)S.B[4], B5 = (T)S.B[5],
          B6 = (T)S.B[6], B7 = (T)S.B[7], B8 = (T)S.B[8];
  const T gpref = (T)S.green_pref;
  T w2h[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];
  for (int k = 0; k < S.S * QEQ_MAX_SPECIES; ++k) w2h[k] = (T)(0.5 * S.w2[k]);
  for (int idx = threadIdx.x; idx < np * K; idx += blockDim.x) {
    int j = idx / K, mx = idx - j * K;
    int mmx = (mx == 0) ? 0 : K - mx;
    int2 pr = xpairs[it.y + j];
    int my = pr.x / K2, mz = pr.x - my * K2;
    int c0 = (mx <= K / 2) ? mx : mx - K;
    int c1 = (my <= K1 / 2) ? my : my - K1;
    int c2 = (mz <= K2 / 2) ? mz : mz - K2;
    T Gx = (T)c0 * B0 + (T)c1 * B3 + (T)c2 * B6;
    T Gy = (T)c0 * B1 + (T)c1 * B4 + (T)c2 * B7;
    T Gz = (T)c0 * B2 + (T)c1 * B5 + (T)c2 * B8;
    T G2 = Gx * Gx + Gy * Gy + Gz * Gz;
    T pref = (G2 > (T)0) ? gpref * bm0[mx] * bm1[my] * bm2[mz] / G2 : (T)0;
    V Qh[QEQ_MAX_SPECIES];
    for (int c = 0; c < ncm; ++c) {
      V za = R[((j * 2 + 0) * ncm + c) * K + mx];
      V zb = R[((j * 2 + 1) * ncm + c) * K + mmx];
      // F[Q_2c] = (Z(m) + conj Z(-m))/2,  F[Q_2c+1] = (Z(m) - conj Z(-m))/(2i)
      Qh[2 * c] = {(T)0.5 * (za.x + zb.x), (T)0.5 * (za.y - zb.y)};
      Qh[2 * c + 1] = {(T)0.5 * (za.y + zb.y), (T)-0.5 * (za.x - zb.x)};
    }
    V Ph[QEQ_MAX_SPECIES];
    for (int s = 0; s < 2 * ncm; ++s) Ph[s] = {(T)0, (T)0};
    if (pref != (T)0) {
      for (int s = 0; s < S.S; ++s)
        for (int t = 0; t < S.S; ++t) {
          T gst = pref * exp(-G2 * w2h[s * QEQ_MAX_SPECIES + t]);
          Ph[s].x += gst * Qh[t].x;
          Ph[s].y += gst * Qh[t].y;
        }
    }
    for (int c = 0; c < ncm; ++c) {
      V p0 = Ph[2 * c], p1 = Ph[2 * c + 1];
      // W(m) = P_2c + i P_2c+1 ; W(-m) = conj(P_2c) + i conj(P_2c+1)
      R[((j * 2 + 0) * ncm + c) * K + mx] = {p0.x - p1.y, p0.y + p1.x};
      R[((j * 2 + 1) * ncm + c) * K + mmx] = {p0.x + p1.y, -p0.y + p1.x};
    }
  }
  __syncthreads();
  V* res = fft_lines<T>(R, other, nslot, K, fp, tw_s, (T)1);
  for (int idx = threadIdx.x; idx < nslot * K; idx += blockDim.x) {
    int slot = idx % nslot, e = idx / nslot;
    int c = slot % ncm, jab = slot / ncm;
    int2 pr = xpairs[it.y + (jab >> 1)];
    if ((jab & 1) && pr.y == pr.x) continue;  // self-paired line: written from its A copy
    int l = (jab & 1) ? pr.y : pr.x;
    mesh[S.mesh_off + (int64_t)c * S.M + l + (int64_t)e * estride] = res[slot * K + e];
  }
}

// ------------------------------------------------------------------ spreading
template <typename T, int P>
__global__ void k_spread(const StructDev* __restrict__ st, const int* __restrict__ bin_struct,
                         const int* __restrict__ bin_start, const int* __restrict__ base,
                         const T* __restrict__ wts, const int* __restrict__ spec, const double* __restrict__ x,
                         const PcgScalars* __restrict__ sc, int use_active, typename C2<T>::t* __restrict__ mesh) {
  using V = typename C2<T>::t;
  const int g = blockIdx.x;
  const int s = bin_struct[g];
  const StructDev& S = st[s];
  if (use_active && !sc[s].active) return;
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncm = S.ncm;
  int gl = g - S.bin_off;
  int bc[3];
  bc[2] = gl % S.nb[2];
  bc[1] = (gl / S.nb[2]) % S.nb[1];
  bc[0] = gl / (S.nb[2] * S.nb[1]);
  int x0[3], ext[3];
  for (int d = 0; d < 3; ++d) {
    x0[d] = bc[d] * QEQ_BIN;
    ext[d] = min(QEQ_BIN, S.K[d] - x0[d]);
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* acc = reinterpret_cast<T*>(smem_raw);  // [nw][ncm][512][2]
  const int bsz = QEQ_BIN * QEQ_BIN * QEQ_BIN;
  T* wsm = acc + (size_t)nw * ncm * bsz * 2;  // [nw][3][P] weights
  int* lsm = reinterpret_cast<int*>(wsm + nw * 3 * P);  // [nw][3][P] local indices
  int* cnt = lsm + nw * 3 * P;                          // [nw][3]
  for (int i = threadIdx.x; i < nw * ncm * bsz * 2; i += blockDim.x) acc[i] = (T)0;
  // candidate bins per direction: the bins of points x0 .. x0+ext+P-2 (mod K)
  __shared__ int cand[3][8], ncand[3];
  if (threadIdx.x < 3) {
    int d = threadIdx.x, nc = 0;
    int span = ext[d] + P - 1;
    if (span > S.K[d]) span = S.K[d];
    for (int k = 0; k < span; ++k) {
      int bn = ((x0[d] + k) % S.K[d]) / QEQ_BIN;
      bool seen = false;
      for (int q = 0; q < nc; ++q) seen |= (cand[d][q] == bn);
      if (!seen && nc < 8) cand[d][nc++] = bn;
    }
    ncand[d] = nc;
  }
  __syncthreads();
  T* my = acc + (size_t)w * ncm * bsz * 2;
  T* mw = wsm + w * 3 * P;
  int* ml = lsm + w * 3 * P;
  int* mc = cnt + w * 3;
  int order = 0;
  for (int i0 = 0; i0 < ncand[0]; ++i0)
    for (int i1 = 0; i1 < ncand[1]; ++i1)
      for (int i2 = 0; i2 < ncand[2]; ++i2) {
        int gb = S.bin_off + (cand[0][i0] * S.nb[1] + cand[1][i1]) * S.nb[2] + cand[2][i2];
        int t0 = bin_start[gb], t1 = bin_start[gb + 1];
        for (int t = t0; t < t1; ++t, ++order) {
          if ((order % nw) != w) continue;
          int bs = base[t];
          int f[3] = {bs & 1023, (bs >> 10) & 1023, (bs >> 20) & 1023};
          if (lane < 3) {
            int d = lane, n = 0;
            for (int j = 0; j < P; ++j) {
              int k = f[d] - (P - 1) + j;
              if (k < 0) k += S.K[d];
              int loc = k - x0[d];
              if (loc >= 0 && loc < ext[d]) {
                ml[d * P + n] = loc;
                mw[d * P + n] = wts[(size_t)t * 3 * QEQ_MAXP + d * QEQ_MAXP + (P - 1 - j)];
                ++n;
              }
            }
            mc[d] = n;
          }
          __syncwarp();
          int n0 = mc[0], n1 = mc[1], n2 = mc[2];
          int tot = n0 * n1 * n2;
          int sp = spec[t];
          int cm = sp >> 1, part = sp & 1;
          T qv = (T)x[t];
          T* dst = my + (size_t)cm * bsz * 2 + part;
          for (int c = lane; c < tot; c += 32) {
            int iz = c % n2, r = c / n2;
            int iy = r % n1, ix = r / n1;
            int pt = (ml[ix] * QEQ_BIN + ml[P + iy]) * QEQ_BIN + ml[2 * P + iz];
            dst[pt * 2] += qv * mw[ix] * mw[P + iy] * mw[2 * P + iz];
          }
          __syncwarp();
        }
      }
  __syncthreads();
  for (int i = threadIdx.x; i < ncm * bsz; i += blockDim.x) {
    int cm = i / bsz, pt = i - cm * bsz;
    int lz = pt % QEQ_BIN, ly = (pt / QEQ_BIN) % QEQ_BIN, lx = pt / (QEQ_BIN * QEQ_BIN);
    if (lx >= ext[0] || ly >= ext[1] || lz >= ext[2]) continue;
    V v = {(T)0, (T)0};
    for (int ww = 0; ww < nw; ++ww) {
      v.x += acc[(((size_t)ww * ncm + cm) * bsz + pt) * 2];
      v.y += acc[(((size_t)ww * ncm + cm) * bsz + pt) * 2 + 1];
    }
    int64_t gi = S.mesh_off + (int64_t)cm * S.M + ((int64_t)(x0[0] + lx) * S.K[1] + (x0[1] + ly)) * S.K[2] +
                 (x0[2] + lz);
    mesh[gi] = v;
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

template <typename T, int P>
__global__ void k_gather(const StructDev* __restrict__ st, const int* __restrict__ bin_struct,
                         const int* __restrict__ bin_start, const int* __restrict__ base,
                         const T* __restrict__ wts, const int* __restrict__ spec, const double* __restrict__ J,
                         const double* __restrict__ x, const int64_t* __restrict__ row, const int* __restrict__ col,
                         const double* __restrict__ v64, const float* __restrict__ v32, int with_J, int with_pairs,
                         PcgScalars* __restrict__ sc, int use_active, int fuse_pAp, double* __restrict__ part,
                         int* __restrict__ counter, const typename C2<T>::t* __restrict__ mesh,
                         double* __restrict__ y) {
  using V = typename C2<T>::t;
  const int g = blockIdx.x;
  const int s = bin_struct[g];
  const StructDev& S = st[s];
  if (use_active && !sc[s].active) return;
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncm = S.ncm;
  int gl = g - S.bin_off;
  int bc[3];
  bc[2] = gl % S.nb[2];
  bc[1] = (gl / S.nb[2]) % S.nb[1];
  bc[0] = gl / (S.nb[2] * S.nb[1]);
  int x0[3], len[3];
  for (int d = 0; d < 3; ++d) {
    x0[d] = bc[d] * QEQ_BIN;
    len[d] = min(QEQ_BIN, S.K[d] - x0[d]) + P - 1;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* reg = reinterpret_cast<V*>(smem_raw);  // [ncm][len0][len1][len2]
  const int rsz = len[0] * len[1] * len[2];
  for (int i = threadIdx.x; i < ncm * rsz; i += blockDim.x) {
    int cm = i / rsz, pt = i - cm * rsz;
    int lz = pt % len[2], ly = (pt / len[2]) % len[1], lx = pt / (len[2] * len[1]);
    int kx = x0[0] - (P - 1) + lx, ky = x0[1] - (P - 1) + ly, kz = x0[2] - (P - 1) + lz;
    kx = ((kx % S.K[0]) + S.K[0]) % S.K[0];
    ky = ((ky % S.K[1]) + S.K[1]) % S.K[1];
    kz = ((kz % S.K[2]) + S.K[2]) % S.K[2];
    reg[i] = mesh[S.mesh_off + (int64_t)cm * S.M + ((int64_t)kx * S.K[1] + ky) * S.K[2] + kz];
  }
  __syncthreads();
  const T* vals = pair_vals<T>(v64, v32);
  double blk = 0.0;
  int t0 = bin_start[g], t1 = bin_start[g + 1];
  for (int t = t0 + w; t < t1; t += nw) {
    int bs = base[t];
    int f[3] = {bs & 1023, (bs >> 10) & 1023, (bs >> 20) & 1023};
    int sp = spec[t];
    int cm = sp >> 1, part = sp & 1;
    const T* wt = wts + (size_t)t * 3 * QEQ_MAXP;
    const V* rg = reg + (size_t)cm * rsz;
    // stencil point f - (P-1) + j sits at local index f - x0 + j and carries weight M_p(w + P-1-j)
    int o0 = f[0] - x0[0], o1 = f[1] - x0[1], o2 = f[2] - x0[2];
    T acc = (T)0;
    for (int c = lane; c < P * P * P; c += 32) {
      int jz = c % P, r = c / P;
      int jy = r % P, jx = r / P;
      V v = rg[((o0 + jx) * len[1] + (o1 + jy)) * len[2] + (o2 + jz)];
      T val = part ? v.y : v.x;
      acc += wt[P - 1 - jx] * wt[QEQ_MAXP + P - 1 - jy] * wt[2 * QEQ_MAXP + P - 1 - jz] * val;
    }
    if (with_pairs) {
      int64_t r0 = row[t], r1 = row[t + 1];
      for (int64_t k = r0 + lane; k < r1; k += 32) acc += vals[k] * (T)x[col[k]];
    }
    acc = warp_sum<T>(acc);
    if (lane == 0) {
      double xi = x[t];
      double loc = S.self_s[sp] * xi;
      if (with_J) loc += J[t] * xi;
      const PcgScalars& c = sc[s];
      for (int tt = 0; tt < S.S; ++tt) loc -= S.corr[sp * QEQ_MAX_SPECIES + tt] * c.xsum[tt];
      double yi = (double)acc + loc;
      y[t] = yi;
      blk += xi * yi;
    }
  }
  if (fuse_pAp) {
    // deterministic per-structure reduction of x.y over the structure's bins
    __shared__ double wsum[32];
    if (lane == 0) wsum[w] = blk;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int i = 0; i < nw; ++i) b += wsum[i];
      part[g] = b;
      __threadfence();
      int nbs = S.nb[0] * S.nb[1] * S.nb[2];
      int prev = atomicAdd(&counter[s], 1);
      if (prev == nbs - 1) {
        __threadfence();
        double tot = 0.0;
        for (int i = 0; i < nbs; ++i) tot += ((volatile double*)part)[S.bin_off + i];
        PcgScalars& c = sc[s];
        c.pAp = tot;
        c.alpha = (tot != 0.0) ? c.rz / tot : 0.0;
        counter[s] = 0;
      }
    }
  }
}

// ------------------------------------------------------------------ per-species sums of x
__global__ void k_species_sums(const Chunk* __restrict__ chunks, const StructDev* __restrict__ st,
                               const int* __restrict__ spec, const double* __restrict__ x,
                               PcgScalars* __restrict__ sc, int use_active, double* __restrict__ part,
                               int* __restrict__ counter) {
  const Chunk ch = chunks[blockIdx.x];
  if (use_active && !sc[ch.s].active) return;
  __shared__ double red[QEQ_MAX_SPECIES][33];
  double loc[QEQ_MAX_SPECIES];
  for (int k = 0; k < QEQ_MAX_SPECIES; ++k) loc[k] = 0.0;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) loc[spec[a]] += x[a];
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
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int prev = atomicAdd(&counter[ch.s], 1);
    if (prev == ch.count - 1) {
      __threadfence();
      PcgScalars& c = sc[ch.s];
      for (int k = 0; k < QEQ_MAX_SPECIES; ++k) {
        double tot = 0.0;
        for (int i = 0; i < ch.count; ++i)
          tot += ((volatile double*)part)[(size_t)(ch.first + i) * QEQ_MAX_SPECIES + k];
        c.xsum[k] = tot;
      }
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
  const int nw_spread = F32 ? 8 : 4;
  const int maxncm = Pl->max_ncm;
  int rec = 0;
  auto mark = [&]() -> cudaError_t { return ev ? cudaEventRecord(ev[rec++], s) : cudaSuccess; };
  count_launch(Pl, 8);
  QEQ_CUDA_TRY(mark());
  // stage 0: per-species sums of x (width-correction terms)
  k_species_sums<<<Pl->n_chunks, 256, 0, s>>>(Pl->d_chunks, Pl->d_st, Pl->d_spec, x, Pl->d_sc, use_active,
                                               Pl->d_part, Pl->d_counter);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  // stage 1: spreading
  {
    size_t sm = (size_t)nw_spread * maxncm * 512 * 2 * sizeof(T) +
                (size_t)nw_spread * 3 * P * (sizeof(T) + sizeof(int)) + nw_spread * 3 * sizeof(int) + 64;
    k_spread<T, P><<<Pl->total_bins, nw_spread * 32, sm, s>>>(Pl->d_st, Pl->d_bin_struct, Pl->d_bin_start,
                                                              Pl->d_base, wts, Pl->d_spec, x, Pl->d_sc, use_active,
                                                              mesh);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  QEQ_CUDA_TRY(mark());
  const size_t smf = csz * (size_t)Pl->fft_smem_elems;
  // stages 2-6: forward z, forward y, x + reciprocal multiply + inverse x, inverse y, inverse z
  k_fft_z<T><<<Pl->n_zitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_zitems, Pl->d_tw64, Pl->d_tw32, Pl->d_sc,
                                             use_active, mesh, (T)-1);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_y<T><<<Pl->n_yitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_yitems, Pl->d_tw64, Pl->d_tw32, Pl->d_sc,
                                             use_active, mesh, (T)-1, Pl->ly);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_x_green<T><<<Pl->n_xitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_xitems, Pl->d_xpairs, bmod,
                                                   Pl->d_tw64, Pl->d_tw32, Pl->d_sc, use_active, mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_y<T><<<Pl->n_yitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_yitems, Pl->d_tw64, Pl->d_tw32, Pl->d_sc,
                                             use_active, mesh, (T)1, Pl->ly);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_fft_z<T><<<Pl->n_zitems, 256, smf, s>>>(Pl->d_st, Pl->d_fft, Pl->d_zitems, Pl->d_tw64, Pl->d_tw32, Pl->d_sc,
                                             use_active, mesh, (T)1);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  // stage 7: gathering + real-space pairs + local terms (+ x.y per structure)
  {
    int reg = QEQ_BIN + P - 1;
    size_t sm = csz * (size_t)maxncm * reg * reg * reg + 64;
    int with_pairs = Pl->pair_cap > 0;
    k_gather<T, P><<<Pl->total_bins, 256, sm, s>>>(Pl->d_st, Pl->d_bin_struct, Pl->d_bin_start, Pl->d_base, wts,
                                                   Pl->d_spec, Pl->d_J, x, Pl->d_row, Pl->d_col, Pl->d_val64,
                                                   Pl->d_val32, with_J, with_pairs, Pl->d_sc, use_active, fuse_pAp,
                                                   Pl->d_part + (size_t)Pl->n_chunks * QEQ_MAX_SPECIES,
                                                   Pl->d_counter + Pl->n_struct, mesh, y);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  QEQ_CUDA_TRY(mark());
  return cudaSuccess;
}

template <typename T, int P>
cudaError_t set_smem_attrs() {
  const int big = 200 * 1024;
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_spread<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_gather<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
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
