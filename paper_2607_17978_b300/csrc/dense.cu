// 4G charge training on cached dense matrices (Sec. "4G-HDNNP Charge Training"):
// the Coulomb matrix E of every training structure (no hardness) is assembled once,
// the bordered matrix A' = [[E + diag J, 1], [1^T, 0]] of eq. (4G_qeq_prime) is
// inverted whenever the learned hardness J changes, and each training step's charges
// are one matrix-vector product q' = -A'^{-1} chi', chi' = (chi, -q_tot).  The adjoint
// of that product gives the training gradients: with (lam, nu) = A'^{-1} (dL/dq, 0),
// dL/dchi = -lam and dL/dJ_i = -lam_i q_i.
//
// E is the periodic Gaussian-charge Coulomb matrix of eq. (elec_energy) with the G = 0
// term dropped, by the Ewald split of SI "Ewald Summation" with one width omega >= every
// gamma_ij, so that all pairs share the reciprocal Gaussian:
//   real space    k_e sum_n [erfc(r/(sqrt2 omega)) - erfc(r/(sqrt2 gamma_ij))]/r  (r < r_c)
//   reciprocal    k_e (4 pi/V) sum_{G != 0} exp(-G^2 omega^2/2) cos(G.(r_i - r_j))/G^2
//   self (i = j)  k_e sqrt(2/pi) (1/gamma_ii - 1/omega)
//   G = 0 width   -k_e (2 pi/V)(omega^2 - gamma_ij^2)
// Everything is FP64.  One CTA per 32 x 32 tile of E; one CTA per structure for the
// inverse (Cholesky A = U^T U, U^{-1} by back substitution, A^{-1} = U^{-1} U^{-T}, then
// the border by the Schur complement s = 1^T A^{-1} 1).  Every sum runs in a fixed order.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "qeq_internal.cuh"

namespace {

constexpr double kPiD = 3.14159265358979323846;

struct DenseStructDev {
  double h[9];
  double hinv[9];
  double V;
  double omega;  // Ewald width, >= every gamma_ij of the structure
  double rc2;    // real-space cutoff squared
  double ext[3]; // r_c / (distance between lattice planes) per direction
  double sigma[QEQ_MAX_SPECIES];
  int n;         // atoms
  int S;         // species
  int M[3];      // phase tables: m_d in [-M_d, M_d]
  int W;         // sum_d (2 M_d + 1)
  int ng;        // G vectors of the half space
  int g_off;
  int64_t atom_off;
  int64_t e_off;   // E, n x n
  int64_t k_off;   // A'^{-1}, (n + 1) x (n + 1)
  int64_t ph_off;  // phase tables, n x W complex
};

struct DenseG {
  int m[3];
  int pad;
  double f;  // 2 k_e (4 pi / V) exp(-G^2 omega^2 / 2) / G^2 (factor 2: the -G partner)
};

}  // namespace

struct qeq_dense_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_struct = 0, n_species = 0, max_n = 0;
  int64_t n_atoms = 0;
  double k_e = 14.3996454784, tol = 1e-12;
  std::vector<DenseStructDev> hs;
  std::vector<int4> tiles;
  DenseStructDev* d_st = nullptr;
  DenseG* d_g = nullptr;
  int4* d_tiles = nullptr;
  int* d_atom_struct = nullptr;
  double* d_frac = nullptr;   // 3 per atom, wrapped fractional coordinates
  double2* d_ph = nullptr;    // phase tables
  double* d_E = nullptr;
  double* d_K = nullptr;
  double* d_Y = nullptr;      // U^{-1} during the inversion
  // QEQ_MIXED: the inverse in FP32 (the B300's FP32 pipe is ~64x its FP64 pipe), charges and
  // gradients refined in FP64 against the exact bordered matrix (E in FP64, J kept here)
  int mixed = 0;
  float* d_K32 = nullptr;
  float* d_Y32 = nullptr;
  double* d_Jc = nullptr;
  double* d_qtot = nullptr;
  std::vector<double> h_qtot;
  int* d_err = nullptr;
  int err_host = 0;
  bool assembled = false, inverted = false;
  int64_t launches = 0;
  std::string last_error;
};

namespace {

enum { DERR_INPUT = 1, DERR_SPECIES = 2, DERR_NOT_PD = 4 };

// wrapped fractional coordinates and the phase tables exp(i 2 pi m u_d), m = -M_d..M_d
__global__ void k_dense_phases(const DenseStructDev* __restrict__ st, const int* __restrict__ atom_struct, int64_t n,
                               const double* __restrict__ pos, const int32_t* __restrict__ species,
                               double* __restrict__ frac, double2* __restrict__ ph, int* __restrict__ err) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const DenseStructDev& S = st[atom_struct[a]];
  double r[3] = {pos[3 * a], pos[3 * a + 1], pos[3 * a + 2]};
  int bad = 0;
  if (!isfinite(r[0]) || !isfinite(r[1]) || !isfinite(r[2])) {
    bad |= DERR_INPUT;
    r[0] = r[1] = r[2] = 0.0;
  }
  const int sp = species[a];
  if (sp < 0 || sp >= S.S) bad |= DERR_SPECIES;
  if (bad) atomicOr(err, bad);
  const int64_t loc = a - S.atom_off;
  double2* t = ph + S.ph_off + loc * S.W;
  int base = 0;
  for (int d = 0; d < 3; ++d) {
    double u = r[0] * S.hinv[d] + r[1] * S.hinv[3 + d] + r[2] * S.hinv[6 + d];
    u -= floor(u);
    if (u >= 1.0) u = 0.0;
    frac[3 * a + d] = u;
    for (int m = -S.M[d]; m <= S.M[d]; ++m) {
      double s, c;
      sincospi(2.0 * m * u, &s, &c);
      t[base + m + S.M[d]] = make_double2(c, s);
    }
    base += 2 * S.M[d] + 1;
  }
}

// One 32 x 32 tile of E per CTA: thread t owns row t / 8 and columns (t mod 8) + 8 k.
constexpr int kTile = 32, kGChunk = 32;  // 2 x 32 x 33 x 16 B of phases: under the 48 KB static limit

__global__ void __launch_bounds__(256) k_dense_assemble(const DenseStructDev* __restrict__ st,
                                                        const int4* __restrict__ tiles,
                                                        const double* __restrict__ frac,
                                                        const int32_t* __restrict__ species,
                                                        const DenseG* __restrict__ gl,
                                                        const double2* __restrict__ ph, double k_e,
                                                        double* __restrict__ E) {
  __shared__ double2 pi_[kTile][kGChunk + 1];
  __shared__ double2 pj_[kTile][kGChunk + 1];
  __shared__ double fg[kGChunk];
  __shared__ double ui[kTile][3], uj[kTile][3], si[kTile], sj[kTile];
  const int4 tl = tiles[blockIdx.x];
  const DenseStructDev& S = st[tl.x];
  const int n = S.n, i0 = tl.y * kTile, j0 = tl.z * kTile;
  const int t = threadIdx.x;
  if (t < kTile) {
    const int i = i0 + t, j = j0 + t;
    for (int d = 0; d < 3; ++d) {
      ui[t][d] = (i < n) ? frac[3 * (S.atom_off + i) + d] : 0.0;
      uj[t][d] = (j < n) ? frac[3 * (S.atom_off + j) + d] : 0.0;
    }
    int spi = (i < n) ? species[S.atom_off + i] : 0, spj = (j < n) ? species[S.atom_off + j] : 0;
    spi = min(max(spi, 0), S.S - 1);
    spj = min(max(spj, 0), S.S - 1);
    si[t] = S.sigma[spi];
    sj[t] = S.sigma[spj];
  }
  __syncthreads();
  const int r = t >> 3, c0 = t & 7;
  const double w = S.omega, pref = k_e * 4.0 * kPiD / S.V;
  const double inv_sw = 1.0 / (sqrt(2.0) * w);
  double acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + 8 * k;
    const int i = i0 + r, j = j0 + c;
    double a = 0.0;
    if (i < n && j < n) {
      const double g = sqrt(si[r] * si[r] + sj[c] * sj[c]);
      a = -0.5 * pref * (w * w - g * g);  // G = 0 width term
      if (i == j) a += k_e * sqrt(2.0 / kPiD) * (1.0 / g - 1.0 / w);
      if (w > g) {  // real-space images within r_c
        const double inv_sg = 1.0 / (sqrt(2.0) * g);
        double f[3];
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
          f[d] = uj[c][d] - ui[r][d];
          f[d] -= rint(f[d]);
          lo[d] = (int)ceil(-S.ext[d] - f[d]);
          hi[d] = (int)floor(S.ext[d] - f[d]);
        }
        for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
          for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
            for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
              if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;
              const double x = f[0] + n0, y = f[1] + n1, z = f[2] + n2;
              const double dx = x * S.h[0] + y * S.h[3] + z * S.h[6];
              const double dy = x * S.h[1] + y * S.h[4] + z * S.h[7];
              const double dz = x * S.h[2] + y * S.h[5] + z * S.h[8];
              const double d2 = dx * dx + dy * dy + dz * dz;
              if (d2 >= S.rc2) continue;
              if (d2 < 1e-24) {  // coincident images: the r -> 0 limit
                a += k_e * sqrt(2.0 / kPiD) * (1.0 / g - 1.0 / w);
                continue;
              }
              const double rr = sqrt(d2);
              a += k_e * (erfc(rr * inv_sw) - erfc(rr * inv_sg)) / rr;
            }
      }
    }
    acc[k] = a;
  }
  // reciprocal part: phases of the tile's atoms for a chunk of G vectors, then the products
  const double2* phb = ph + S.ph_off;
  const int o1 = 2 * S.M[0] + 1, o2 = o1 + 2 * S.M[1] + 1;
  for (int g0 = 0; g0 < S.ng; g0 += kGChunk) {
    const int ngc = min(kGChunk, S.ng - g0);
    __syncthreads();
    if (t < ngc) fg[t] = gl[S.g_off + g0 + t].f;
    for (int e = t; e < 2 * kTile * ngc; e += blockDim.x) {
      const int side = e / (kTile * ngc), rem = e - side * kTile * ngc;
      const int at = rem / ngc, g = rem - at * ngc;
      const int atom = (side ? j0 : i0) + at;
      double2 v = make_double2(0.0, 0.0);
      if (atom < n) {
        const DenseG G = gl[S.g_off + g0 + g];
        const double2* tb = phb + (int64_t)atom * S.W;
        const double2 a = tb[G.m[0] + S.M[0]], b = tb[o1 + G.m[1] + S.M[1]], c = tb[o2 + G.m[2] + S.M[2]];
        const double abr = a.x * b.x - a.y * b.y, abi = a.x * b.y + a.y * b.x;
        v = make_double2(abr * c.x - abi * c.y, abr * c.y + abi * c.x);
      }
      if (side)
        pj_[at][g] = v;
      else
        pi_[at][g] = v;
    }
    __syncthreads();
    for (int g = 0; g < ngc; ++g) {
      const double2 p = pi_[r][g];
      const double fgg = fg[g];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double2 q = pj_[c0 + 8 * k][g];
        acc[k] += fgg * (p.x * q.x + p.y * q.y);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + r, j = j0 + c0 + 8 * k;
    if (i < n && j < n) E[S.e_off + (int64_t)i * n + j] = acc[k];
  }
}

__device__ __forceinline__ double dense_block_sum(double a, double* red) {
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  double tot = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];  // every thread, same order
  __syncthreads();
  return tot;
}

// A'^{-1} of one structure per CTA (n <= QEQ_DENSE_MAX_ATOMS), in the K buffer (ld n + 1),
// in the arithmetic type T (double; float for the refined FP32 inverse).
template <typename T>
__device__ __forceinline__ T dense_block_sum_t(T a, T* red) {
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  T tot = (T)0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];  // every thread, same order
  __syncthreads();
  return tot;
}

template <typename T>
__global__ void __launch_bounds__(256) k_dense_invert(const DenseStructDev* __restrict__ st,
                                                      const double* __restrict__ E, const double* __restrict__ J,
                                                      T* __restrict__ Kbuf, T* __restrict__ Ybuf,
                                                      int* __restrict__ err) {
  __shared__ T col[QEQ_DENSE_MAX_ATOMS];
  __shared__ T red[8];
  __shared__ int fail;
  const DenseStructDev& S = st[blockIdx.x];
  const int n = S.n, ld = n + 1, t = threadIdx.x, nt = blockDim.x;
  T* U = Kbuf + S.k_off;  // A, then U (upper rows), then A^{-1}, then A'^{-1}
  T* Y = Ybuf + S.e_off;  // U^{-1}, upper, row-major (ld n)
  const double* Es = E + S.e_off;
  if (t == 0) fail = 0;
  for (int64_t e = t; e < (int64_t)n * n; e += nt) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    U[(int64_t)i * ld + j] = (T)(Es[e] + (i == j ? J[S.atom_off + i] : 0.0));
  }
  __syncthreads();
  // Cholesky A = U^T U, row by row: U_jj = sqrt(A_jj - sum_k U_kj^2),
  // U_ji = (A_ji - sum_{k<j} U_ki U_kj) / U_jj for i > j (threads over i: coalesced rows k)
  for (int j = 0; j < n; ++j) {
    for (int k = t; k < j; k += nt) col[k] = U[(int64_t)k * ld + j];
    __syncthreads();
    T part = (T)0;
    for (int k = t; k < j; k += nt) part += col[k] * col[k];
    const T dsum = dense_block_sum_t<T>(part, red);
    const T djj = U[(int64_t)j * ld + j] - dsum;
    if (!(djj > (T)0)) {  // not positive definite (uniform across the block)
      if (t == 0) {
        atomicOr(err, DERR_NOT_PD);
        fail = 1;
      }
      break;
    }
    const T ujj = sqrt(djj);
    for (int i = j + 1 + t; i < n; i += nt) {
      T s = U[(int64_t)j * ld + i];
      for (int k = 0; k < j; ++k) s -= U[(int64_t)k * ld + i] * col[k];
      U[(int64_t)j * ld + i] = s / ujj;
    }
    __syncthreads();
    if (t == 0) U[(int64_t)j * ld + j] = ujj;
    __syncthreads();
  }
  __syncthreads();
  if (fail) return;
  // Y = U^{-1} (upper), rows from the bottom: Y_ic = (delta_ic - sum_{k=i+1..c} U_ik Y_kc) / U_ii
  for (int i = n - 1; i >= 0; --i) {
    for (int k = i + t; k < n; k += nt) col[k] = U[(int64_t)i * ld + k];
    __syncthreads();
    const T inv = (T)1 / col[i];
    for (int c = i + t; c < n; c += nt) {
      T s = (c == i) ? (T)1 : (T)0;
      for (int k = i + 1; k <= c; ++k) s -= col[k] * Y[(int64_t)k * n + c];
      Y[(int64_t)i * n + c] = s * inv;
    }
    for (int c = t; c < i; c += nt) Y[(int64_t)i * n + c] = (T)0;
    __syncthreads();
  }
  // A^{-1} = Y Y^T: entry (a, b) = sum_{k >= max(a, b)} Y_ak Y_bk, 32 x 32 tiles through shared memory
  T* ta = col;  // reuse: 2 x 16 x 32 values = 1024 (two half-height staging buffers)
  for (int tb = 0; tb * 32 < n; ++tb)
    for (int tA = 0; tA <= tb; ++tA) {
      const int a0 = tA * 32, b0 = tb * 32;
      const int r = t >> 3, c0 = t & 7;
      T acc[4] = {(T)0, (T)0, (T)0, (T)0};
      for (int k0 = b0; k0 < n; k0 += 16) {  // Y_ak = 0 for k < a, and a, b < b0 + 32
        __syncthreads();
        for (int e = t; e < 2 * 32 * 16; e += nt) {
          const int side = e >> 9, rem = e & 511, row = rem >> 4, kk = rem & 15;
          const int gr = (side ? b0 : a0) + row, gk = k0 + kk;
          ta[e] = (gr < n && gk < n) ? Y[(int64_t)gr * n + gk] : (T)0;
        }
        __syncthreads();
        for (int kk = 0; kk < 16; ++kk) {
          const T ya = ta[(r << 4) + kk];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += ya * ta[512 + ((c0 + 8 * q) << 4) + kk];
        }
      }
      // the k < b0 part is zero for rows of b (Y upper), so the loop from b0 is complete
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = a0 + r, b = b0 + c0 + 8 * q;
        if (a < n && b < n) {
          U[(int64_t)a * ld + b] = acc[q];
          U[(int64_t)b * ld + a] = acc[q];
        }
      }
    }
  __syncthreads();
  // border: v = A^{-1} 1, s = 1^T v; A'^{-1} = [[A^{-1} - v v^T / s, v / s], [v^T / s, -1 / s]]
  for (int a = t; a < n; a += nt) {
    T v = (T)0;
    for (int b = 0; b < n; ++b) v += U[(int64_t)a * ld + b];
    col[a] = v;
  }
  __syncthreads();
  T part = (T)0;
  for (int a = t; a < n; a += nt) part += col[a];
  const T s = dense_block_sum_t<T>(part, red);
  const T is = (T)1 / s;
  for (int64_t e = t; e < (int64_t)n * n; e += nt) {
    const int a = (int)(e / n), b = (int)(e - (int64_t)a * n);
    U[(int64_t)a * ld + b] -= col[a] * col[b] * is;
  }
  for (int a = t; a < n; a += nt) {
    U[(int64_t)a * ld + n] = col[a] * is;
    U[(int64_t)n * ld + a] = col[a] * is;
  }
  if (t == 0) U[(int64_t)n * ld + n] = -is;
}

// y = A'^{-1} (x, x_n) per structure, one warp per row (lanes over the row: coalesced);
// mode 0: x = -chi, x_n = q_tot -> q = y[:n], mu = -y[n]; mode 1: x = dL/dq, x_n = 0 ->
// dL/dchi = -y[:n], dL/dJ = -y[:n] q
template <int MODE>
__global__ void __launch_bounds__(256) k_dense_apply(const DenseStructDev* __restrict__ st,
                                                     const double* __restrict__ Kbuf, const double* __restrict__ x,
                                                     const double* __restrict__ qtot, const double* __restrict__ q,
                                                     double* __restrict__ o1, double* __restrict__ o2) {
  const DenseStructDev& S = st[blockIdx.x];
  const int n = S.n, ld = n + 1, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double* K = Kbuf + S.k_off;
  const double* xs = x + S.atom_off;
  const double xn = MODE == 0 ? qtot[blockIdx.x] : 0.0;
  for (int a = w; a <= n; a += (blockDim.x >> 5)) {
    double acc = 0.0;
    for (int b = lane; b < n; b += 32) acc += K[(int64_t)a * ld + b] * (MODE == 0 ? -xs[b] : xs[b]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double y = acc + K[(int64_t)a * ld + n] * xn;
      if (MODE == 0) {
        if (a < n)
          o1[S.atom_off + a] = y;
        else if (o2)
          o2[blockIdx.x] = -y;
      } else if (a < n) {
        o1[S.atom_off + a] = -y;
        if (o2) o2[S.atom_off + a] = -y * q[S.atom_off + a];
      }
    }
  }
}

// FP64 solution of A' x = b with the FP32 inverse, by iterative refinement:
// x = K32 b, then twice r = b - A' x (A' = [[E + diag J, 1], [1^T, 0]] in FP64), x += K32 r.
// Each step shrinks the error by about cond(A') * eps_FP32; two steps give FP64 accuracy for
// the well-conditioned QEq matrices.  One CTA per structure, x and r in shared memory.
// MODE 0: b = (-chi, q_tot) -> q = x[:n], mu = -x[n];  MODE 1: b = (dL/dq, 0) ->
// dL/dchi = -x[:n], dL/dJ = -x[:n] q.
template <int MODE>
__global__ void __launch_bounds__(256) k_dense_refine(const DenseStructDev* __restrict__ st,
                                                      const float* __restrict__ K32, const double* __restrict__ E,
                                                      const double* __restrict__ J, const double* __restrict__ xin,
                                                      const double* __restrict__ qtot, const double* __restrict__ q,
                                                      double* __restrict__ o1, double* __restrict__ o2) {
  __shared__ double xs[QEQ_DENSE_MAX_ATOMS + 1];
  __shared__ double bs[QEQ_DENSE_MAX_ATOMS + 1];
  __shared__ double rs[QEQ_DENSE_MAX_ATOMS + 1];
  __shared__ double red[8];
  const DenseStructDev& S = st[blockIdx.x];
  const int n = S.n, ld = n + 1, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float* K = K32 + S.k_off;
  const double* Es = E + S.e_off;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    bs[a] = MODE == 0 ? -xin[S.atom_off + a] : xin[S.atom_off + a];
    xs[a] = 0.0;
  }
  if (threadIdx.x == 0) {
    bs[n] = MODE == 0 ? qtot[blockIdx.x] : 0.0;
    xs[n] = 0.0;
  }
  __syncthreads();
  // r = b initially (x = 0); then three applications of K32, two residuals
  for (int a = threadIdx.x; a <= n; a += blockDim.x) rs[a] = bs[a];
  __syncthreads();
  for (int step = 0; step < 3; ++step) {
    // x += K32 r, one warp per row, FP64 accumulation
    for (int a = w; a <= n; a += nw) {
      double acc = 0.0;
      for (int b = lane; b <= n; b += 32) acc += (double)K[(int64_t)a * ld + b] * rs[b];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) xs[a] += acc;
    }
    __syncthreads();
    if (step == 2) break;
    // r = b - A' x in FP64
    for (int a = w; a < n; a += nw) {
      double acc = 0.0;
      for (int b = lane; b < n; b += 32) acc += Es[(int64_t)a * n + b] * xs[b];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) rs[a] = bs[a] - (acc + J[S.atom_off + a] * xs[a] + xs[n]);
    }
    double part = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) part += xs[a];
    const double sx = dense_block_sum(part, red);
    if (threadIdx.x == 0) rs[n] = bs[n] - sx;
    __syncthreads();
  }
  for (int a = threadIdx.x; a <= n; a += blockDim.x) {
    const double y = xs[a];
    if (MODE == 0) {
      if (a < n)
        o1[S.atom_off + a] = y;
      else if (o2)
        o2[blockIdx.x] = -y;
    } else if (a < n) {
      o1[S.atom_off + a] = -y;
      if (o2) o2[S.atom_off + a] = -y * q[S.atom_off + a];
    }
  }
}

__global__ void k_f2d(const float* __restrict__ a, int64_t n, double* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

qeq_status dfail(qeq_dense_s* D, qeq_status s, const std::string& m) {
  D->last_error = m;
  return s;
}

qeq_status dcuda(qeq_dense_s* D, cudaError_t e, const char* what) {
  D->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return QEQ_ERR_CUDA;
}

#define DTRY(expr)                                      \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return dcuda(D, e_, #expr);  \
  } while (0)

// device error bits -> status (and clear them)
qeq_status dense_check(qeq_dense_s* D) {
  DTRY(cudaMemcpyAsync(&D->err_host, D->d_err, sizeof(int), cudaMemcpyDeviceToHost, D->stream));
  DTRY(cudaStreamSynchronize(D->stream));
  if (D->err_host) {
    const int e = D->err_host;
    DTRY(cudaMemsetAsync(D->d_err, 0, sizeof(int), D->stream));
    DTRY(cudaStreamSynchronize(D->stream));
    if (e & DERR_NOT_PD) return dfail(D, QEQ_ERR_NOT_PD, "E + diag J is not positive definite");
    return dfail(D, QEQ_ERR_INVALID, (e & DERR_SPECIES) ? "species index out of range" : "non-finite position");
  }
  return QEQ_OK;
}

void dense_free(qeq_dense_s* D) {
  void* p[] = {D->d_st, D->d_g, D->d_tiles, D->d_atom_struct, D->d_frac, D->d_ph,
               D->d_E,  D->d_K, D->d_Y,     D->d_qtot,        D->d_err,         D->d_K32, D->d_Y32, D->d_Jc};
  for (void* x : p)
    if (x) cudaFree(x);
}

template <typename T>
cudaError_t dense_upload(T** dst, const std::vector<T>& v) {
  QEQ_CUDA_TRY(cudaMalloc((void**)dst, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty()) QEQ_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return cudaSuccess;
}

}  // namespace

extern "C" qeq_status qeq_dense_create(const qeq_plan_desc* desc, void* cuda_stream, qeq_dense* out) {
  if (!desc || !out || desc->n_struct < 1 || !desc->atom_offsets || !desc->cells || !desc->sigma ||
      desc->n_species < 1 || desc->n_species > QEQ_MAX_SPECIES)
    return QEQ_ERR_INVALID;
  *out = nullptr;
  qeq_dense_s* D = new qeq_dense_s();
  D->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&D->device);
  D->n_struct = desc->n_struct;
  D->n_species = desc->n_species;
  if (desc->coulomb_k > 0) D->k_e = desc->coulomb_k;
  if (desc->ewald_tol > 0) D->tol = desc->ewald_tol;
  D->mixed = desc->precision == QEQ_MIXED ? 1 : 0;
  const double xr = erfc_inv(D->tol);                   // erfc(r_c / (sqrt2 omega)) = tol
  const double gq = sqrt(2.0 * log(1.0 / D->tol));      // exp(-g_c^2 omega^2 / 2) = tol
  std::vector<DenseG> gl;
  int64_t e_off = 0, k_off = 0, ph_off = 0;
  std::vector<int> atom_struct;
  auto bad = [&](qeq_status s, const std::string& m) {
    qeq_status r = dfail(D, s, m);
    // the handle is not returned: report through the status only
    delete D;
    return r;
  };
  for (int s = 0; s < D->n_struct; ++s) {
    DenseStructDev T{};
    const double* h = desc->cells + 9 * (size_t)s;
    for (int k = 0; k < 9; ++k) T.h[k] = h[k];
    T.V = fabs(det3(h));
    if (!(T.V > 0.0) || !std::isfinite(T.V)) return bad(QEQ_ERR_INVALID, "singular cell");
    inv3(h, T.hinv);
    const int64_t a0 = desc->atom_offsets[s], a1 = desc->atom_offsets[s + 1];
    if (a1 <= a0) return bad(QEQ_ERR_INVALID, "structure without atoms");
    if (a1 - a0 > QEQ_DENSE_MAX_ATOMS) return bad(QEQ_ERR_CAPACITY, "structure larger than QEQ_DENSE_MAX_ATOMS");
    T.n = (int)(a1 - a0);
    T.atom_off = a0;
    const double* sig = desc->sigma + (size_t)desc->n_species * s;
    int Ss = desc->n_species;
    while (Ss > 1 && !(sig[Ss - 1] > 0.0)) --Ss;
    T.S = Ss;
    double smax = 0.0;
    for (int a = 0; a < Ss; ++a) {
      if (!(sig[a] > 0.0) || !std::isfinite(sig[a])) return bad(QEQ_ERR_NOT_PD, "sigma must be finite and > 0");
      T.sigma[a] = sig[a];
      smax = std::max(smax, sig[a]);
    }
    double wd[3];
    plane_widths(h, T.V, wd);
    // omega >= every gamma; among those, the cheapest: erfc pairs ~ 40 FP64 operations per
    // image, reciprocal ~ 3 per G vector and entry
    const double gmax = sqrt(2.0) * smax;
    double best = 1e300, wbest = gmax;
    for (double w = gmax; w < gmax + 40.0; w *= 1.02) {
      const double rc = sqrt(2.0) * w * xr, gc = gq / w;
      const double nimg = 4.0 / 3.0 * kPiD * rc * rc * rc / T.V + 1.0;
      const double ngv = 0.5 * 4.0 / 3.0 * kPiD * gc * gc * gc * T.V / (8.0 * kPiD * kPiD * kPiD);
      const double cost = 40.0 * nimg + 3.0 * ngv;
      if (cost < best) {
        best = cost;
        wbest = w;
      }
    }
    T.omega = wbest;
    const double rc = sqrt(2.0) * wbest * xr, gc = gq / wbest;
    T.rc2 = rc * rc;
    for (int d = 0; d < 3; ++d) {
      T.ext[d] = rc / wd[d];
      T.M[d] = (int)floor(gc * wd[d] / (2.0 * kPiD)) + 1;
    }
    T.W = (2 * T.M[0] + 1) + (2 * T.M[1] + 1) + (2 * T.M[2] + 1);
    T.g_off = (int)gl.size();
    const double pref = D->k_e * 4.0 * kPiD / T.V;
    for (int m0 = 0; m0 <= T.M[0]; ++m0)
      for (int m1 = (m0 == 0 ? 0 : -T.M[1]); m1 <= T.M[1]; ++m1)
        for (int m2 = ((m0 == 0 && m1 == 0) ? 1 : -T.M[2]); m2 <= T.M[2]; ++m2) {
          double G[3];
          for (int e = 0; e < 3; ++e)
            G[e] = 2.0 * kPiD * (m0 * T.hinv[3 * e] + m1 * T.hinv[3 * e + 1] + m2 * T.hinv[3 * e + 2]);
          const double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
          if (G2 > gc * gc) continue;
          DenseG g{};
          g.m[0] = m0;
          g.m[1] = m1;
          g.m[2] = m2;
          g.f = 2.0 * pref * exp(-0.5 * G2 * wbest * wbest) / G2;
          gl.push_back(g);
        }
    T.ng = (int)gl.size() - T.g_off;
    T.e_off = e_off;
    T.k_off = k_off;
    T.ph_off = ph_off;
    e_off += (int64_t)T.n * T.n;
    k_off += (int64_t)(T.n + 1) * (T.n + 1);
    ph_off += (int64_t)T.n * T.W;
    const int nt = (T.n + kTile - 1) / kTile;
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) D->tiles.push_back(make_int4(s, a, b, 0));
    for (int64_t a = a0; a < a1; ++a) atom_struct.push_back(s);
    D->max_n = std::max(D->max_n, T.n);
    D->hs.push_back(T);
  }
  D->n_atoms = desc->atom_offsets[D->n_struct];
  if ((int64_t)atom_struct.size() != D->n_atoms || desc->atom_offsets[0] != 0)
    return bad(QEQ_ERR_INVALID, "atom offsets must start at 0 and increase");
  D->h_qtot.assign(D->n_struct, 0.0);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dense_upload(&D->d_st, D->hs);
  if (e == cudaSuccess) e = dense_upload(&D->d_g, gl);
  if (e == cudaSuccess) e = dense_upload(&D->d_tiles, D->tiles);
  if (e == cudaSuccess) e = dense_upload(&D->d_atom_struct, atom_struct);
  if (e == cudaSuccess) e = cudaMalloc(&D->d_frac, sizeof(double) * 3 * (size_t)D->n_atoms);
  if (e == cudaSuccess) e = cudaMalloc(&D->d_ph, sizeof(double2) * std::max<int64_t>(1, ph_off));
  if (e == cudaSuccess) e = cudaMalloc(&D->d_E, sizeof(double) * std::max<int64_t>(1, e_off));
  if (D->mixed) {
    if (e == cudaSuccess) e = cudaMalloc(&D->d_Y32, sizeof(float) * std::max<int64_t>(1, e_off));
    if (e == cudaSuccess) e = cudaMalloc(&D->d_K32, sizeof(float) * std::max<int64_t>(1, k_off));
    if (e == cudaSuccess) e = cudaMalloc(&D->d_Jc, sizeof(double) * std::max<int64_t>(1, D->n_atoms));
  } else {
    if (e == cudaSuccess) e = cudaMalloc(&D->d_Y, sizeof(double) * std::max<int64_t>(1, e_off));
    if (e == cudaSuccess) e = cudaMalloc(&D->d_K, sizeof(double) * std::max<int64_t>(1, k_off));
  }
  if (e == cudaSuccess) e = cudaMalloc(&D->d_qtot, sizeof(double) * D->n_struct);
  if (e == cudaSuccess) e = cudaMalloc(&D->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(D->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    dense_free(D);
    delete D;
    return QEQ_ERR_OOM;
  }
  *out = D;
  return QEQ_OK;
}

extern "C" void qeq_dense_destroy(qeq_dense D) {
  if (!D) return;
  dense_free(D);
  delete D;
}

extern "C" const char* qeq_dense_last_error(qeq_dense D) { return D ? D->last_error.c_str() : "null handle"; }

extern "C" qeq_status qeq_dense_assemble(qeq_dense D, const double* d_pos, const int32_t* d_species) {
  if (!D) return QEQ_ERR_INVALID;
  if (!d_pos || !d_species) return dfail(D, QEQ_ERR_INVALID, "null pointer");
  DTRY(cudaSetDevice(D->device));
  const int nb = (int)((D->n_atoms + 255) / 256);
  k_dense_phases<<<nb, 256, 0, D->stream>>>(D->d_st, D->d_atom_struct, D->n_atoms, d_pos, d_species, D->d_frac,
                                            D->d_ph, D->d_err);
  DTRY(cudaGetLastError());
  k_dense_assemble<<<(int)D->tiles.size(), 256, 0, D->stream>>>(D->d_st, D->d_tiles, D->d_frac, d_species, D->d_g,
                                                                 D->d_ph, D->k_e, D->d_E);
  DTRY(cudaGetLastError());
  D->launches += 2;
  D->inverted = false;
  qeq_status st = dense_check(D);
  D->assembled = (st == QEQ_OK);
  return st;
}

extern "C" qeq_status qeq_dense_invert(qeq_dense D, const double* d_J) {
  if (!D) return QEQ_ERR_INVALID;
  if (!d_J) return dfail(D, QEQ_ERR_INVALID, "null pointer");
  if (!D->assembled) return dfail(D, QEQ_ERR_INVALID, "call qeq_dense_assemble first");
  DTRY(cudaSetDevice(D->device));
  if (D->mixed) {
    k_dense_invert<float><<<D->n_struct, 256, 0, D->stream>>>(D->d_st, D->d_E, d_J, D->d_K32, D->d_Y32, D->d_err);
    DTRY(cudaGetLastError());
    DTRY(cudaMemcpyAsync(D->d_Jc, d_J, sizeof(double) * D->n_atoms, cudaMemcpyDeviceToDevice, D->stream));
  } else {
    k_dense_invert<double><<<D->n_struct, 256, 0, D->stream>>>(D->d_st, D->d_E, d_J, D->d_K, D->d_Y, D->d_err);
    DTRY(cudaGetLastError());
  }
  D->launches += 1;
  qeq_status st = dense_check(D);
  D->inverted = (st == QEQ_OK);
  return st;
}

extern "C" qeq_status qeq_dense_charges(qeq_dense D, const double* d_chi, const double* h_qtot, double* d_q,
                                        double* d_mu) {
  if (!D) return QEQ_ERR_INVALID;
  if (!d_chi || !d_q) return dfail(D, QEQ_ERR_INVALID, "null pointer");
  if (!D->inverted) return dfail(D, QEQ_ERR_INVALID, "call qeq_dense_invert first");
  DTRY(cudaSetDevice(D->device));
  for (int s = 0; s < D->n_struct; ++s) D->h_qtot[s] = h_qtot ? h_qtot[s] : 0.0;
  DTRY(cudaMemcpyAsync(D->d_qtot, D->h_qtot.data(), sizeof(double) * D->n_struct, cudaMemcpyHostToDevice,
                       D->stream));
  if (D->mixed)
    k_dense_refine<0><<<D->n_struct, 256, 0, D->stream>>>(D->d_st, D->d_K32, D->d_E, D->d_Jc, d_chi, D->d_qtot,
                                                          nullptr, d_q, d_mu);
  else
    k_dense_apply<0><<<D->n_struct, 256, 0, D->stream>>>(D->d_st, D->d_K, d_chi, D->d_qtot, nullptr, d_q, d_mu);
  DTRY(cudaGetLastError());
  D->launches += 1;
  DTRY(cudaStreamSynchronize(D->stream));  // h_qtot staging is reused by the next call
  return QEQ_OK;
}

extern "C" qeq_status qeq_dense_backward(qeq_dense D, const double* d_q, const double* d_gq, double* d_gchi,
                                         double* d_gJ) {
  if (!D) return QEQ_ERR_INVALID;
  if (!d_gq || !d_gchi || (d_gJ && !d_q)) return dfail(D, QEQ_ERR_INVALID, "null pointer");
  if (!D->inverted) return dfail(D, QEQ_ERR_INVALID, "call qeq_dense_invert first");
  DTRY(cudaSetDevice(D->device));
  if (D->mixed)
    k_dense_refine<1><<<D->n_struct, 256, 0, D->stream>>>(D->d_st, D->d_K32, D->d_E, D->d_Jc, d_gq, nullptr, d_q,
                                                          d_gchi, d_gJ);
  else
    k_dense_apply<1><<<D->n_struct, 256, 0, D->stream>>>(D->d_st, D->d_K, d_gq, nullptr, d_q, d_gchi, d_gJ);
  DTRY(cudaGetLastError());
  D->launches += 1;
  return QEQ_OK;
}

extern "C" qeq_status qeq_dense_matrix(qeq_dense D, int32_t s, int32_t which, double* d_out) {
  if (!D) return QEQ_ERR_INVALID;
  if (s < 0 || s >= D->n_struct || !d_out || (which != 0 && which != 1))
    return dfail(D, QEQ_ERR_INVALID, "bad structure index, matrix selector or pointer");
  if ((which == 0 && !D->assembled) || (which == 1 && !D->inverted))
    return dfail(D, QEQ_ERR_INVALID, "matrix not computed yet");
  DTRY(cudaSetDevice(D->device));
  const DenseStructDev& T = D->hs[s];
  const int64_t cnt = which == 0 ? (int64_t)T.n * T.n : (int64_t)(T.n + 1) * (T.n + 1);
  if (which == 1 && D->mixed) {  // the FP32 inverse, widened
    k_f2d<<<(int)((cnt + 255) / 256), 256, 0, D->stream>>>(D->d_K32 + T.k_off, cnt, d_out);
    DTRY(cudaGetLastError());
    return QEQ_OK;
  }
  const double* src = which == 0 ? D->d_E + T.e_off : D->d_K + T.k_off;
  DTRY(cudaMemcpyAsync(d_out, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, D->stream));
  return QEQ_OK;
}

extern "C" qeq_status qeq_dense_query(qeq_dense D, int32_t s, double* h_omega, int32_t* h_ng, int64_t* h_launches) {
  if (!D || s < 0 || s >= D->n_struct) return QEQ_ERR_INVALID;
  if (h_omega) *h_omega = D->hs[s].omega;
  if (h_ng) *h_ng = D->hs[s].ng;
  if (h_launches) *h_launches = D->launches;
  return QEQ_OK;
}
