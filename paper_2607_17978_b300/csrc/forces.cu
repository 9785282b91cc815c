// Electrostatic forces of the force trick and the element-resolved potentials of the
// electrostatic embedding.
//
// Force trick (SI "Fourth-Generation HDNNPs and Charge Equilibration", eq. 4g_force_trick):
// with lambda solving (A + J)^T lambda = -dE/dq (a second qeq_solve with chi := dE/dq and
// q_tot = 0), the electrostatic part of the force on atom k is
//
//   F_k = -dE_elec/dR_k|_q - lambda^T (dA/dR_k) q = -(q_k + lambda_k) g_q(k) - q_k g_lambda(k)
//
// where g_x(k) = d/dR_k sum_j E_kj x_j is the gradient, at atom k, of the potential of the
// charges x (E symmetric; the self and width-correction terms do not depend on positions).
// g_x comes from the same plane-wave machinery as the matvec (Sec. 2.4 "Electrostatics
// Solvers": the potential meshes are differentiated through the B-spline interpolation)
// plus the derivative of the screened real-space pair term (SI "Ewald Summation").
//
// Electrostatic embedding (Sec. 2.2, ee4G, Fig. 1c): Gamma[i, z] = sum_{j of element z}
// E_ij q_j, one FP64 matvec of the charges of each element.
#include <math.h>

#include <type_traits>

#include "neighbors.cuh"
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

// g_x at every atom (sorted order), one warp per atom: the mesh part differentiates the
// B-spline weights (dM_p(t)/dt = M_{p-1}(t) - M_{p-1}(t - 1)) and maps mesh to Cartesian
// derivatives with K_d h^{-1}; the real-space part walks the neighbouring bins.
// T: the potential mesh's precision (the plan's: FP32 meshes and weights in QEQ_MIXED); the
// stencil sums of each lane run in T, the sums over lanes and the pair term in FP64.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_force_grad(const StructDev* __restrict__ st,
                                                    const int* __restrict__ sorted_struct, int64_t n,
                                                    const int* __restrict__ base, const T* __restrict__ wts,
                                                    const int* __restrict__ spec, const double* __restrict__ posc,
                                                    const float4* __restrict__ posc32,
                                                    const int* __restrict__ bin_start, const double* __restrict__ x,
                                                    const typename C2<T>::t* __restrict__ mesh, double k_e,
                                                    double* __restrict__ g0, double* __restrict__ g1,
                                                    double* __restrict__ g2) {
  using V = typename C2<T>::t;
  __shared__ NbrWarpSmem ws[8];
  __shared__ T dw[8][3][QEQ_MAXP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a = (int64_t)blockIdx.x * 8 + w;
  if (a >= n) return;  // whole warp
  const StructDev& S = st[sorted_struct[a]];
  const int sp = spec[a];
  const int bs = base[a];
  const int f[3] = {bs & 1023, (bs >> 10) & 1023, (bs >> 20) & 1023};
  const T* wt = wts + (size_t)a * 3 * QEQ_MAXP;
  if (lane < 3) {  // derivative weights of direction d = lane
    const int d = lane;
    double u = posc[3 * a] * S.hinv[d] + posc[3 * a + 1] * S.hinv[3 + d] + posc[3 * a + 2] * S.hinv[6 + d];
    u -= floor(u);
    // the offset inside the stencil's base cell, as in the weights (the round trip
    // through Cartesian coordinates moves it by rounding only; keep it in [0, 1))
    double xw = u * S.K[d] - f[d];
    if (xw > 0.5 * S.K[d]) xw -= S.K[d];
    xw = fmin(fmax(xw, 0.0), 1.0 - 1e-16);
    double m1[QEQ_MAXP];
    bspline_weights(xw, P - 1, m1);  // M_{p-1}(xw + j), j < p - 1
#pragma unroll
    for (int j = 0; j < P; ++j) dw[w][d][j] = (T)(((j < P - 1) ? m1[j] : 0.0) - ((j >= 1) ? m1[j - 1] : 0.0));
  }
  __syncwarp();
  // mesh part: lanes own 8 z x 4 rows of the P^3 stencil
  const V* mg = mesh + S.mesh_off + (int64_t)(sp >> 1) * S.Mp;
  const int part = sp & 1;
  T D0t = (T)0, D1t = (T)0, D2t = (T)0;
  const int jz = lane & 7, rsub = lane >> 3;
  if (jz < P) {
    int kz = f[2] - (P - 1) + jz;
    if (kz < 0) kz += S.K[2];
    const T wz = wt[2 * QEQ_MAXP + P - 1 - jz], dz = dw[w][2][P - 1 - jz];
    for (int r = rsub; r < P * P; r += 4) {
      const int jx = r / P, jy = r - (r / P) * P;
      int kx = f[0] - (P - 1) + jx;
      if (kx < 0) kx += S.K[0];
      int ky = f[1] - (P - 1) + jy;
      if (ky < 0) ky += S.K[1];
      const V v2 = mg[((int64_t)kx * S.K[1] + ky) * S.P[2] + kz];
      const T v = part ? v2.y : v2.x;
      const T wx = wt[P - 1 - jx], wy = wt[QEQ_MAXP + P - 1 - jy];
      const T dx = dw[w][0][P - 1 - jx], dy = dw[w][1][P - 1 - jy];
      D0t += dx * wy * wz * v;
      D1t += wx * dy * wz * v;
      D2t += wx * wy * dz * v;
    }
  }
  double D0 = (double)D0t, D1 = (double)D1t, D2 = (double)D2t;
  // real-space part: d/dR_a of sum_j x_j v(|R_j' - R_a|) = sum_j x_j v'(r) (R_a - R_j')/r
  double r0 = 0.0, r1 = 0.0, r2s = 0.0;
  if (S.any_narrow && S.narrow[sp]) {
    const int bb[3] = {f[0] / QEQ_BIN, f[1] / QEQ_BIN, f[2] / QEQ_BIN};
    const double ra0 = posc[3 * a], ra1 = posc[3 * a + 1], ra2 = posc[3 * a + 2];
    const double rc2 = S.r_cut * S.r_cut;
    const uint32_t mask = S.narrow[sp];
    const double two_over_sqrtpi = 1.12837916709551257390;
    // FP32 distance prefilter with a margin above FP32 position rounding (as the pair
    // list's walk): only candidates that may lie within r_cut get the FP64 test
    const float4 pa = posc32[a];
    const double ext = norm3d(S.h[0], S.h[1], S.h[2]) + norm3d(S.h[3], S.h[4], S.h[5]) + norm3d(S.h[6], S.h[7], S.h[8]);
    const float out2 = (float)((S.r_cut + 1e-3 + 1e-6 * ext) * (S.r_cut + 1e-3 + 1e-6 * ext));
    warp_neighbour_walk(S, bb, S.rs_range, bin_start, ws[w],
                        [&](bool valid, int t, const double* sh, const float* sh32, bool zero, int) {
      if (!valid || !((mask >> spec[t]) & 1u) || (zero && t == a)) return;
      const float4 pt = posc32[t];
      const float fx = pt.x + sh32[0] - pa.x, fy = pt.y + sh32[1] - pa.y, fz = pt.z + sh32[2] - pa.z;
      if (fx * fx + fy * fy + fz * fz > out2) return;
      const double dx = posc[3 * t] + sh[0] - ra0, dy = posc[3 * t + 1] + sh[1] - ra1,
                   dz = posc[3 * t + 2] + sh[2] - ra2;
      const double d2 = dx * dx + dy * dy + dz * dz;
      if (d2 >= rc2 || d2 < 1e-24) return;  // coincident atoms: no force between them
      const double r = sqrt(d2);
      const int kk = sp * QEQ_MAX_SPECIES + spec[t];
      const double A = S.inv_sw[kk], B = S.inv_sg[kk];
      const double dv = k_e * ((-A * exp(-A * A * d2) + B * exp(-B * B * d2)) * two_over_sqrtpi / r -
                               (erfc(A * r) - erfc(B * r)) / d2);
      const double c = -x[t] * dv / r;
      r0 += c * dx;
      r1 += c * dy;
      r2s += c * dz;
    });
  }
  for (int o = 16; o > 0; o >>= 1) {
    D0 += __shfl_xor_sync(0xffffffffu, D0, o);
    D1 += __shfl_xor_sync(0xffffffffu, D1, o);
    D2 += __shfl_xor_sync(0xffffffffu, D2, o);
    r0 += __shfl_xor_sync(0xffffffffu, r0, o);
    r1 += __shfl_xor_sync(0xffffffffu, r1, o);
    r2s += __shfl_xor_sync(0xffffffffu, r2s, o);
  }
  if (lane == 0) {
    // d/dR_c = sum_d d/dX_d K_d dX... with X_d = K_d (R h^{-1})_d
    const double E0 = D0 * S.K[0], E1 = D1 * S.K[1], E2 = D2 * S.K[2];
    g0[a] = E0 * S.hinv[0] + E1 * S.hinv[1] + E2 * S.hinv[2] + r0;
    g1[a] = E0 * S.hinv[3] + E1 * S.hinv[4] + E2 * S.hinv[5] + r1;
    g2[a] = E0 * S.hinv[6] + E1 * S.hinv[7] + E2 * S.hinv[8] + r2s;
  }
}

// F[perm a] = -(q_a + lambda_a) g_q(a) - q_a g_lambda(a); gradients component-major
// (gq[c][a]); lambda == NULL: no lambda term
__global__ void k_force_assemble(const int* __restrict__ perm, int64_t n, const double* __restrict__ q,
                                 const double* __restrict__ lam, const double* __restrict__ gq0,
                                 const double* __restrict__ gq1, const double* __restrict__ gq2,
                                 const double* __restrict__ gl0, const double* __restrict__ gl1,
                                 const double* __restrict__ gl2, double* __restrict__ F) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const double qa = q[a];
  const int64_t i = perm[a];
  double f0 = -qa * gq0[a], f1 = -qa * gq1[a], f2 = -qa * gq2[a];
  if (lam) {
    const double la = lam[a];
    f0 -= la * gq0[a] + qa * gl0[a];
    f1 -= la * gq1[a] + qa * gl1[a];
    f2 -= la * gq2[a] + qa * gl2[a];
  }
  F[3 * i] = f0;
  F[3 * i + 1] = f1;
  F[3 * i + 2] = f2;
}

__global__ void k_sort_in_f(const int* __restrict__ perm, int64_t n, const double* __restrict__ src,
                            double* __restrict__ dst) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) dst[a] = src[perm[a]];
}

// x_a = q_a for atoms of element z, else 0 (sorted order)
__global__ void k_mask_species(const int* __restrict__ spec, int64_t n, int z, const double* __restrict__ q,
                               double* __restrict__ xz) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) xz[a] = (spec[a] == z) ? q[a] : 0.0;
}

// Gamma[perm a][z] = y_a
__global__ void k_scatter_column(const int* __restrict__ perm, int64_t n, const double* __restrict__ y, int z,
                                 int nz, double* __restrict__ G) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) G[(int64_t)perm[a] * nz + z] = y[a];
}

// ---------------------------------------------------------------- strain derivative
// Real-space part of d/d eps_ab [w^T E q], per atom a (one warp):
//   w_a sum_{t,n} q_t v'(r) d_a d_b / r,  d = R_t + n - R_a
// over the same narrow pairs as the matvec (images of a itself included: their
// separation is strained too).  Components xx yy zz xy xz yz to o0..o5, sorted order.
__global__ void __launch_bounds__(256) k_virial_real(const StructDev* __restrict__ st,
                                                     const int* __restrict__ sorted_struct, int64_t n,
                                                     const int* __restrict__ base, const int* __restrict__ spec,
                                                     const double* __restrict__ posc, const float4* __restrict__ posc32,
                                                     const int* __restrict__ bin_start, const double* __restrict__ w,
                                                     const double* __restrict__ q, double k_e,
                                                     double* __restrict__ o0, double* __restrict__ o1,
                                                     double* __restrict__ o2, double* __restrict__ o3,
                                                     double* __restrict__ o4, double* __restrict__ o5) {
  __shared__ NbrWarpSmem ws[8];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t a = (int64_t)blockIdx.x * 8 + wp;
  if (a >= n) return;  // whole warp
  const StructDev& S = st[sorted_struct[a]];
  const int sp = spec[a];
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (S.any_narrow && S.narrow[sp] && w[a] != 0.0) {
    const int bs = base[a];
    const int bb[3] = {(bs & 1023) / QEQ_BIN, ((bs >> 10) & 1023) / QEQ_BIN, ((bs >> 20) & 1023) / QEQ_BIN};
    const double ra0 = posc[3 * a], ra1 = posc[3 * a + 1], ra2 = posc[3 * a + 2];
    const double rc2 = S.r_cut * S.r_cut;
    const uint32_t mask = S.narrow[sp];
    const double two_over_sqrtpi = 1.12837916709551257390;
    // FP32 distance prefilter with a margin above FP32 position rounding (as the pair
    // list's walk): only candidates that may lie within r_cut get the FP64 test
    const float4 pa = posc32[a];
    const double ext = norm3d(S.h[0], S.h[1], S.h[2]) + norm3d(S.h[3], S.h[4], S.h[5]) + norm3d(S.h[6], S.h[7], S.h[8]);
    const float out2 = (float)((S.r_cut + 1e-3 + 1e-6 * ext) * (S.r_cut + 1e-3 + 1e-6 * ext));
    warp_neighbour_walk(S, bb, S.rs_range, bin_start, ws[wp],
                        [&](bool valid, int t, const double* sh, const float* sh32, bool zero, int) {
      if (!valid || !((mask >> spec[t]) & 1u) || (zero && t == a)) return;
      const float4 pt = posc32[t];
      const float fx = pt.x + sh32[0] - pa.x, fy = pt.y + sh32[1] - pa.y, fz = pt.z + sh32[2] - pa.z;
      if (fx * fx + fy * fy + fz * fz > out2) return;
      const double dx = posc[3 * t] + sh[0] - ra0, dy = posc[3 * t + 1] + sh[1] - ra1,
                   dz = posc[3 * t + 2] + sh[2] - ra2;
      const double d2 = dx * dx + dy * dy + dz * dz;
      if (d2 >= rc2 || d2 < 1e-24) return;
      const double r = sqrt(d2);
      const int kk = sp * QEQ_MAX_SPECIES + spec[t];
      const double A = S.inv_sw[kk], B = S.inv_sg[kk];
      const double dv = k_e * ((-A * exp(-A * A * d2) + B * exp(-B * B * d2)) * two_over_sqrtpi / r -
                               (erfc(A * r) - erfc(B * r)) / d2);
      const double c = q[t] * dv / r;
      v[0] += c * dx * dx;
      v[1] += c * dy * dy;
      v[2] += c * dz * dz;
      v[3] += c * dx * dy;
      v[4] += c * dx * dz;
      v[5] += c * dy * dz;
    });
  }
#pragma unroll
  for (int k = 0; k < 6; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0) {
    const double wa = w[a];
    o0[a] = wa * v[0];
    o1[a] = wa * v[1];
    o2[a] = wa * v[2];
    o3[a] = wa * v[3];
    o4[a] = wa * v[4];
    o5[a] = wa * v[5];
  }
}

// per-thread values summed over the block in a fixed order (shuffle tree per warp, warps
// in order); valid in thread 0.  red: blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum_fixed(double a, double* red) {
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
  __syncthreads();
  return tot;
}

// the 7 x-pass sums of every unit of structure s (block s), in unit order
__global__ void __launch_bounds__(256) k_virial_units(const int* __restrict__ xoff, int nsubx,
                                                      const double* __restrict__ units, double* __restrict__ out) {
  __shared__ double red[8];
  const int s = blockIdx.x;
  const int first = xoff[s] * nsubx, count = (xoff[s + 1] - xoff[s]) * nsubx;
  for (int k = 0; k < 7; ++k) {
    const double t = ordered_block_sum(units, first, count, 8, k, red);
    if (threadIdx.x == 0) out[8 * s + k] = t;
  }
}

// D[9 s + 3 a + b] = fa R_A + fb R_B (reciprocal, R = -delta sum E + the G_a G_b sums)
//   + sum over the structure's atoms of the real-space parts
//   + delta_ab sum_st wsum_s corr_st qsum_t (the G = 0 width term ~ 1/V).
// One CTA per reduction chunk: the chunk's 6 real-space sums and per-species sums of w
// and q go to part[chunk * kStressPart ..]; the structure's last chunk to finish (counter)
// combines the partials in chunk order and writes D.
constexpr int kStressPart = 6 + 2 * QEQ_MAX_SPECIES;

__global__ void __launch_bounds__(256) k_stress_finish(const Chunk* __restrict__ chunks,
                                                       const StructDev* __restrict__ st,
                                                       const double* __restrict__ rA, const double* __restrict__ rB,
                                                       double fa, double fb, const double* __restrict__ o0,
                                                       const double* __restrict__ o1, const double* __restrict__ o2,
                                                       const double* __restrict__ o3, const double* __restrict__ o4,
                                                       const double* __restrict__ o5, const int* __restrict__ spec,
                                                       const double* __restrict__ w, const double* __restrict__ q,
                                                       double* __restrict__ part, int* __restrict__ counter,
                                                       double* __restrict__ D) {
  __shared__ double red[8];
  __shared__ bool last;
  const Chunk ch = chunks[blockIdx.x];
  const StructDev& S = st[ch.s];
  const double* parts[6] = {o0, o1, o2, o3, o4, o5};
  double v[kStressPart];
#pragma unroll
  for (int k = 0; k < kStressPart; ++k) v[k] = 0.0;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] += parts[k][a];
    const int z = spec[a];
#pragma unroll
    for (int t = 0; t < QEQ_MAX_SPECIES; ++t)
      if (t == z) {
        v[6 + t] += w[a];
        v[6 + QEQ_MAX_SPECIES + t] += q[a];
      }
  }
#pragma unroll
  for (int k = 0; k < kStressPart; ++k) {
    const double tot = block_sum_fixed(v[k], red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * kStressPart + k] = tot;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const int prev = atomicAdd(counter + ch.s, 1);
    last = (prev == ch.count - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x != 0) return;
  double tot[kStressPart];
  for (int k = 0; k < kStressPart; ++k) tot[k] = 0.0;
  for (int c = 0; c < ch.count; ++c)  // chunk order: deterministic
    for (int k = 0; k < kStressPart; ++k) tot[k] += ((volatile double*)part)[(size_t)(ch.first + c) * kStressPart + k];
  counter[ch.s] = 0;
  double corr = 0.0;
  for (int z = 0; z < S.S; ++z)
    for (int t = 0; t < S.S; ++t) corr += tot[6 + z] * S.corr[z * QEQ_MAX_SPECIES + t] * tot[6 + QEQ_MAX_SPECIES + t];
  double R[7];
  for (int k = 0; k < 7; ++k) R[k] = fa * rA[8 * ch.s + k] + (rB ? fb * rB[8 * ch.s + k] : 0.0);
  const double diag = corr - R[0];
  double* o = D + 9 * (size_t)ch.s;
  o[0] = R[1] + tot[0] + diag;
  o[4] = R[2] + tot[1] + diag;
  o[8] = R[3] + tot[2] + diag;
  o[1] = o[3] = R[4] + tot[3];
  o[2] = o[6] = R[5] + tot[4];
  o[5] = o[7] = R[6] + tot[5];
}

// w = q/2 + lambda (lambda sorted in w on entry, or NULL: w = q/2); x = w + q
__global__ void k_stress_vectors(int64_t n, const double* __restrict__ q, int have_lambda, double* __restrict__ w,
                                 double* __restrict__ x) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const double wa = 0.5 * q[a] + (have_lambda ? w[a] : 0.0);
  w[a] = wa;
  x[a] = wa + q[a];
}

__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] - b[i];
}

template <typename T, int P>
cudaError_t launch_force_grad(qeq_plan_s* Pl, const double* x, double* const g[3]) {
  count_launch(Pl);
  const int nbw = (int)((Pl->n_atoms + 7) / 8);  // one warp per atom
  const T* wts = std::is_same<T, float>::value ? (const T*)(const void*)Pl->d_wts32 : (const T*)(const void*)Pl->d_wts;
  const typename C2<T>::t* mesh = reinterpret_cast<const typename C2<T>::t*>(Pl->d_mesh);
  k_force_grad<T, P><<<nbw, 256, 0, Pl->stream>>>(Pl->d_st, Pl->d_key, Pl->n_atoms, Pl->d_base, wts, Pl->d_spec,
                                                   Pl->d_posc, Pl->d_posc32, Pl->d_bin_start, x, mesh,
                                                   Pl->desc.coulomb_k, g[0], g[1], g[2]);
  return cudaGetLastError();
}

// the potential meshes in the plan's precision (FP32 in QEQ_MIXED: the narrow FP64 pipe makes
// FP64 passes 16-18x slower; FP32 meshes carry ~3e-7 of the potentials' size), then the gradient
cudaError_t force_grad(qeq_plan_s* P, const double* x, double* const g[3]) {
  if (P->precision == QEQ_MIXED) {
    QEQ_CUDA_TRY(launch_mesh_potential32(P, x));
    if (P->max_p == 4) return launch_force_grad<float, 4>(P, x, g);
    if (P->max_p == 6) return launch_force_grad<float, 6>(P, x, g);
    return launch_force_grad<float, 8>(P, x, g);
  }
  QEQ_CUDA_TRY(launch_mesh_potential(P, x));
  if (P->max_p == 4) return launch_force_grad<double, 4>(P, x, g);
  if (P->max_p == 6) return launch_force_grad<double, 6>(P, x, g);
  return launch_force_grad<double, 8>(P, x, g);
}

}  // namespace

// g_q (and g_lambda) at every atom, then F in input order.  q, lambda: input order.
cudaError_t launch_forces(qeq_plan_s* P, const double* q, const double* lambda, double* F) {
  cudaStream_t s = P->stream;
  const int64_t n = P->n_atoms;
  const int nb = (int)((n + 255) / 256);
  count_launch(P, lambda ? 2 : 1);
  k_sort_in_f<<<nb, 256, 0, s>>>(P->d_perm, n, q, P->d_q);
  if (lambda) k_sort_in_f<<<nb, 256, 0, s>>>(P->d_perm, n, lambda, P->d_z);
  QEQ_CUDA_TRY(cudaGetLastError());
  // gradients in the solver's work vectors (component-major): nothing is allocated
  double* const gq[3] = {P->d_r, P->d_p, P->d_Ap};
  double* const gl[3] = {P->d_x, P->d_q1, P->d_r1};
  QEQ_CUDA_TRY(force_grad(P, P->d_q, gq));
  if (lambda) QEQ_CUDA_TRY(force_grad(P, P->d_z, gl));
  count_launch(P);
  k_force_assemble<<<nb, 256, 0, s>>>(P->d_perm, n, P->d_q, lambda ? P->d_z : nullptr, gq[0], gq[1], gq[2], gl[0],
                                      gl[1], gl[2], F);
  return cudaGetLastError();
}

// Gamma[i][z] = (E q_z)_i with q_z = q on the atoms of element z, one FP64 matvec per
// element (no hardness).  q: input order; Gamma: n x n_species, input order.
cudaError_t launch_embedding(qeq_plan_s* P, const double* q, double* Gamma) {
  cudaStream_t s = P->stream;
  const int64_t n = P->n_atoms;
  const int nb = (int)((n + 255) / 256);
  const int nz = P->desc.n_species;
  count_launch(P);
  k_sort_in_f<<<nb, 256, 0, s>>>(P->d_perm, n, q, P->d_q);
  QEQ_CUDA_TRY(cudaGetLastError());
  for (int z = 0; z < nz; ++z) {
    count_launch(P);
    k_mask_species<<<nb, 256, 0, s>>>(P->d_spec, n, z, P->d_q, P->d_x);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(launch_matvec(P, QEQ_FP64, P->d_x, P->d_Ap, 0, 0, 0, nullptr));
    count_launch(P);
    k_scatter_column<<<nb, 256, 0, s>>>(P->d_perm, n, P->d_Ap, z, nz, Gamma);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// Strain derivative of W = w^T E q, w = q/2 + lambda, per structure.  Reciprocal part by
// polarisation, W = 1/4 [Q(w + q) - Q(w - q)] with Q(x) = x^T E_rec x (one mesh pass per
// vector; without lambda W = Q(q)/2 needs one); real-space part per atom; G = 0 width
// term from species sums.  Work vectors: q in d_q, w in d_z, the mesh vector in d_chi
// (scratch once the atoms are prepared), real-space parts in d_r d_p d_Ap d_x d_q1 d_r1,
// per-structure reciprocal sums in d_part.
cudaError_t launch_stress(qeq_plan_s* P, const double* q, const double* lambda, double* D) {
  cudaStream_t s = P->stream;
  const int64_t n = P->n_atoms;
  const int nb = (int)((n + 255) / 256);
  const int ns = P->n_struct;
  count_launch(P, lambda ? 3 : 2);
  k_sort_in_f<<<nb, 256, 0, s>>>(P->d_perm, n, q, P->d_q);
  if (lambda) k_sort_in_f<<<nb, 256, 0, s>>>(P->d_perm, n, lambda, P->d_z);
  k_stress_vectors<<<nb, 256, 0, s>>>(n, P->d_q, lambda ? 1 : 0, P->d_z, P->d_chi);
  QEQ_CUDA_TRY(cudaGetLastError());
  count_launch(P);
  k_virial_real<<<(int)((n + 7) / 8), 256, 0, s>>>(P->d_st, P->d_key, n, P->d_base, P->d_spec, P->d_posc,
                                                    P->d_posc32, P->d_bin_start, P->d_z, P->d_q, P->desc.coulomb_k, P->d_r,
                                                    P->d_p, P->d_Ap, P->d_x, P->d_q1, P->d_r1);
  QEQ_CUDA_TRY(cudaGetLastError());
  double* rA = P->d_part;
  double* rB = P->d_part + 8 * (size_t)ns;
  const double* units = reinterpret_cast<const double*>(P->d_mesh2);
  int nsubx = 1;
  // lambda: Q(w + q) then Q(w - q); no lambda: Q(q) (w + q = 3q/2 would do as well)
  QEQ_CUDA_TRY(launch_mesh_virial(P, lambda ? P->d_chi : P->d_q, &nsubx));
  count_launch(P);
  k_virial_units<<<ns, 256, 0, s>>>(P->d_xitem_off, nsubx, units, rA);
  QEQ_CUDA_TRY(cudaGetLastError());
  if (lambda) {
    count_launch(P);
    k_sub<<<nb, 256, 0, s>>>(n, P->d_z, P->d_q, P->d_chi);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(launch_mesh_virial(P, P->d_chi, &nsubx));
    count_launch(P);
    k_virial_units<<<ns, 256, 0, s>>>(P->d_xitem_off, nsubx, units, rB);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  count_launch(P);
  k_stress_finish<<<P->n_chunks, 256, 0, s>>>(P->d_chunks, P->d_st, rA, lambda ? rB : nullptr, lambda ? 0.25 : 0.5,
                                              -0.25, P->d_r, P->d_p, P->d_Ap, P->d_x, P->d_q1, P->d_r1, P->d_spec,
                                              P->d_z, P->d_q, P->d_stress_part, P->d_counter + 3 * ns, D);
  return cudaGetLastError();
}
