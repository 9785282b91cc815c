// Per-solve atom preparation: wrap and bin the atoms on the mesh, counting-sort
// them by bin (deterministic order inside a bin), gather per-atom data in the
// sorted order with the B-spline weights of the particle-mesh interpolation
// (SI "Particle-Particle-Particle-Mesh Method"; smooth PME B-splines), and build
// the real-space pair list of the Ewald split (SI "Ewald Summation").
#include <math.h>

#include "neighbors.cuh"
#include "qeq_internal.cuh"

namespace {

__device__ __forceinline__ void atomic_or_err(int* err, int bit) { atomicOr(err, bit); }

// fractional coordinates u = r h^{-1}, wrapped to [0, 1)
__device__ __forceinline__ void frac_wrap(const StructDev& S, const double* r, double* u) {
  for (int d = 0; d < 3; ++d) {
    double v = r[0] * S.hinv[d] + r[1] * S.hinv[3 + d] + r[2] * S.hinv[6 + d];
    v -= floor(v);
    if (v >= 1.0) v = 0.0;  // -tiny -> 1.0 after floor
    u[d] = v;
  }
}

__global__ void k_bin_atoms(const StructDev* __restrict__ st, const int* __restrict__ atom_struct, int64_t n,
                            const double* __restrict__ pos, const int32_t* __restrict__ species,
                            const double* __restrict__ chi, const double* __restrict__ J, int* __restrict__ key,
                            int* __restrict__ bin_count, int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const StructDev& S = st[atom_struct[i]];
  double r[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  int bad = 0;
  if (!isfinite(r[0]) || !isfinite(r[1]) || !isfinite(r[2])) bad |= ERRBIT_NONFINITE;
  if (chi && !isfinite(chi[i])) bad |= ERRBIT_NONFINITE;
  if (J && !isfinite(J[i])) bad |= ERRBIT_NONFINITE;
  int sp = species[i];
  if (sp < 0 || sp >= S.S) bad |= ERRBIT_SPECIES;
  if (J && !(J[i] > 0.0)) bad |= ERRBIT_J;
  if (bad) {
    atomic_or_err(err, bad);
    r[0] = r[1] = r[2] = 0.0;
  }
  double u[3];
  frac_wrap(S, r, u);
  int b[3];
  for (int d = 0; d < 3; ++d) {
    int f = (int)floor(u[d] * S.K[d]);
    if (f >= S.K[d]) f = S.K[d] - 1;
    if (f < 0) f = 0;
    b[d] = f / QEQ_BIN;
  }
  int g = S.bin_off + (b[0] * S.nb[1] + b[1]) * S.nb[2] + b[2];
  key[i] = g;
  atomicAdd(&bin_count[g], 1);
}

// ---------------------------------------------------------------- exclusive scan
template <typename OutT>
__global__ void k_scan_blocks(const int* __restrict__ in, int64_t n, OutT* __restrict__ out,
                              OutT* __restrict__ block_sums) {
  __shared__ OutT warp_tot[32];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  OutT v = (i < n) ? (OutT)in[i] : (OutT)0;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  OutT x = v;
  for (int o = 1; o < 32; o <<= 1) {
    OutT y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    OutT t = (lane < nw) ? warp_tot[lane] : (OutT)0;
    for (int o = 1; o < 32; o <<= 1) {
      OutT y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;
  }
  __syncthreads();
  OutT pre = (w > 0) ? warp_tot[w - 1] : (OutT)0;
  if (i < n) out[i] = pre + x - v;  // exclusive
  if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = pre + x;
}

template <typename OutT>
__global__ void k_scan_sums(OutT* __restrict__ sums, int nblocks, OutT* __restrict__ total) {
  // single thread: the number of blocks is small (n / 1024)
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  OutT acc = 0;
  for (int b = 0; b < nblocks; ++b) {
    OutT t = sums[b];
    sums[b] = acc;
    acc += t;
  }
  *total = acc;
}

template <typename OutT>
__global__ void k_scan_add(OutT* __restrict__ out, int64_t n, const OutT* __restrict__ sums) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
}

// out[0..n) = exclusive scan of in, out[n] = total.  tmp holds ceil(n/1024) OutT.
template <typename OutT>
cudaError_t exclusive_scan(const int* in, int64_t n, OutT* out, OutT* tmp, cudaStream_t s) {
  int nb = (int)((n + 1023) / 1024);
  if (nb == 0) {
    QEQ_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(OutT), s));
    return cudaSuccess;
  }
  k_scan_blocks<OutT><<<nb, 1024, 0, s>>>(in, n, out, tmp);
  k_scan_sums<OutT><<<1, 32, 0, s>>>(tmp, nb, out + n);
  k_scan_add<OutT><<<nb, 1024, 0, s>>>(out, n, tmp);
  return cudaGetLastError();
}

__global__ void k_scatter(const int* __restrict__ key, int64_t n, const int* __restrict__ bin_start,
                          int* __restrict__ bin_fill, int* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int g = key[i];
  int slot = bin_start[g] + atomicAdd(&bin_fill[g], 1);
  perm[slot] = (int)i;
}

// insertion sort inside each bin: the sorted order does not depend on atomics
__global__ void k_sort_bins(const int* __restrict__ bin_start, int nbins, int* __restrict__ perm) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nbins) return;
  int a = bin_start[g], b = bin_start[g + 1];
  for (int i = a + 1; i < b; ++i) {
    int v = perm[i];
    int j = i - 1;
    while (j >= a && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

__global__ void k_gather_sorted(const StructDev* __restrict__ st, const int* __restrict__ atom_struct,
                                const int* __restrict__ perm, int64_t n, const double* __restrict__ pos,
                                const int32_t* __restrict__ species, const double* __restrict__ chi,
                                const double* __restrict__ J, int maxp, int* __restrict__ base,
                                double* __restrict__ wts, float* __restrict__ wts32, int* __restrict__ spec,
                                double* __restrict__ Js, double* __restrict__ chis, double* __restrict__ dinv,
                                double* __restrict__ posc, float4* __restrict__ posc32) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  int i = perm[a];
  const StructDev& S = st[atom_struct[i]];
  double r[3] = {pos[3 * (int64_t)i], pos[3 * (int64_t)i + 1], pos[3 * (int64_t)i + 2]};
  int sp = species[i];
  double Ji = J ? J[i] : 0.0, ci = chi ? chi[i] : 0.0;
  if (!isfinite(r[0]) || !isfinite(r[1]) || !isfinite(r[2])) r[0] = r[1] = r[2] = 0.0;
  if (sp < 0 || sp >= S.S) sp = 0;
  double u[3];
  frac_wrap(S, r, u);
  int f[3];
  for (int d = 0; d < 3; ++d) {
    double x = u[d] * S.K[d];
    int fi = (int)floor(x);
    if (fi >= S.K[d]) fi = S.K[d] - 1;
    if (fi < 0) fi = 0;
    f[d] = fi;
    double w = x - fi;
    if (w < 0.0) w = 0.0;
    if (w >= 1.0) w = 1.0 - 1e-16;
    double m[QEQ_MAXP];
    bspline_weights(w, S.p, m);
    for (int j = 0; j < S.p; ++j) {
      wts[(size_t)a * 3 * maxp + d * maxp + j] = m[j];
      wts32[(size_t)a * 3 * maxp + d * maxp + j] = (float)m[j];
    }
  }
  base[a] = f[0] | (f[1] << 10) | (f[2] << 20);
  spec[a] = sp;
  Js[a] = Ji;
  chis[a] = ci;
  dinv[a] = 1.0 / (fmax(Ji, 0.0) + S.diag_s[sp]);
  double c[3];
  for (int d = 0; d < 3; ++d) {
    c[d] = u[0] * S.h[d] + u[1] * S.h[3 + d] + u[2] * S.h[6 + d];
    posc[3 * a + d] = c[d];
  }
  posc32[a] = make_float4((float)c[0], (float)c[1], (float)c[2], 0.f);
}

// ---------------------------------------------------------------- real-space pairs
// Real-space pairs of atom a (one warp per atom): every (j, image) with
// |r_j + n h - r_a| < r_cut whose species pair has a real-space term; count
// (FILL == 0) or write the CSR row (FILL == 1) in the walk's candidate order.
// Distances are tested in FP32 with a margin well above FP32 position rounding;
// only candidates inside the margin band are decided in FP64, so the cutoff is
// the exact FP64 test.  FILL first records (column, image) per pair, then the
// warp computes the FP64 values over its finished row with every lane busy.
template <int FILL>
__global__ void __launch_bounds__(256) k_pairs(const StructDev* __restrict__ st, const int* __restrict__ bin_start,
                                               int64_t n, const int* __restrict__ base, const int* __restrict__ spec,
                                               const double* __restrict__ posc, const float4* __restrict__ posc32,
                                               int* __restrict__ row_cnt, const int64_t* __restrict__ row, int64_t cap,
                                               int* __restrict__ col, double* __restrict__ val64,
                                               float* __restrict__ val32, int* __restrict__ err, double k_e,
                                               const int* __restrict__ sorted_struct) {
  __shared__ NbrWarpSmem ws[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a = (int64_t)blockIdx.x * 8 + w;
  if (a >= n) return;  // whole warp
  const StructDev& S = st[sorted_struct[a]];
  const int sa = spec[a];
  const uint32_t mask = S.narrow[sa];
  if (!S.any_narrow || mask == 0) {
    if (!FILL && lane == 0) row_cnt[a] = 0;
    return;
  }
  const int bs = base[a];
  const int bb[3] = {(bs & 1023) / QEQ_BIN, ((bs >> 10) & 1023) / QEQ_BIN, ((bs >> 20) & 1023) / QEQ_BIN};
  const double ra0 = posc[3 * a], ra1 = posc[3 * a + 1], ra2 = posc[3 * a + 2];
  const float4 pa = posc32[a];
  const double rc = S.r_cut, rc2 = rc * rc;
  // FP32 rounding of |r| is below ~1e-7 of the cell's extent: 1e-6 of it plus 1e-3 A is safe
  const double ext = norm3d(S.h[0], S.h[1], S.h[2]) + norm3d(S.h[3], S.h[4], S.h[5]) + norm3d(S.h[6], S.h[7], S.h[8]);
  const double marg = 1e-3 + 1e-6 * ext;
  const float in2 = (float)((rc - marg) * (rc - marg)), out2 = (float)((rc + marg) * (rc + marg));
  const int64_t out = FILL ? row[a] : 0;
  int cnt = 0;
  warp_neighbour_walk(S, bb, S.rs_range, bin_start, ws[w],
                      [&](bool valid, int t, const double* sh, const float* sh32, bool zero, int code) {
    bool acc = false, band = false;
    if (valid && ((mask >> spec[t]) & 1u) && !(zero && t == a)) {
      const float4 pt = posc32[t];
      const float dx = pt.x + sh32[0] - pa.x, dy = pt.y + sh32[1] - pa.y, dz = pt.z + sh32[2] - pa.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      acc = r2 < in2;
      band = !acc && r2 <= out2;
    }
    if (__any_sync(0xffffffffu, band) && band) {  // rare: the exact FP64 test
      const double dx = posc[3 * t] + sh[0] - ra0, dy = posc[3 * t + 1] + sh[1] - ra1,
                   dz = posc[3 * t + 2] + sh[2] - ra2;
      acc = dx * dx + dy * dy + dz * dz < rc2;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, acc);
    if (FILL && acc) {
      const int64_t o = out + cnt + __popc(bal & ((1u << lane) - 1u));
      if (o < cap) {
        col[o] = t;
        val64[o] = (double)code;  // replaced by the pair value below
      }
    }
    cnt += __popc(bal);
  });
  if (FILL) {
    __syncwarp();
    const int64_t m = min((int64_t)cnt, cap - out);
    for (int64_t k = lane; k < m; k += 32) {
      const int64_t o = out + k;
      const int t = col[o];
      int s[3];
      unpack_image((int)val64[o], s);
      double d2 = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double dd = posc[3 * t + d] + (s[0] * S.h[d] + s[1] * S.h[3 + d] + s[2] * S.h[6 + d]) -
                          (d == 0 ? ra0 : (d == 1 ? ra1 : ra2));
        d2 += dd * dd;
      }
      const double r = sqrt(d2);
      const int kk = sa * QEQ_MAX_SPECIES + spec[t];
      double v;
      if (r > 1e-12)
        v = (erfc(r * S.inv_sw[kk]) - erfc(r * S.inv_sg[kk])) / r;
      else  // coincident atoms: the r -> 0 limit
        v = (2.0 / sqrt(M_PI)) * (S.inv_sg[kk] - S.inv_sw[kk]);
      v *= k_e;
      val64[o] = v;
      val32[o] = (float)v;
    }
  }
  if (lane == 0) {
    if (!FILL) row_cnt[a] = cnt;
    if (FILL && out + cnt > cap) atomicOr(err, ERRBIT_PAIRCAP);
  }
}

__global__ void k_sorted_struct(const int* __restrict__ atom_struct, const int* __restrict__ perm, int64_t n,
                                int* __restrict__ out) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) out[a] = atom_struct[perm[a]];
}

}  // namespace

cudaError_t launch_prepare_atoms(qeq_plan_s* P, const double* pos, const int32_t* species, const double* chi,
                                 const double* J, int need_pairs) {
  cudaStream_t s = P->stream;
  int64_t n = P->n_atoms;
  int nb = (int)((n + 255) / 256);
  QEQ_CUDA_TRY(cudaMemsetAsync(P->d_bin_count, 0, sizeof(int) * (P->total_bins + 1), s));
  QEQ_CUDA_TRY(cudaMemsetAsync(P->d_bin_fill, 0, sizeof(int) * (P->total_bins + 1), s));
  count_launch(P, need_pairs ? 5 + 3 + 2 + 3 : 5 + 3);
  k_bin_atoms<<<nb, 256, 0, s>>>(P->d_st, P->d_atom_struct, n, pos, species, chi, J, P->d_key, P->d_bin_count,
                                  P->d_err);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(exclusive_scan<int>(P->d_bin_count, P->total_bins, P->d_bin_start, P->d_scan_tmp, s));
  k_scatter<<<nb, 256, 0, s>>>(P->d_key, n, P->d_bin_start, P->d_bin_fill, P->d_perm);
  k_sort_bins<<<(P->total_bins + 255) / 256, 256, 0, s>>>(P->d_bin_start, P->total_bins, P->d_perm);
  // sorted structure index reuses d_key (no longer needed)
  k_sorted_struct<<<nb, 256, 0, s>>>(P->d_atom_struct, P->d_perm, n, P->d_key);
  k_gather_sorted<<<nb, 256, 0, s>>>(P->d_st, P->d_atom_struct, P->d_perm, n, pos, species, chi, J, QEQ_MAXP,
                                      P->d_base, P->d_wts, P->d_wts32, P->d_spec, P->d_J, P->d_chi, P->d_dinv,
                                      P->d_posc, P->d_posc32);
  QEQ_CUDA_TRY(cudaGetLastError());
  if (need_pairs) {
    const int nbw = (int)((n + 7) / 8);  // one warp per atom
    k_pairs<0><<<nbw, 256, 0, s>>>(P->d_st, P->d_bin_start, n, P->d_base, P->d_spec, P->d_posc, P->d_posc32,
                                    P->d_row_cnt,
                                    nullptr, 0, nullptr, nullptr, nullptr, P->d_err, P->desc.coulomb_k, P->d_key);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(exclusive_scan<int64_t>(P->d_row_cnt, n, P->d_row, (int64_t*)P->d_scan_tmp, s));
    k_pairs<1><<<nbw, 256, 0, s>>>(P->d_st, P->d_bin_start, n, P->d_base, P->d_spec, P->d_posc, P->d_posc32,
                                    nullptr,
                                    P->d_row, P->pair_cap, P->d_col, P->d_val64, P->d_val32, P->d_err,
                                    P->desc.coulomb_k, P->d_key);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  P->have_atoms = true;
  return cudaSuccess;
}
