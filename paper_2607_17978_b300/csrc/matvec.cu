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
// multiply separates them with Z(m) and conj(Z(-m)).  The FFT passes (fft.cuh)
// stream whole mesh lines through shared memory with TMA bulk copies; the
// x-direction FFT, the multiply and the inverse x-direction FFT run in one kernel
// over pairs of mesh lines (y,z) and (-y,-z).  Spreading and gathering work on
// 16^3 bricks whose atoms were sorted by prep.cu; spreading accumulates each
// brick row in registers (no atomics, fixed order) and writes each mesh point once.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "fft.cuh"
#include "qeq_internal.cuh"

namespace {

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
    const int e = (d == 2) ? QEQ_BRICK_Z : QEQ_BRICK_XY;
    B.x0[d] = bc[d] * e;
    B.ext[d] = min(e, S.K[d] - B.x0[d]);
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
// shared memory: stencil starts relative to the brick, 16-bit masks of the brick
// rows the stencil covers in x and y, and its weights laid out on the brick's 16
// positions per direction (0 where the stencil does not reach; x pre-multiplied by
// the charge).  Every thread then adds, atom after atom in a fixed order, its
// row's contribution: the spread is deterministic and each mesh point is written
// to global memory once.
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
  T wz[QEQ_SPB][QEQ_BRICK_Z];   // z weights on the brick's z positions (0 outside the stencil)
  T wx[QEQ_SPB][QEQ_BRICK_XY];  // q * x weights on the brick's x rows
  T wy[QEQ_SPB][QEQ_BRICK_XY];  // y weights on the brick's y rows
  unsigned mask[QEQ_SPB];       // x rows (bits 0-15) and y rows (bits 16-31) the stencil covers
  int off[QEQ_SPB];             // stencil starts ox | oy << 10 | oz << 20, species part << 30
  int atom[QEQ_SPB];            // the candidate's atom (sorted index)
};

// The P stored B-spline weights of one direction of atom t (16-byte loads: the weight
// rows of 3 QEQ_MAXP values start on 16-byte boundaries).
template <typename T>
__device__ __forceinline__ void load_weights8(const T* __restrict__ src, T (&w)[QEQ_MAXP]);
template <>
__device__ __forceinline__ void load_weights8<float>(const float* __restrict__ src, float (&w)[QEQ_MAXP]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(src)), b = __ldg(reinterpret_cast<const float4*>(src) + 1);
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
template <>
__device__ __forceinline__ void load_weights8<double>(const double* __restrict__ src, double (&w)[QEQ_MAXP]) {
#pragma unroll
  for (int i = 0; i < QEQ_MAXP / 2; ++i) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(src) + i);
    w[2 * i] = a.x;
    w[2 * i + 1] = a.y;
  }
}
static_assert(QEQ_MAXP == 8 && (3 * QEQ_MAXP * 4) % 16 == 0, "weight rows are loaded as 16-byte vectors");

// the brick's rows as they are written out: 256 rows of 16 z (one pad element per row)
constexpr int kSpreadStageLd = QEQ_BRICK_Z + 1;

template <typename T, int P>
constexpr size_t spread_smem() {
  const size_t rec = sizeof(SpreadRecs<T, P>);
  const size_t stage = (size_t)QEQ_BRICK_XY * QEQ_BRICK_XY * kSpreadStageLd * 2 * sizeof(T);
  return rec > stage ? rec : stage;
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_spread(const StructDev* __restrict__ st, const int* __restrict__ brick_struct,
                         const int* __restrict__ brick_cand, const int* __restrict__ bin_start, const int* __restrict__ base,
                         const T* __restrict__ wts, const int* __restrict__ spec, const double* __restrict__ x,
                         const float* __restrict__ x32, const PcgScalars* __restrict__ sc, int use_active,
                         typename C2<T>::t* __restrict__ mesh) {
  using V = typename C2<T>::t;
  const int g = blockIdx.x;
  const int s = brick_struct[g];
  const StructDev& S = st[s];
  if (use_active && !sc[s].active) return;
  // warp w owns the brick rows x in [4 (w mod 4), +4), y in [8 (w / 4), +8)
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int lx = (w & 3) * 4 + (lane >> 3), ly = (w >> 2) * 8 + (lane & 7);
  const Brick B = brick_of(S, g);
  const int K0 = S.K[0], K1 = S.K[1], K2 = S.K[2];
  __shared__ int cand[3][8], ncand[3];
  __shared__ int bin_beg[512], bin_pre[513];
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SpreadRecs<T, P>& R = *reinterpret_cast<SpreadRecs<T, P>*>(smem_raw);
  if (tid < QEQ_BRICK_CAND) {  // the brick's candidate bins per direction (plan table)
    const int v = brick_cand[(size_t)g * QEQ_BRICK_CAND + tid];
    if (tid < 3) ncand[tid] = v;
    else if (tid >= 4) cand[(tid - 4) >> 3][(tid - 4) & 7] = v;
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
    T re[QEQ_BRICK_Z], im[QEQ_BRICK_Z];
#pragma unroll
    for (int z = 0; z < QEQ_BRICK_Z; ++z) re[z] = im[z] = (T)0;
    for (int c0 = 0; c0 < total; c0 += QEQ_SPB) {
      const int nbat = min(QEQ_SPB, total - c0);
      if (c0 > 0) __syncthreads();  // the previous batch is consumed
      // staging, one thread per candidate: its atom, stencil starts and covered rows
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
          const unsigned xm = stencil_rows<P>(o[0], K0, B.ext[0]);
          const unsigned ym = stencil_rows<P>(o[1], K1, B.ext[1]);
          const unsigned zm = stencil_rows<P>(o[2], K2, B.ext[2]);
          if (zm) mask = xm | (ym << 16);
          R.off[tid] = o[0] | (o[1] << 10) | (o[2] << 20) | ((sp & 1) << 30);
        }
        R.mask[tid] = mask;
        R.atom[tid] = t;
      }
      __syncthreads();
      // ... then every thread: one direction of a kept record, its P weights read as
      // 16-byte vectors and laid out on the brick's 16 positions (periodic images added)
      for (int idx = tid; idx < nbat * 3; idx += blockDim.x) {
        const int r = idx / 3, d = idx - 3 * r;
        if (!R.mask[r]) continue;
        const int t = R.atom[r];
        T w[QEQ_MAXP];
        load_weights8<T>(wts + (size_t)t * 3 * QEQ_MAXP + d * QEQ_MAXP, w);
        const T scale = (d == 0) ? xval<T>(x, x32, t) : (T)1;
        T* dst = (d == 0) ? R.wx[r] : (d == 1) ? R.wy[r] : R.wz[r];
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[k] = (T)0;
        const int o = (R.off[r] >> (10 * d)) & 1023, K = S.K[d];
        const int ext = (d == 0) ? B.ext[0] : (d == 1) ? B.ext[1] : B.ext[2];  // B stays in registers
#pragma unroll
        for (int j = 0; j < P; ++j) {
          int k = o + j;
          if (k >= K) k -= K;
          for (; k < ext; k += K) dst[k] += scale * w[P - 1 - j];
        }
      }
      __syncthreads();
      // every thread adds its row's share, atom after atom.  A warp ballots the records
      // whose stencil covers one of its 4 x rows and one of its 8 y rows (32 records per
      // ballot) and visits only those, in record order.
      const unsigned xsel = 0xFu << (4 * (w & 3)), ysel = 0xFFu << (16 + 8 * (w >> 2));
      for (int i0 = 0; i0 < nbat; i0 += 32) {
        const int ii = i0 + lane;
        const unsigned mm = ii < nbat ? R.mask[ii] : 0u;
        unsigned bal = __ballot_sync(0xffffffffu, (mm & xsel) != 0u && (mm & ysel) != 0u);
        while (bal) {
          const int k = i0 + __ffs(bal) - 1;
          bal &= bal - 1u;
          // 0 on lanes whose row the stencil does not cover
          const T r = R.wx[k][lx] * R.wy[k][ly];
          const T* wz = R.wz[k];
          if ((R.off[k] >> 30) & 1) {
#pragma unroll
            for (int z = 0; z < QEQ_BRICK_Z; ++z) im[z] += r * wz[z];
          } else {
#pragma unroll
            for (int z = 0; z < QEQ_BRICK_Z; ++z) re[z] += r * wz[z];
          }
        }
      }
      __syncthreads();
    }
    // write the brick through shared memory: a warp stores four whole rows (16 z points,
    // contiguous in layout L0) per instruction instead of one point of 32 rows
    __syncthreads();  // the records are consumed
    {
      V* stage = reinterpret_cast<V*>(smem_raw);
#pragma unroll
      for (int z = 0; z < QEQ_BRICK_Z; ++z) stage[(lx * QEQ_BRICK_XY + ly) * kSpreadStageLd + z] = V{re[z], im[z]};
      __syncthreads();
      const int zz = (lane & 7) * 2;
      for (int row = (tid >> 5) * 4 + (lane >> 3); row < QEQ_BRICK_XY * QEQ_BRICK_XY; row += 32) {
        const int rx = row >> 4, ry = row & 15;
        if (rx < B.ext[0] && ry < B.ext[1]) {
          V* mg = mesh + S.mesh_off + (int64_t)cm * S.Mp +
                  ((int64_t)(B.x0[0] + rx) * K1 + (B.x0[1] + ry)) * S.P[2] + B.x0[2];
          if (zz < B.ext[2]) mg[zz] = stage[row * kSpreadStageLd + zz];
          if (zz + 1 < B.ext[2]) mg[zz + 1] = stage[row * kSpreadStageLd + zz + 1];
        }
      }
      __syncthreads();  // the staging area is reused by the next complex mesh's records
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
      const V* mg = mesh + S.mesh_off + (int64_t)(sp >> 1) * S.Mp;
      const int bs = base[t];
      const int f0 = bs & 1023, f1 = (bs >> 10) & 1023, f2 = (bs >> 20) & 1023;
      const T* wt = wts + (size_t)t * 3 * QEQ_MAXP;
      T acc = (T)0;
      if (jz < P) {
        int kz = f2 - (P - 1) + jz;
        if (kz < 0) kz += S.K[2];
        const T wzj = wt[2 * QEQ_MAXP + P - 1 - jz];
        T racc = (T)0;
        if constexpr (P == 8) {
          // lane rows: y = rsub and rsub + 4, all 8 x; the 16 loads are issued before
          // any is used, the y weights are read once
          const int K1 = S.K[1];
          const int64_t P2 = S.P[2];
          int ky0 = f1 - 7 + rsub;
          if (ky0 < 0) ky0 += K1;
          int ky1 = f1 - 3 + rsub;
          if (ky1 < 0) ky1 += K1;
          const T wy0 = wt[QEQ_MAXP + 7 - rsub], wy1 = wt[QEQ_MAXP + 3 - rsub];
          V v0[8], v1[8];
#pragma unroll
          for (int jx = 0; jx < 8; ++jx) {
            int kx = f0 - 7 + jx;
            if (kx < 0) kx += S.K[0];
            const V* rowp = mg + (int64_t)kx * K1 * P2 + kz;
            v0[jx] = __ldg(rowp + ky0 * P2);
            v1[jx] = __ldg(rowp + ky1 * P2);
          }
#pragma unroll
          for (int jx = 0; jx < 8; ++jx)
            racc += wt[7 - jx] * (wy0 * (part_ ? v0[jx].y : v0[jx].x) + wy1 * (part_ ? v1[jx].y : v1[jx].x));
        } else {
          // a constant trip count (P^2/4 rows per lane) lets the loads be in flight at once
#pragma unroll
          for (int i = 0; i < P * P / 4; ++i) {
            const int r = rsub + 4 * i;
            const int jx = r / P, jy = r - (r / P) * P;
            int kx = f0 - (P - 1) + jx;
            if (kx < 0) kx += S.K[0];
            int ky = f1 - (P - 1) + jy;
            if (ky < 0) ky += S.K[1];
            const V v = __ldg(mg + ((int64_t)kx * S.K[1] + ky) * S.P[2] + kz);
            racc += wt[P - 1 - jx] * wt[QEQ_MAXP + P - 1 - jy] * (part_ ? v.y : v.x);
          }
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
  const int nspec = st[ch.s].S;  // FP64 work only for the structure's own species
  __shared__ double red[QEQ_MAX_SPECIES][33];
  double loc[QEQ_MAX_SPECIES];
#pragma unroll
  for (int k = 0; k < QEQ_MAX_SPECIES; ++k) loc[k] = 0.0;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const int sp = spec[a];
    const double xa = x[a];
    if (x32) x32[a] = (float)xa;
#pragma unroll
    for (int k = 0; k < QEQ_MAX_SPECIES; ++k)
      if (k < nspec) loc[k] += (sp == k) ? xa : 0.0;
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < QEQ_MAX_SPECIES; ++k) {
    if (k >= nspec) break;
    double v = warp_sum<double>(loc[k]);
    if (lane == 0) red[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < nspec) {
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
      const double tot = (k < nspec) ? ordered_block_sum(part, ch.first, ch.count, QEQ_MAX_SPECIES, k, red2) : 0.0;
      if (threadIdx.x == 0) sc[ch.s].xsum[k] = tot;
    }
    if (threadIdx.x == 0) counter[ch.s] = 0;
  }
}

// ------------------------------------------------------------------ Fourier preconditioner
// The coarse spread takes v = D^-1 (r - shift 1) (shift: the PCG's running estimate of
// mu, 0 for the ones vector).  The preconditioner's output enters the projected
// direction z = M^-1 r - (1.M^-1 r / 1.M^-1 1) M^-1 1, which the shift leaves unchanged
// (it adds a multiple of M^-1 1 to M^-1 r); without it r carries mu 1, and near
// convergence the part of v that matters is ~1e-6 of max|v|.
__device__ __forceinline__ double pre_shift(const PcgScalars& c, int ones_input) {
  return ones_input ? 0.0 : c.shift;
}
// Power-of-two scale of the fixed-point coarse spread: max |v| is at most
// max|r - shift| max D^-1 (max D^-1 alone for the ones vector), mapped to 2^23 (the
// resolution of an FP32 mantissa); a contribution (B-spline weight product at most
// (2/3)^3 < 2^-1.75) stays below 2^21.25, so a tile point's 32-bit sum is exact for
// fewer than 2^9 contributions: a tile group with kPreTileMaxAtoms atoms or more adds
// straight to the 64-bit mesh (a point gets ~20 in dense matter).
__device__ __forceinline__ double pre_fixed_scale(const PcgScalars& c, int ones_input) {
  const double sh = pre_shift(c, ones_input);
  double b = c.dinv_max * (ones_input ? 1.0 : fmax(fabs(c.r_max - sh), fabs(c.r_min - sh)));
  if (!(b > 0.0) || !isfinite(b)) b = 1.0;
  int e;
  frexp(b, &e);                    // b < 2^e
  return ldexp(1.0, 23 - e);
}
constexpr int kPreTileMaxAtoms = 512;

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

// v = D^-1 r spread on the coarse mesh in fixed point: every contribution is rounded to
// an integer multiple of 2^-e (e per structure, from a bound on max |v|, pre_fixed_scale)
// and added with integer atomics.  Integer addition does not depend on the order of the
// additions, so the coarse mesh, and with it every preconditioned solve, is bitwise
// reproducible.  One CTA per tile group (plan: QEQ_PRE_TILE_G^2 fine bin columns, a run
// of z bins): its atoms add their 64 contributions into the group's tile of the coarse
// mesh in shared memory (32-bit integer atomics), then the tile's nonzero partial sums go
// to the 64-bit mesh (one global atomic per point instead of one per contribution; a
// tile point gets the contributions of the ~20 atoms around it).  A contribution outside
// the tile (only possible through rounding at a bin edge) goes straight to the mesh.
// The sums are those of one atomic per contribution, bit for bit.
// k_pre_fixed_to_float turns the sums back into the FP32 mesh.
__global__ void __launch_bounds__(256) k_pre_spread_tiles(
    const StructDev* __restrict__ stf, const StructDev* __restrict__ stp, const int4* __restrict__ tiles, int gz,
    const int* __restrict__ bin_start, const int* __restrict__ pbase, const float* __restrict__ pw,
    const double* __restrict__ dinv, const double* __restrict__ r, const PcgScalars* __restrict__ sc, int use_active,
    int ones_input, unsigned long long* __restrict__ imesh) {
  extern __shared__ __align__(16) int tile[];
  const int4 tg = tiles[blockIdx.x];
  const int s = tg.x;
  if (use_active && !sc[s].active) return;
  const StructDev& F = stf[s];
  const StructDev& C = stp[s];
  const int K0 = C.K[0], K1 = C.K[1], K2 = C.K[2];
  int ox, ex, oy, ey, oz, ez;
  pre_tile_range(tg.y, QEQ_PRE_TILE_G, F.nb[0], K0, F.K[0], ox, ex);
  pre_tile_range(tg.z, QEQ_PRE_TILE_G, F.nb[1], K1, F.K[1], oy, ey);
  pre_tile_range(tg.w, gz, F.nb[2], K2, F.K[2], oz, ez);
  const int npts = ex * ey * ez;
  for (int i = threadIdx.x; i < npts; i += blockDim.x) tile[i] = 0;
  const double scale = pre_fixed_scale(sc[s], ones_input);
  const double sh = pre_shift(sc[s], ones_input);
  unsigned long long* m = imesh + C.mesh_off;
  const int bz1 = min(tg.w + gz, F.nb[2]);
  int ntot = 0;  // atoms of the group (the same on every thread)
  for (int c = 0; c < QEQ_PRE_TILE_G * QEQ_PRE_TILE_G; ++c) {
    const int bx = tg.y + c / QEQ_PRE_TILE_G, by = tg.z + c % QEQ_PRE_TILE_G;
    if (bx >= F.nb[0] || by >= F.nb[1]) continue;
    const int col = F.bin_off + (bx * F.nb[1] + by) * F.nb[2];
    ntot += bin_start[col + bz1] - bin_start[col + tg.w];
  }
  const bool use_tile = ntot < kPreTileMaxAtoms;
  __syncthreads();
  for (int c = 0; c < QEQ_PRE_TILE_G * QEQ_PRE_TILE_G; ++c) {
    const int bx = tg.y + c / QEQ_PRE_TILE_G, by = tg.z + c % QEQ_PRE_TILE_G;
    if (bx >= F.nb[0] || by >= F.nb[1]) continue;
    const int col = F.bin_off + (bx * F.nb[1] + by) * F.nb[2];
    const int a0 = bin_start[col + tg.w], na = bin_start[col + bz1] - a0;
    // 16 items per atom: its (x, y) stencil rows, 4 z points each
    for (int it = threadIdx.x; it < na * 16; it += blockDim.x) {
      const int a = a0 + (it >> 4), jx = (it >> 2) & 3, jy = it & 3;
      const int bs = pbase[a];
      const float* w = pw + (size_t)a * 12;
      // the scale is a power of two: scaling the FP32 value is exact (|vs| <= 2^23)
      const float vs = (float)((double)(float)(dinv[a] * (r[a] - sh)) * scale);
      int kx = (bs & 1023) - jx;
      if (kx < 0) kx += K0;
      int ky = ((bs >> 10) & 1023) - jy;
      if (ky < 0) ky += K1;
      int tx = kx - ox;
      if (tx < 0) tx += K0;
      int ty = ky - oy;
      if (ty < 0) ty += K1;
      const float wxy = vs * w[jx] * w[4 + jy];
      const int fz = (bs >> 20) & 1023;
#pragma unroll
      for (int jz = 0; jz < 4; ++jz) {
        int kz = fz - jz;
        if (kz < 0) kz += K2;
        int tz = kz - oz;
        if (tz < 0) tz += K2;
        const int v = __float2int_rn(wxy * w[8 + jz]);
        if (use_tile && tx < ex && ty < ey && tz < ez)
          atomicAdd(&tile[(tx * ey + ty) * ez + tz], v);
        else
          atomicAdd(&m[((int64_t)kx * K1 + ky) * C.P[2] + kz], (unsigned long long)(long long)v);
      }
    }
  }
  __syncthreads();
  if (!use_tile) return;
  for (int i = threadIdx.x; i < npts; i += blockDim.x) {
    const int v = tile[i];
    if (v == 0) continue;
    const int tz = i % ez, txy = i / ez, ty = txy % ey, tx = txy / ey;
    int kx = ox + tx, ky = oy + ty, kz = oz + tz;
    if (kx >= K0) kx -= K0;
    if (ky >= K1) ky -= K1;
    if (kz >= K2) kz -= K2;
    atomicAdd(&m[((int64_t)kx * K1 + ky) * C.P[2] + kz], (unsigned long long)(long long)v);
  }
}

// fixed-point coarse mesh -> FP32 complex mesh (real part), structure found by bisection;
// the scale is a power of two, so v 2^-e rounds once to FP32 either way
__global__ void k_pre_fixed_to_float(const StructDev* __restrict__ stp, int ns, int64_t total,
                                     const PcgScalars* __restrict__ sc, int ones_input,
                                     const unsigned long long* __restrict__ imesh, float2* __restrict__ mesh) {
  int cur = -1;
  float inv = 0.f;
  int64_t end = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (cur < 0 || i >= end) {
      int lo = 0, hi = ns - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (stp[mid].mesh_off <= i) lo = mid;
        else hi = mid - 1;
      }
      cur = lo;
      end = (lo + 1 < ns) ? stp[lo + 1].mesh_off : total;
      inv = (float)(1.0 / pre_fixed_scale(sc[lo], ones_input));
    }
    mesh[i] = make_float2(__ll2float_rn((long long)imesh[i]) * inv, 0.f);
  }
}

// u = D^-1 (r - shift - phi), phi the interpolated coarse potential; per-structure sum of u
__global__ void k_pre_gather(const Chunk* __restrict__ chunks, const StructDev* __restrict__ stp,
                             const int* __restrict__ pbase, const float* __restrict__ pw,
                             const double* __restrict__ dinv, const double* __restrict__ r,
                             const float2* __restrict__ mesh, PcgScalars* __restrict__ sc, int use_active,
                             int slot, double* __restrict__ u, double* __restrict__ part, int* __restrict__ counter) {
  const Chunk ch = chunks[blockIdx.x];
  if (use_active && !sc[ch.s].active) return;
  const StructDev& S = stp[ch.s];
  const float2* m = mesh + S.mesh_off;
  const double sh = pre_shift(sc[ch.s], slot == 1);  // as the spread (k_pre_spread_tiles)
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
        const float2* row = m + ((int64_t)kx * S.K[1] + ky) * S.P[2];
        float rs = 0.f;
        for (int jz = 0; jz < 4; ++jz) {
          int kz = f[2] - jz;
          if (kz < 0) kz += S.K[2];
          rs += w[8 + jz] * row[kz].x;
        }
        phi += w[jx] * w[4 + jy] * rs;
      }
    }
    double ua = dinv[a] * (r[a] - sh - (double)phi);
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
// Persistent grid of an FFT pass: the resident CTAs of all SMs, at most one per unit.
int fft_grid(qeq_plan_s* P, const void* fn, size_t smem, int nunits, int threads) {
  int blocks = 0;
  for (int i = 0; i < P->n_occ; ++i)
    if (P->occ[i].fn == fn && P->occ[i].smem == smem) {
      blocks = P->occ[i].blocks;
      break;
    }
  if (blocks == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem) != cudaSuccess || blocks < 1) {
      cudaGetLastError();
      blocks = 1;
    }
    if (P->n_occ < (int)(sizeof(P->occ) / sizeof(P->occ[0]))) P->occ[P->n_occ++] = {fn, smem, blocks};
  }
  return std::max(1, std::min(nunits, blocks * P->num_sms));
}

// The five FFT passes (buffers a: L0 / L2, b: L1 / L3): ZF a -> b, YF b -> a, X a -> b,
// YI b -> a, ZI a in place.  mark() records a stage event after each pass.
template <typename T, bool PRE, class Mark>
cudaError_t launch_fft_passes(qeq_plan_s* Pl, const FftGeom& g, const int* kmax, const StructDev* st,
                              const int4* zit, int nz, const int4* yit, int ny, const int4* yiit, int nyi,
                              const int4* xit, int nx, int use_active, typename C2<T>::t* a, typename C2<T>::t* b,
                              int max_species, Mark mark) {
  using V = typename C2<T>::t;
  constexpr bool F32 = std::is_same<T, float>::value;
  constexpr int FT = F32 ? QEQ_FFT_THREADS32 : 256;  // threads per CTA (the kernels' launch bounds)
  cudaStream_t s = Pl->stream;
  const T* bmod = (const T*)(F32 ? (const void*)Pl->d_bmod32
                                 : (std::is_same<T, dd>::value ? (const void*)Pl->d_bmod_dd : (const void*)Pl->d_bmod));
  const int sub = F32 ? g.sub32 : g.sub64;
  const int subx = F32 ? g.subx32 : g.subx64;
  const int nsub = (g.tl + sub - 1) / sub, nsubx = (g.tlx + subx - 1) / subx;
  const int ldz = F32 ? g.ldz32 : g.ldz64, ldy = F32 ? g.ldy32 : g.ldy64, ldx = F32 ? g.ldx32 : g.ldx64;
  const size_t smz = 128 + 2 * (size_t)fft_buf(kmax[2], ldz, sub, sizeof(V), 1, 0).bytes;
  const size_t smy = 128 + 2 * (size_t)fft_buf(kmax[1], ldy, sub, sizeof(V), 1, 0).bytes;
  const int* tabs = Pl->d_fft_tabs;
  int* err = Pl->d_err;
  {
    auto fn = k_fft_tile<T, PASS_ZF>;
    fn<<<fft_grid(Pl, (const void*)fn, smz, nz * nsub, FT), FT, smz, s>>>(
        st, Pl->d_fft, zit, nz, g.tl, sub, kmax[2], ldz, Pl->d_tw64, Pl->d_tw32, tabs, Pl->d_sc, use_active, a, b, err);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(mark());
  }
  {
    auto fn = k_fft_tile<T, PASS_YF>;
    fn<<<fft_grid(Pl, (const void*)fn, smy, ny * nsub, FT), FT, smy, s>>>(
        st, Pl->d_fft, yit, ny, g.tl, sub, kmax[1], ldy, Pl->d_tw64, Pl->d_tw32, tabs, Pl->d_sc, use_active, b, a, err);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(mark());
  }
  {
    const int stall = PRE ? 0 : Pl->test_stall;
    if (PRE || max_species <= 2) {
      auto fn = k_fft_x_green<T, PRE, 2>;
      const size_t smx = 128 + 2 * (size_t)fft_buf(kmax[0], ldx, 2 * subx, sizeof(V), 2,
                                                   fft_x_extra(subx, 1, sizeof(T))).bytes;
      fn<<<fft_grid(Pl, (const void*)fn, smx, nx * nsubx, FT), FT, smx, s>>>(
          st, Pl->d_fft, xit, nx, g.tlx, subx, kmax[0], ldx, bmod, Pl->d_tw64, Pl->d_tw32, tabs, Pl->d_sc,
          use_active, a, b, err, stall);
    } else {
      constexpr int HX = QEQ_MAX_SPECIES / 2;
      auto fn = k_fft_x_green<T, false, QEQ_MAX_SPECIES>;
      const size_t smx = 128 + 2 * (size_t)fft_buf(kmax[0], ldx, 2 * HX * subx, sizeof(V), 2,
                                                   fft_x_extra(subx, HX, sizeof(T))).bytes;
      fn<<<fft_grid(Pl, (const void*)fn, smx, nx * nsubx, FT), FT, smx, s>>>(
          st, Pl->d_fft, xit, nx, g.tlx, subx, kmax[0], ldx, bmod, Pl->d_tw64, Pl->d_tw32, tabs, Pl->d_sc,
          use_active, a, b, err, stall);
    }
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(mark());
  }
  {
    auto fn = k_fft_tile<T, PASS_YI>;
    fn<<<fft_grid(Pl, (const void*)fn, smy, nyi * nsub, FT), FT, smy, s>>>(
        st, Pl->d_fft, yiit, nyi, g.tl, sub, kmax[1], ldy, Pl->d_tw64, Pl->d_tw32, tabs, Pl->d_sc, use_active, b, a,
        err);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(mark());
  }
  {
    auto fn = k_fft_tile<T, PASS_ZI>;
    fn<<<fft_grid(Pl, (const void*)fn, smz, nz * nsub, FT), FT, smz, s>>>(
        st, Pl->d_fft, zit, nz, g.tl, sub, kmax[2], ldz, Pl->d_tw64, Pl->d_tw32, tabs, Pl->d_sc, use_active, a, a, err);
    QEQ_CUDA_TRY(cudaGetLastError());
    QEQ_CUDA_TRY(mark());
  }
  return cudaSuccess;
}

template <typename T, int P>
cudaError_t matvec_impl(qeq_plan_s* Pl, const double* x, double* y, int with_J, int use_active, int fuse_pAp,
                        cudaEvent_t* ev) {
  using V = typename C2<T>::t;
  constexpr bool F32 = std::is_same<T, float>::value;
  cudaStream_t s = Pl->stream;
  V* mesh = reinterpret_cast<V*>(Pl->d_mesh);
  const T* wts = F32 ? (const T*)(const void*)Pl->d_wts32 : (const T*)(const void*)Pl->d_wts;
  const T* bmod = F32 ? (const T*)(const void*)Pl->d_bmod32 : (const T*)(const void*)Pl->d_bmod;
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
    k_spread<T, P><<<Pl->total_bricks, 256, spread_smem<T, P>(), s>>>(Pl->d_st, Pl->d_brick_struct, Pl->d_brick_cand, Pl->d_bin_start, Pl->d_base, wts,
                                                      Pl->d_spec, x, x32, Pl->d_sc, use_active, mesh);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  QEQ_CUDA_TRY(mark());
  V* mesh2 = reinterpret_cast<V*>(Pl->d_mesh2);
  QEQ_CUDA_TRY((launch_fft_passes<T, false>(Pl, Pl->geo, Pl->fft_kmax, Pl->d_st, Pl->d_zitems, Pl->n_zitems, Pl->d_yitems,
                                            Pl->n_yitems, Pl->d_yiitems, Pl->n_yiitems, Pl->d_xitems, Pl->n_xitems,
                                            use_active, mesh, mesh2, Pl->max_species, mark)));
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

// FP64 mesh <-> double-float mesh, in place (16 bytes per complex point either way)
__global__ void k_mesh_to_dd(double2* __restrict__ m, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = m[i];
    ddc c;
    c.x = dd(v.x);
    c.y = dd(v.y);
    reinterpret_cast<ddc*>(m)[i] = c;
  }
}
__global__ void k_mesh_from_dd(double2* __restrict__ m, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ddc c = reinterpret_cast<const ddc*>(m)[i];
    m[i] = make_double2((double)c.x, (double)c.y);
  }
}

// The FP64-accurate matvec of a mixed-precision plan (final checks, energies, force_fp64):
// FP64 species sums, spread, gather and local terms as matvec_impl<double>, the five FFT
// passes in double-float arithmetic on the FP32 pipes (dd.cuh; ~2^-44 relative per
// operation, far below what the checks resolve).
template <int P>
cudaError_t matvec_check_dd(qeq_plan_s* Pl, const double* x, double* y, int with_J, int use_active, int fuse_pAp,
                            cudaEvent_t* ev) {
  cudaStream_t s = Pl->stream;
  double2* mesh = Pl->d_mesh;
  int rec = 0;
  auto mark = [&]() -> cudaError_t { return ev ? cudaEventRecord(ev[rec++], s) : cudaSuccess; };
  count_launch(Pl, 10);
  QEQ_CUDA_TRY(mark());
  k_species_sums<<<Pl->n_chunks, 256, 0, s>>>(Pl->d_chunks, Pl->d_st, Pl->d_spec, x, Pl->d_sc, use_active,
                                               Pl->d_part, Pl->d_counter, nullptr);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  k_spread<double, P><<<Pl->total_bricks, 256, spread_smem<double, P>(), s>>>(
      Pl->d_st, Pl->d_brick_struct, Pl->d_brick_cand, Pl->d_bin_start, Pl->d_base, Pl->d_wts, Pl->d_spec, x, nullptr,
      Pl->d_sc, use_active, mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  const int nb = (int)std::min<int64_t>((Pl->total_mesh + 255) / 256, (int64_t)Pl->num_sms * 16);
  k_mesh_to_dd<<<nb, 256, 0, s>>>(mesh, Pl->total_mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY(mark());
  QEQ_CUDA_TRY((launch_fft_passes<dd, false>(Pl, Pl->geo, Pl->fft_kmax, Pl->d_st, Pl->d_zitems, Pl->n_zitems,
                                             Pl->d_yitems, Pl->n_yitems, Pl->d_yiitems, Pl->n_yiitems, Pl->d_xitems,
                                             Pl->n_xitems, use_active, reinterpret_cast<ddc*>(mesh),
                                             reinterpret_cast<ddc*>(Pl->d_mesh2), Pl->max_species, mark)));
  k_mesh_from_dd<<<nb, 256, 0, s>>>(mesh, Pl->total_mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  {
    const int with_pairs = Pl->pair_cap > 0;
    k_gather_direct<double, P><<<Pl->n_chunks * Pl->gather_split, 256, 0, s>>>(
        Pl->d_chunks, Pl->d_st, Pl->d_base, Pl->d_wts, Pl->d_spec, Pl->d_J, x, nullptr, Pl->d_row, Pl->d_col,
        Pl->d_val64, Pl->d_val32, with_J, with_pairs, Pl->d_sc, use_active, fuse_pAp,
        Pl->d_part + (size_t)Pl->n_chunks * QEQ_MAX_SPECIES, Pl->d_counter + Pl->n_struct, mesh, y, Pl->gather_split);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  QEQ_CUDA_TRY(mark());
  return cudaSuccess;
}

cudaError_t set_smem_attrs_dd() {
  const int big = 227 * 1024 - 12 * 1024;
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<dd, PASS_ZF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<dd, PASS_YF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<dd, PASS_YI>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<dd, PASS_ZI>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<dd, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<dd, false, QEQ_MAX_SPECIES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return cudaSuccess;
}

template <typename T, int P>
cudaError_t set_smem_attrs() {
  const int big = 227 * 1024 - 12 * 1024;  // leaves room for the kernels' static shared arrays
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_spread<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)spread_smem<T, P>()));
  if (P == 4) {  // the FFT kernels do not depend on the B-spline order: set them once
    QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<T, PASS_ZF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<T, PASS_YF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<T, PASS_YI>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_tile<T, PASS_ZI>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<T, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<T, false, QEQ_MAX_SPECIES>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    if (std::is_same<T, float>::value)
      QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<float, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        big));
    if (std::is_same<T, double>::value) {
      QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<double, false, 2, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, big));
      QEQ_CUDA_TRY(cudaFuncSetAttribute(k_fft_x_green<double, false, QEQ_MAX_SPECIES, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    }
  }
  return cudaSuccess;
}

// FP64 potential meshes of x (spread and the five FFT passes; no gather): the mesh
// buffer then holds phi_s in layout L0 for the force and embedding kernels
template <int P>
cudaError_t potential_impl(qeq_plan_s* Pl, const double* x) {
  cudaStream_t s = Pl->stream;
  double2* mesh = Pl->d_mesh;
  count_launch(Pl, 6);
  k_spread<double, P><<<Pl->total_bricks, 256, spread_smem<double, P>(), s>>>(
      Pl->d_st, Pl->d_brick_struct, Pl->d_brick_cand, Pl->d_bin_start, Pl->d_base, Pl->d_wts, Pl->d_spec, x, nullptr,
      Pl->d_sc, 0, mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  return launch_fft_passes<double, false>(Pl, Pl->geo, Pl->fft_kmax, Pl->d_st, Pl->d_zitems, Pl->n_zitems,
                                         Pl->d_yitems, Pl->n_yitems, Pl->d_yiitems, Pl->n_yiitems, Pl->d_xitems,
                                         Pl->n_xitems, 0, mesh, Pl->d_mesh2, Pl->max_species,
                                         []() { return cudaSuccess; });
}

// Strain derivative sums of the reciprocal quadratic form of x (FP64): spread, forward z
// and y passes, then the x pass in its VIR mode, which leaves 8 doubles per x-pass unit
// in d_mesh2 (units of structure s: items xitem_off[s] .. xitem_off[s+1], times *nsub_out)
template <int P>
cudaError_t virial_impl(qeq_plan_s* Pl, const double* x, int* nsub_out) {
  constexpr int FT = 256;  // FP64 FFT kernels
  cudaStream_t s = Pl->stream;
  double2* a = Pl->d_mesh;
  double2* b = Pl->d_mesh2;
  const FftGeom& g = Pl->geo;
  const int* kmax = Pl->fft_kmax;
  count_launch(Pl, 4);
  k_spread<double, P><<<Pl->total_bricks, 256, spread_smem<double, P>(), s>>>(
      Pl->d_st, Pl->d_brick_struct, Pl->d_brick_cand, Pl->d_bin_start, Pl->d_base, Pl->d_wts, Pl->d_spec, x, nullptr,
      Pl->d_sc, 0, a);
  QEQ_CUDA_TRY(cudaGetLastError());
  const int sub = g.sub64, subx = g.subx64;
  const int nsub = (g.tl + sub - 1) / sub, nsubx = (g.tlx + subx - 1) / subx;
  const size_t smz = 128 + 2 * (size_t)fft_buf(kmax[2], g.ldz64, sub, sizeof(double2), 1, 0).bytes;
  const size_t smy = 128 + 2 * (size_t)fft_buf(kmax[1], g.ldy64, sub, sizeof(double2), 1, 0).bytes;
  {
    auto fn = k_fft_tile<double, PASS_ZF>;
    fn<<<fft_grid(Pl, (const void*)fn, smz, Pl->n_zitems * nsub, FT), FT, smz, s>>>(
        Pl->d_st, Pl->d_fft, Pl->d_zitems, Pl->n_zitems, g.tl, sub, kmax[2], g.ldz64, Pl->d_tw64, Pl->d_tw32,
        Pl->d_fft_tabs, Pl->d_sc, 0, a, b, Pl->d_err);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  {
    auto fn = k_fft_tile<double, PASS_YF>;
    fn<<<fft_grid(Pl, (const void*)fn, smy, Pl->n_yitems * nsub, FT), FT, smy, s>>>(
        Pl->d_st, Pl->d_fft, Pl->d_yitems, Pl->n_yitems, g.tl, sub, kmax[1], g.ldy64, Pl->d_tw64, Pl->d_tw32,
        Pl->d_fft_tabs, Pl->d_sc, 0, b, a, Pl->d_err);
    QEQ_CUDA_TRY(cudaGetLastError());
  }
  const int nx = Pl->n_xitems;
  if (Pl->max_species <= 2) {
    auto fn = k_fft_x_green<double, false, 2, true>;
    const size_t smx = 128 + 2 * (size_t)fft_buf(kmax[0], g.ldx64, 2 * subx, sizeof(double2), 2,
                                                 fft_x_extra(subx, 1, sizeof(double))).bytes;
    fn<<<fft_grid(Pl, (const void*)fn, smx, nx * nsubx, FT), FT, smx, s>>>(
        Pl->d_st, Pl->d_fft, Pl->d_xitems, nx, g.tlx, subx, kmax[0], g.ldx64, Pl->d_bmod, Pl->d_tw64, Pl->d_tw32,
        Pl->d_fft_tabs, Pl->d_sc, 0, a, b, Pl->d_err, 0);
  } else {
    constexpr int HX = QEQ_MAX_SPECIES / 2;
    auto fn = k_fft_x_green<double, false, QEQ_MAX_SPECIES, true>;
    const size_t smx = 128 + 2 * (size_t)fft_buf(kmax[0], g.ldx64, 2 * HX * subx, sizeof(double2), 2,
                                                 fft_x_extra(subx, HX, sizeof(double))).bytes;
    fn<<<fft_grid(Pl, (const void*)fn, smx, nx * nsubx, FT), FT, smx, s>>>(
        Pl->d_st, Pl->d_fft, Pl->d_xitems, nx, g.tlx, subx, kmax[0], g.ldx64, Pl->d_bmod, Pl->d_tw64, Pl->d_tw32,
        Pl->d_fft_tabs, Pl->d_sc, 0, a, b, Pl->d_err, 0);
  }
  *nsub_out = nsubx;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mesh_virial(qeq_plan_s* P, const double* x, int* nsub_out) {
  if (P->max_p == 4) return virial_impl<4>(P, x, nsub_out);
  if (P->max_p == 6) return virial_impl<6>(P, x, nsub_out);
  return virial_impl<8>(P, x, nsub_out);
}

// FP32 potential meshes of x (the mixed-precision path): x in FP32, FP32 spread and passes
__global__ void k_to_f32(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

template <int P>
cudaError_t potential32_impl(qeq_plan_s* Pl, const double* x) {
  cudaStream_t s = Pl->stream;
  float2* mesh = reinterpret_cast<float2*>(Pl->d_mesh);
  count_launch(Pl, 7);
  k_to_f32<<<(int)((Pl->n_atoms + 255) / 256), 256, 0, s>>>(x, Pl->n_atoms, Pl->d_x32);
  k_spread<float, P><<<Pl->total_bricks, 256, spread_smem<float, P>(), s>>>(
      Pl->d_st, Pl->d_brick_struct, Pl->d_brick_cand, Pl->d_bin_start, Pl->d_base, Pl->d_wts32, Pl->d_spec, x,
      Pl->d_x32, Pl->d_sc, 0, mesh);
  QEQ_CUDA_TRY(cudaGetLastError());
  return launch_fft_passes<float, false>(Pl, Pl->geo, Pl->fft_kmax, Pl->d_st, Pl->d_zitems, Pl->n_zitems,
                                        Pl->d_yitems, Pl->n_yitems, Pl->d_yiitems, Pl->n_yiitems, Pl->d_xitems,
                                        Pl->n_xitems, 0, mesh, reinterpret_cast<float2*>(Pl->d_mesh2),
                                        Pl->max_species, []() { return cudaSuccess; });
}

cudaError_t launch_mesh_potential32(qeq_plan_s* P, const double* x) {
  if (P->max_p == 4) return potential32_impl<4>(P, x);
  if (P->max_p == 6) return potential32_impl<6>(P, x);
  return potential32_impl<8>(P, x);
}

cudaError_t launch_mesh_potential(qeq_plan_s* P, const double* x) {
  if (P->max_p == 4) return potential_impl<4>(P, x);
  if (P->max_p == 6) return potential_impl<6>(P, x);
  return potential_impl<8>(P, x);
}

cudaError_t matvec_set_attributes() {
  QEQ_CUDA_TRY((set_smem_attrs<float, 4>()));
  QEQ_CUDA_TRY((set_smem_attrs<float, 6>()));
  QEQ_CUDA_TRY((set_smem_attrs<float, 8>()));
  QEQ_CUDA_TRY((set_smem_attrs<double, 4>()));
  QEQ_CUDA_TRY((set_smem_attrs<double, 6>()));
  QEQ_CUDA_TRY((set_smem_attrs<double, 8>()));
  QEQ_CUDA_TRY(cudaFuncSetAttribute(k_pre_spread_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
  QEQ_CUDA_TRY(set_smem_attrs_dd());
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
  if (P->precision == QEQ_MIXED && P->dd_check) {  // FP64-accurate product of a mixed plan, large meshes
    if (p == 4) return matvec_check_dd<4>(P, x, y, with_J, use_active, fuse_pAp, ev);
    if (p == 6) return matvec_check_dd<6>(P, x, y, with_J, use_active, fuse_pAp, ev);
    return matvec_check_dd<8>(P, x, y, with_J, use_active, fuse_pAp, ev);
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
  count_launch(P, 8);
  // fixed-point sums in the second coarse buffer (8 bytes per point, like the float2 mesh)
  unsigned long long* imesh = reinterpret_cast<unsigned long long*>(P->d_pmesh2);
  QEQ_CUDA_TRY(cudaMemsetAsync(imesh, 0, sizeof(unsigned long long) * (size_t)P->total_pmesh, s));
  k_pre_spread_tiles<<<P->n_pre_tiles, 256, P->pre_tile_smem, s>>>(
      P->d_st, P->d_stp, P->d_pre_tiles, P->pre_tile_gz, P->d_bin_start, P->d_pbase, P->d_pw, P->d_dinv, r, P->d_sc,
      use_active, slot == 1, imesh);
  {
    const int nb = (int)std::min<int64_t>((P->total_pmesh + 255) / 256, 148 * 16);
    k_pre_fixed_to_float<<<nb, 256, 0, s>>>(P->d_stp, P->n_struct, P->total_pmesh, P->d_sc, slot == 1, imesh,
                                            P->d_pmesh);
  }
  QEQ_CUDA_TRY(cudaGetLastError());
  QEQ_CUDA_TRY((launch_fft_passes<float, true>(P, P->pgeo, P->pfft_kmax, P->d_stp, P->d_pzitems, P->n_pz, P->d_pyitems, P->n_py,
                                               P->d_pyiitems, P->n_pyi, P->d_pxitems, P->n_px, use_active,
                                               P->d_pmesh, P->d_pmesh2, 1, []() { return cudaSuccess; })));
  k_pre_gather<<<P->n_chunks, 256, 0, s>>>(P->d_chunks, P->d_stp, P->d_pbase, P->d_pw, P->d_dinv, r, P->d_pmesh, P->d_sc,
                                           use_active, slot, u, P->d_part + (size_t)P->n_chunks * QEQ_MAX_SPECIES,
                                           P->d_counter + 3 * P->n_struct);
  return cudaGetLastError();
}
