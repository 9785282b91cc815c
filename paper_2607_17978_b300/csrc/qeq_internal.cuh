// Internal declarations of libqeq: device tables, the plan object and the
// kernels' host launchers.  Not part of the public ABI (include/qeq.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "qeq.h"

#define QEQ_MAX_SPECIES 8
#define QEQ_BIN 8          // mesh points per edge of an atom bin (sorting, real-space search)
#define QEQ_BRICK_XY 16    // spread brick: mesh points in x and y (2 x 2 bins) ...
#define QEQ_BRICK_Z 16     // ... and in z (2 bins)
#define QEQ_BRICK_CAND 28  // per brick: candidate-bin counts per direction (3, pad), bins (3 x 8)
#define QEQ_MAXP 8         // largest supported B-spline order
#define QEQ_MAX_STAGES 12  // radix stages of one FFT length
#ifndef QEQ_CHUNK
#define QEQ_CHUNK 512      // atoms per reduction chunk (one CTA)
#endif
#define QEQ_GATHER_SPLIT_MAX 64  // gather CTAs per reduction chunk

// ---------------------------------------------------------------------------
// Per-structure constants, built on the host by qeq_plan_create.
struct StructDev {
  double pre_g0max;       // preconditioner mesh: largest g0(m), at the smallest nonzero |G|
  double h[9];            // cell rows a1 a2 a3
  double hinv[9];         // h^{-1}: fractional u = r h^{-1}
  double B[9];            // rows 2 pi b_k: G(m) = m0 B[0..2] + m1 B[3..5] + m2 B[6..8]
  double V;
  double green_pref;      // k_e * 4 pi / V
  double r_cut, omega;
  int K[3];               // mesh points per lattice direction
  int nb[3];              // atom bins per direction (ceil(K/QEQ_BIN))
  int rs_range[3];        // bin range searched for real-space pairs
  int S;                  // species of this structure
  int ncm;                // complex meshes = ceil(S/2): species 2c in Re, 2c+1 in Im
  int p;                  // B-spline order
  int any_narrow;         // 1 if some species pair has a real-space term
  int64_t M;              // K0*K1*K2
  int64_t Mp;             // elements per complex mesh in memory (padded layouts, even)
  int64_t mesh_off;       // complex-element offset of this structure's complex mesh 0
  int64_t atom_begin, atom_end;
  int bin_off;            // first global bin of this structure
  int fft_plan[3];        // FFT plan index per direction (FP32 stages; the FP64 and the double-float plans follow it)
  int bmod_off[3];        // offsets into the B-spline modulus table per direction
  int P[3];               // padded line lengths K_d + (K_d & 1) (innermost stride of each layout)
  int brick_off;          // first global brick of this structure
  int nbr[3];             // spread bricks per direction
  double w2[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];     // reciprocal Gaussian width^2 w_st^2
  double corr[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];   // G = 0 width term over r < r_cut (narrow pairs)
  double inv_sw[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES]; // 1/(sqrt2 w_st) (narrow pairs)
  double inv_sg[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES]; // 1/(sqrt2 gamma_st) (narrow pairs)
  double self_s[QEQ_MAX_SPECIES];                   // k_e sqrt(2/pi)(1/gamma_ss - 1/w_ss)
  double diag_s[QEQ_MAX_SPECIES];                   // k_e/(sigma_s sqrt pi): Jacobi diagonal part
  uint32_t narrow[QEQ_MAX_SPECIES];                 // bit t set: pair (s,t) has a real-space term
  double sigma_s[QEQ_MAX_SPECIES];                  // Gaussian width per species
  int feat_range[3];                                // bins searched for descriptor neighbours
  int pad3_;
};

// ---------------------------------------------------------------- host cell geometry
inline double det3(const double* h) {
  return h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
         h[2] * (h[3] * h[7] - h[4] * h[6]);
}

// inverse of the row-major 3x3 matrix h
inline void inv3(const double* h, double* hi) {
  double d = det3(h);
  hi[0] = (h[4] * h[8] - h[5] * h[7]) / d;
  hi[1] = (h[2] * h[7] - h[1] * h[8]) / d;
  hi[2] = (h[1] * h[5] - h[2] * h[4]) / d;
  hi[3] = (h[5] * h[6] - h[3] * h[8]) / d;
  hi[4] = (h[0] * h[8] - h[2] * h[6]) / d;
  hi[5] = (h[2] * h[3] - h[0] * h[5]) / d;
  hi[6] = (h[3] * h[7] - h[4] * h[6]) / d;
  hi[7] = (h[1] * h[6] - h[0] * h[7]) / d;
  hi[8] = (h[0] * h[4] - h[1] * h[3]) / d;
}

// x with erfc(x) = y, by bisection (erfc is decreasing)
inline double erfc_inv(double y) {
  double lo = 0.0, hi = 30.0;
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (erfc(mid) > y)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

// perpendicular distances between opposite faces of the cell
inline void plane_widths(const double* h, double V, double* wd) {
  for (int d = 0; d < 3; ++d) {
    const double* a1 = h + 3 * ((d + 1) % 3);
    const double* a2 = h + 3 * ((d + 2) % 3);
    double cx = a1[1] * a2[2] - a1[2] * a2[1], cy = a1[2] * a2[0] - a1[0] * a2[2], cz = a1[0] * a2[1] - a1[1] * a2[0];
    wd[d] = V / sqrt(cx * cx + cy * cy + cz * cz);
  }
}

// Division by a runtime-invariant divisor d with a multiply and a shift
// (round-up method of Granlund & Montgomery): n / d = (umulhi(n, m) + n) >> s
// for 0 <= n < 2^31.
struct FastDiv {
  uint32_t d, m, s;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  f.s = s;
  f.m = (uint32_t)(((((1ull << s) - d) << 32) / d) + 1);
  return f;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) { return (__umulhi(n, f.m) + n) >> f.s; }

// Cardinal B-spline values M_p(w + j), j = 0..p-1, w in [0,1), by the order recursion
// M_n(x) = [x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)] / (n - 1), starting from M_2.
__device__ __forceinline__ void bspline_weights(double w, int p, double* out) {
  double a[QEQ_MAXP];
  a[0] = w;
  a[1] = 1.0 - w;
  for (int n = 2; n < p; ++n) {  // a[j] = M_n(w + j), j < n  ->  M_{n+1}
    double inv = 1.0 / n;
    a[n] = 0.0;
    for (int j = n; j >= 0; --j) {
      double x = w + j;
      double left = a[j];
      double right = (j > 0) ? a[j - 1] : 0.0;
      a[j] = (x * left + (n + 1 - x) * right) * inv;
    }
  }
  for (int j = 0; j < p; ++j) out[j] = a[j];
}
#endif

// Mixed-radix plan of one FFT length K = R_0 ... R_{m-1} (see fft.cuh): stage s has
// Q_s = R_0...R_{s-1} blocks of L_s = K/Q_s points and stride S_s = L_s/R_s.
struct alignas(16) FftPlanDev {
  int K;
  int nst;
  int radix[QEQ_MAX_STAGES];
  int S[QEQ_MAX_STAGES];
  int L[QEQ_MAX_STAGES];
  int Q[QEQ_MAX_STAGES];
  FastDiv fnb[QEQ_MAX_STAGES];  // K / R_s
  FastDiv fS[QEQ_MAX_STAGES];   // S_s
  FastDiv fK;                   // K
  int tw_off;   // offset of exp(-2 pi i m / K), m < K, in the twiddle tables (even)
  int tab_off;  // int tables, K4 = K rounded up to 4: blk[K/R_{m-1}] at tab_off, freq[K] at +K4, pos[K] at +2 K4
};
static_assert(sizeof(FftPlanDev) % 16 == 0, "FFT plans are bulk-copied");

// One buffer of the FFT passes' shared-memory pipeline (fft.cuh): the unit's FFT plan,
// its twiddles (even count), ntab int tables of K4 entries, `extra` bytes of per-unit
// tables, and the line tile.  Offsets in bytes from the buffer start.
struct FftBuf {
  int tw, tab, extra, tile, bytes;
};
__host__ __device__ inline int fft_align(int x, int a) { return (x + a - 1) / a * a; }
__host__ __device__ inline FftBuf fft_buf(int Kmax, int ldmax, int lines, int elem, int ntab, int extra) {
  FftBuf b;
  b.tw = fft_align((int)sizeof(FftPlanDev), 16);
  b.tab = b.tw + (Kmax + (Kmax & 1)) * elem;
  b.extra = b.tab + ntab * ((Kmax + 3) & ~3) * 4;
  b.tile = fft_align(b.extra + extra, 128);
  b.bytes = fft_align(b.tile + lines * ldmax * elem, 128);
  return b;
}
// per-unit tables of the x pass: input and output line offsets of 2 hx sub slots, 4 line
// constants per pair
__host__ __device__ inline int fft_x_extra(int sub, int hx, int real) {
  return 2 * 2 * hx * sub * 8 + sub * 4 * real;
}

// Per-structure scalars of the PCG (device resident).
struct PcgScalars {
  double rz, rz_new, alpha, beta;
  double s0;          // sum_i 1/D_i
  double shift;       // (1^T D^-1 r)/(1^T D^-1 1)
  double qsum;
  double pAp;
  double r_sum, r_l2, r_max, r_min;   // statistics of the current r: sum, ||P r||_2, max, min
  double tol_inf;     // stop threshold on max |P r|
  double tol_l2;      // optional stop threshold on ||P r||_2 (0 = off)
  double inner;       // factor on both thresholds for the iteration's own (recurrence) residual
  double j_min;
  double q_tot;
  double chi_p2;      // ||P chi||_2^2
  double chi_sum;     // sum chi
  double usum;        // sum of the last preconditioned residual (Fourier preconditioner)
  double w1sum;       // sum of M^-1 1
  double E_lin, E_quad, E_J;  // chi.q, q.Aq, q.Jq
  double xsum[QEQ_MAX_SPECIES];       // per-species sums of the matvec input
  double slack;       // bound on the error of the checked residual (0 for an FP64 check)
  double dmax, dmaxD; // max |q - q1| and max D_i since the last FP64 check
  double dinv_max;    // max_i 1/D_i (scale of the fixed-point coarse spread)
  int active;         // 1 while iterating
  int converged;      // 1 when the recursive residual meets the tolerance
  int iters;
  int restarts;
  int status;
  int n;
  int jacobi;         // 1: the Fourier preconditioner was dropped for Jacobi
  double drop;        // mixed precision: a round of FP32 iterations ends once its residual fell by this factor
  double floor_inf, floor_l2;  // ... below the residual of the round's check (0 in FP64)
  int unconstrained;  // 1: plain PCG on (E + diag J) x = b, no charge constraint (two-RHS solver)
  double tsum;        // two-RHS solver: sum of t (A t = 1)
};

// Stabilised quasi-Newton minimiser (QEQ_FLAG_SQNM): per-structure state.  Vectors live in
// Jacobi-scaled coordinates x = D^{1/2} q; slots 0..QEQ_SQNM_HISTORY-1 hold the last steps dx
// and gradient changes dg.
#define QEQ_SQNM_HISTORY 8
#define QEQ_SQNM_NDOT (5 * QEQ_SQNM_HISTORY + 1)  // dot products per iteration
struct SqnmState {
  double XX[QEQ_SQNM_HISTORY][QEQ_SQNM_HISTORY];  // dx_i . dx_j
  double XG[QEQ_SQNM_HISTORY][QEQ_SQNM_HISTORY];  // dx_i . dg_j
  double GG[QEQ_SQNM_HISTORY][QEQ_SQNM_HISTORY];  // dg_i . dg_j
  double gX[QEQ_SQNM_HISTORY];                    // g . dx_i (current gradient)
  double coef[QEQ_SQNM_HISTORY];                  // step coefficients of dx_i
  double gg;                                      // g . g
  double alpha;                                   // steepest-descent step length in the complement
  double E, E_prev;                               // energy at the current and at the previous point
  double c;                                       // D-weighted mean of A q + chi (the projection)
  int count;                                      // history entries in use
  int head;                                       // slot of the newest entry
  int has_prev;                                   // a previous gradient exists
  int subspace;                                   // significant directions used by the last step
  int revert;                                     // 1: the last step raised the energy and is undone
  int pad_;
};

// Loop counters of the device-paced solve graph (device resident).
struct LoopCtl {
  int outer;          // PCG rounds done in this solve (a round ends with a final check)
  int replays_round;  // replays of the 4-iteration body in this round
  int replays_total;  // ... in this solve
  int pad_;
};

// Atom-chunk for reductions: one CTA, atoms [begin, end) of one structure.
struct Chunk {
  int s;
  int last;     // 1 for the last chunk of its structure
  int64_t begin, end;
  int first;    // first chunk index of the structure
  int count;    // chunks of the structure
};

// Tile sizes of the FFT passes of one set of meshes: item lines (tl, tlx) and, per
// precision, lines per shared-memory tile (sub, subx) with the maximal shared-line
// lengths (ld*) the kernels' dynamic shared memory is sized for.
struct FftGeom {
  int tl = 1, tlx = 1;
  int sub32 = 1, sub64 = 1, subx32 = 1, subx64 = 1;
  int ldz32 = 0, ldz64 = 0, ldy32 = 0, ldy64 = 0, ldx32 = 0, ldx64 = 0;
  int max_ncm = 1;
};

// ---------------------------------------------------------------------------
struct qeq_plan_s {
  qeq_plan_desc desc;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_struct = 0;
  int64_t n_atoms = 0;
  int precision = QEQ_FP64;
  int dd_check = 0;                // mixed plans: FP64-accurate products with double-float FFT passes
  int max_S = 0, max_p = 6;
  std::string last_error;
  std::vector<StructDev> hs;       // host copies
  std::vector<FftPlanDev> hfft;
  std::vector<int64_t> offsets;
  std::vector<double> qtot_h;
  int total_bins = 0;
  int64_t total_mesh = 0;          // complex elements over all structures and complex meshes
  int64_t pair_cap = 0;
  int n_chunks = 0;
  int n_zitems = 0, n_yitems = 0, n_yiitems = 0, n_xitems = 0;
  int64_t workspace_bytes = 0;
  bool have_atoms = false;         // sorted atom data valid for profiling
  bool graph_ok = true;
  int test_stall = 0;              // QEQ_FLAG_TEST_STALL: one x-pass tile's bounded wait runs out

  // device tables
  StructDev* d_st = nullptr;
  FftPlanDev* d_fft = nullptr;
  double2* d_tw64 = nullptr;
  float2* d_tw32 = nullptr;
  double* d_bmod = nullptr;
  float* d_bmod32 = nullptr;
  float* d_bmod_dd = nullptr;      // hi, lo pairs of d_bmod (double-float passes)
  int* d_fft_tabs = nullptr;       // per FFT length: block offsets, frequency of position, position of frequency
  int max_ncm = 1;                 // largest complex-mesh count of any structure
  FftGeom geo;                     // tile sizes of the FFT passes of the matvec mesh
  FftGeom pgeo;                    // ... of the preconditioner mesh
  int num_sms = 148;
  struct OccEntry {
    const void* fn;
    size_t smem;
    int blocks;
  } occ[24];                       // resident CTAs per SM of the persistent FFT kernels (no heap)
  int n_occ = 0;
  int fft_kmax[3] = {1, 1, 1};     // largest mesh size per direction (matvec mesh)
  int pfft_kmax[3] = {1, 1, 1};    // ... (preconditioner mesh)
  int4* d_zitems = nullptr;        // z passes {s, c, x, y0}
  int4* d_yitems = nullptr;        // forward y pass {s, c, z, x0}
  int4* d_yiitems = nullptr;       // inverse y pass {s, c, x, z0}
  int4* d_xitems = nullptr;        // x pass {s, z, y0, lines}
  int* d_xitem_off = nullptr;      // n_struct + 1: first x item of each structure
  double* d_stress_part = nullptr; // per-chunk partial sums of the strain derivative (6 + 2 QEQ_MAX_SPECIES each)
  // SQNM solver (QEQ_FLAG_SQNM only): history dx, dg (QEQ_SQNM_HISTORY x N each), the
  // scaled gradient (N), per-chunk partial dot products, per-structure state
  double *d_sqnm_dx = nullptr, *d_sqnm_dg = nullptr, *d_sqnm_g = nullptr, *d_sqnm_part = nullptr;
  SqnmState* d_sqnm = nullptr;
  int* d_bin_struct = nullptr;     // structure of each global bin
  int* d_brick_struct = nullptr;   // structure of each global brick
  int* d_brick_cand = nullptr;     // QEQ_BRICK_CAND ints per brick (brick_candidates)
  int total_bricks = 0;
  int* d_atom_struct = nullptr;    // structure of each atom (input order)
  Chunk* d_chunks = nullptr;
  // per-solve atom data (sorted order)
  int* d_key = nullptr;            // bin of each input atom
  int* d_bin_count = nullptr;      // total_bins + 1
  int* d_bin_start = nullptr;      // total_bins + 1
  int* d_bin_fill = nullptr;
  int* d_perm = nullptr;           // sorted -> input index
  int* d_scan_tmp = nullptr;
  int* d_base = nullptr;           // packed stencil base indices
  double* d_wts = nullptr;         // B-spline weights, 3*p per atom (FP64)
  float* d_wts32 = nullptr;        // same in FP32
  int* d_spec = nullptr;           // species, sorted
  double* d_J = nullptr;           // hardness, sorted
  double* d_chi = nullptr;
  double* d_dinv = nullptr;        // 1/D_i
  double* d_posc = nullptr;        // Cartesian, wrapped, sorted, 3 per atom
  float4* d_posc32 = nullptr;      // the same in FP32 (x, y, z, 0), for the neighbour-walk distance tests
  // real-space pair list (CSR over sorted atoms)
  int64_t* d_row = nullptr;        // N+1
  int* d_row_cnt = nullptr;        // N
  int* d_col = nullptr;
  double* d_val64 = nullptr;
  float* d_val32 = nullptr;
  // vectors (sorted order)
  double *d_q = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_Ap = nullptr, *d_x = nullptr;
  double *d_q1 = nullptr, *d_r1 = nullptr;  // charges and FP64 residual at the last FP64 check
  float* d_x32 = nullptr;          // FP32 copy of the matvec input (mixed precision), written by the species sums
  // mesh (reinterpreted as float2 in mixed precision)
  double2* d_mesh = nullptr;       // layouts L0 / L2 (see fft.cuh)
  double2* d_mesh2 = nullptr;      // layouts L1 / L3
  // reductions
  double* d_part = nullptr;        // partials: species sums, gather x.y, PCG reductions
  int* d_counter = nullptr;        // n_struct counters for last-block reductions
  PcgScalars* d_sc = nullptr;
  int* d_err = nullptr;            // device error bits
  int* d_done = nullptr;           // all-structures-inactive flag
  int* d_reject = nullptr;         // n_struct: 1 where the network start was rejected
  int* h_done = nullptr;           // pinned mirror
  cudaEvent_t ev_done = nullptr;
  // Fourier preconditioner (coarse mesh per structure)
  int precond = QEQ_PRECOND_JACOBI;
  std::vector<StructDev> hsp;
  StructDev* d_stp = nullptr;
  int4 *d_pzitems = nullptr, *d_pyitems = nullptr, *d_pyiitems = nullptr, *d_pxitems = nullptr;
  int n_pz = 0, n_py = 0, n_pyi = 0, n_px = 0;
  int64_t total_pmesh = 0;
  int gather_split = 1;            // CTAs per reduction chunk in the gather
  int max_species = QEQ_MAX_SPECIES;  // most species of any structure
  float2 *d_pmesh = nullptr, *d_pmesh2 = nullptr;
  double *d_w1 = nullptr, *d_u = nullptr;
  int* d_pbase = nullptr;
  float* d_pw = nullptr;
  int4* d_pre_tiles = nullptr;     // coarse-spread tile groups {structure, bx0, by0, bz0} (pre_tile_range)
  int n_pre_tiles = 0;
  int pre_tile_gz = 0;             // fine bins per tile group in z (QEQ_PRE_TILE_G in x and y)
  int pre_tile_smem = 0;           // bytes of the largest tile (8 bytes per point)
  struct qeq_mlp_s* mlp = nullptr; // warm-start network (not owned)
  float* d_feat = nullptr;         // descriptors, sorted order
  float* d_pred = nullptr;         // network output, sorted order
  int64_t launches = 0;            // kernels launched by this plan (graph replays count their kernels)
  int64_t graph_kernels = 0;       // kernels counted while capturing a graph segment
  bool capturing = false;
  // device-paced solve: one graph per precision holding every PCG round (see solve.cu)
  cudaGraphExec_t graph_solve = nullptr;
  int graph_solve_prec = -1;
  int64_t gk_inner = 0, gk_round = 0;  // kernels per inner body replay / per round outside it
  struct LoopCtl* d_ctl = nullptr;     // device loop counters of the solve graph
};

// Register butterflies: FP32 stages use radices up to 24 (larger ones spill at the
// 128-register budget of two 256-thread CTAs per SM), FP64 stages up to 16.
#define QEQ_MAXR32 24
#define QEQ_MAXR64 16

// depth-first search of fft_radices: ordered factorisations of rem into register radices
// no larger than maxR, no deeper than the best found so far
inline void fft_radices_search(int rem, int d, int* cur, int* best, int& nbest, int maxR) {
  static const int kR[] = {24, 20, 18, 16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  if (rem == 1) {
    if (d == 0) return;
    bool take = nbest < 0 || d < nbest;
    if (!take && d == nbest) {
      const bool co = cur[d - 1] & 1, bo = best[nbest - 1] & 1;
      if (co != bo) {
        take = co;
      } else {
        for (int i = 0; i < d; ++i)
          if (cur[i] != best[i]) {
            take = cur[i] > best[i];
            break;
          }
      }
    }
    if (take) {
      for (int i = 0; i < d; ++i) best[i] = cur[i];
      nbest = d;
    }
    return;
  }
  if (d >= QEQ_MAX_STAGES || (nbest >= 0 && d >= nbest)) return;
  for (int r : kR)
    if (r <= maxR && rem % r == 0) {
      cur[d] = r;
      fft_radices_search(rem / r, d + 1, cur, best, nbest, maxR);
    }
}

// Radices of the FFT stages of length K (K = 2^a 3^b 5^c): the ordered factorisation
// into register butterflies (2 ... maxR) with the fewest stages; among those an odd last
// radix (its contiguous shared-memory reads spread over the banks), then the
// lexicographically largest.  Returns the number of stages, -1 if none.
inline int fft_radices(int K, int* out, int maxR) {
  int best[QEQ_MAX_STAGES] = {0}, cur[QEQ_MAX_STAGES] = {0}, nbest = -1;
  if (K < 2) return -1;
  fft_radices_search(K, 0, cur, best, nbest, maxR);
  for (int i = 0; i < nbest; ++i) out[i] = best[i];
  return nbest;
}

// Stage constants, twiddles (K entries each, from tw_off) and the int tables (3 K4
// entries, K4 = K rounded up to 4, from tab_off: block offset of each natural base u,
// frequency of each block-order position, block-order position of each frequency) of
// one FFT length.
inline bool fft_plan_fill(int K, FftPlanDev& f, double2* tw64, float2* tw32, int* tab, int maxR) {
  f.K = K;
  f.nst = fft_radices(K, f.radix, maxR);
  if (f.nst < 1) return false;
  int Q = 1;
  for (int s = 0; s < f.nst; ++s) {
    f.Q[s] = Q;
    f.L[s] = K / Q;
    f.S[s] = f.L[s] / f.radix[s];
    f.fnb[s] = make_fastdiv(K / f.radix[s]);
    f.fS[s] = make_fastdiv(f.S[s]);
    Q *= f.radix[s];
  }
  f.fK = make_fastdiv(K);
  const double kTwoPi = 6.28318530717958647692;
  for (int m = 0; m < K; ++m) {
    const double ang = -kTwoPi * (double)m / K;
    tw64[m] = make_double2(cos(ang), sin(ang));
    tw32[m] = make_float2((float)cos(ang), (float)sin(ang));
  }
  // every digit tuple (k_0 .. k_{m-1}): position sum_s S_s k_s, frequency sum_s Q_s k_s
  const int m = f.nst;
  int k[QEQ_MAX_STAGES] = {0};
  for (int t = 0; t < K; ++t) {
    int p = 0, fq = 0;
    for (int s = 0; s < m; ++s) {
      p += f.S[s] * k[s];
      fq += f.Q[s] * k[s];
    }
    const int K4 = (K + 3) & ~3;
    tab[K4 + p] = fq;
    tab[2 * K4 + fq] = p;
    if (k[m - 1] == 0) tab[fq] = p;  // natural base u = fq (last digit 0) -> its block's offset
    for (int s = 0; s < m; ++s) {   // next tuple, digit 0 fastest
      if (++k[s] < f.radix[s]) break;
      k[s] = 0;
    }
  }
  return true;
}

// Padded line lengths and the per-complex-mesh size of the four layouts (fft.cuh).
inline void mesh_layout(StructDev& T) {
  for (int d = 0; d < 3; ++d) T.P[d] = T.K[d] + (T.K[d] & 1);
  const int64_t K0 = T.K[0], K1 = T.K[1], K2 = T.K[2];
  int64_t m = K0 * K1 * T.P[2];
  m = std::max(m, K0 * K2 * (int64_t)T.P[1]);
  m = std::max(m, K2 * K1 * (int64_t)T.P[0]);
  T.M = K0 * K1 * K2;
  T.Mp = m;
}

// Shared-memory line strides as the kernels compute them (fft.cuh fft_smem_ld).
inline int fft_ld32(int K) {
  int ld = K + (K & 1);
  return (ld & 3) ? ld : ld + 2;
}
inline int fft_ld64(int K) { return K | 1; }

// Coarse-spread tiles of the Fourier preconditioner: a group of G consecutive fine atom
// bins in one direction (bins b0 .. b0 + G - 1 of nb, QEQ_BIN fine points each, fine length
// Kf) holds atoms whose coarse stencil base f = floor(u Kc) lies in [f0, f1], f0 =
// floor(QEQ_BIN b0 Kc / Kf), f1 = floor(QEQ_BIN (b0 + G) Kc / Kf); their cubic stencils
// (points f - 3 .. f) fill coarse points o .. o + ext - 1 (mod Kc), with one point of margin
// on each side for the rounding of u.  The whole direction when that is no larger.
#define QEQ_PRE_TILE_G 2
__host__ __device__ inline void pre_tile_range(int b0, int G, int nb, int Kc, int Kf, int& o, int& ext) {
  const int b1 = (b0 + G < nb) ? b0 + G : nb;
  const int f0 = (int)(((long long)QEQ_BIN * b0 * Kc) / Kf);
  const int f1 = (int)(((long long)QEQ_BIN * b1 * Kc) / Kf);
  ext = f1 - f0 + 6;
  o = f0 - 4;
  if (ext >= Kc) {
    o = 0;
    ext = Kc;
  } else if (o < 0) {
    o += Kc;
  }
}

// Tile sizes for meshes whose largest sizes per direction are maxK[3] (most complex
// meshes max_ncm): item lines of the y/z passes and of the x pass (2 max_ncm lines per
// pair); FP64 sub-tiles hold half as many lines (the same bytes).
#ifndef QEQ_FFT_MAX_LINES
#define QEQ_FFT_MAX_LINES 64
#endif
#ifndef QEQ_FFT_POW2
#define QEQ_FFT_POW2 1  // line counts rounded down to powers of two (the stores group lines so)
#endif
#ifndef QEQ_FFT_BUDGET_KB
#define QEQ_FFT_BUDGET_KB 36  // lines per FFT buffer (two buffers per CTA, two CTAs per SM)
#endif
inline FftGeom fft_geometry(const int* maxK, int max_ncm) {
  FftGeom g;
  g.max_ncm = max_ncm;
  g.ldz32 = fft_ld32(maxK[2]);
  g.ldz64 = fft_ld64(maxK[2]);
  g.ldy32 = fft_ld32(maxK[1]);
  g.ldy64 = fft_ld64(maxK[1]);
  g.ldx32 = fft_ld32(maxK[0]);
  g.ldx64 = fft_ld64(maxK[0]);
  // two buffers per CTA and two CTAs per SM: about 36 KB of lines per buffer, as many
  // lines per work unit as fit (short lines: up to 64, so that a unit's stages and barriers
  // cover enough points)
  const int ldyz = std::max(g.ldz32, g.ldy32);
  const int64_t budget = (int64_t)QEQ_FFT_BUDGET_KB * 1024;
  int tl = (int)std::max<int64_t>(1, std::min<int64_t>(QEQ_FFT_MAX_LINES, budget / ((int64_t)ldyz * 8)));
  if (QEQ_FFT_POW2)
    while (tl & (tl - 1)) tl &= tl - 1;  // largest power of two not above
  g.tl = tl;
  g.sub32 = tl;
  g.sub64 = std::max(1, tl / 2);
  int tlx = (int)std::max<int64_t>(1, std::min<int64_t>(QEQ_FFT_MAX_LINES / 2,
                                                         budget / ((int64_t)2 * max_ncm * g.ldx32 * 8)));
  if (QEQ_FFT_POW2)
    while (tlx & (tlx - 1)) tlx &= tlx - 1;
  g.tlx = tlx;
  g.subx32 = tlx;
  g.subx64 = std::max(1, tlx / 2);
  return g;
}

// Candidate bins of spread brick (bc0, bc1, bc2) of structure T with B-spline order p: per
// direction the distinct bins of the positions x0 .. x0 + ext + p - 2 (mod K) in order, the
// bins that can hold an atom whose stencil reaches the brick.  out: QEQ_BRICK_CAND ints,
// counts at 0..2, bins of direction d at 4 + 8 d.
inline void brick_candidates(const StructDev& T, int p, const int* bc, int* out) {
  for (int i = 0; i < QEQ_BRICK_CAND; ++i) out[i] = 0;
  for (int d = 0; d < 3; ++d) {
    const int e = (d == 2) ? QEQ_BRICK_Z : QEQ_BRICK_XY;
    const int x0 = bc[d] * e, ext = std::min(e, T.K[d] - x0);
    const int span = std::min(ext + p - 1, T.K[d]);
    int nc = 0;
    for (int k = 0; k < span; ++k) {
      const int bn = ((x0 + k) % T.K[d]) / QEQ_BIN;
      bool seen = false;
      for (int q = 0; q < nc; ++q) seen |= (out[4 + 8 * d + q] == bn);
      if (!seen && nc < 8) out[4 + 8 * d + nc++] = bn;
    }
    out[d] = nc;
  }
}

// Work lists of the FFT passes of one structure (shared by qeq_plan_create and the
// allocation-free entry point).  Z items {s, c, x, y0} and inverse-y items {s, c, x, z0},
// forward-y items {s, c, z, x0} cover tl lines; x items {s, z, y0, lines} cover up to
// tlx lines (z <= K2/2, and y <= K1/2 on the planes that are their own mirror).
template <class AddZ, class AddY, class AddYI, class AddX>
inline void fft_work_lists(const StructDev& T, int s, int tl, int tlx, AddZ addz, AddY addy, AddYI addyi,
                           AddX addx) {
  const int K0 = T.K[0], K1 = T.K[1], K2 = T.K[2];
  for (int c = 0; c < T.ncm; ++c)
    for (int x = 0; x < K0; ++x)
      for (int y0 = 0; y0 < K1; y0 += tl) addz(make_int4(s, c, x, y0));
  for (int c = 0; c < T.ncm; ++c)
    for (int z = 0; z < K2; ++z)
      for (int x0 = 0; x0 < K0; x0 += tl) addy(make_int4(s, c, z, x0));
  for (int c = 0; c < T.ncm; ++c)
    for (int x = 0; x < K0; ++x)
      for (int z0 = 0; z0 < K2; z0 += tl) addyi(make_int4(s, c, x, z0));
  for (int z = 0; 2 * z <= K2; ++z) {
    const bool self = (z == 0) || (2 * z == K2);
    const int ylast = self ? K1 / 2 : K1 - 1;
    for (int y0 = 0; y0 <= ylast; y0 += tlx) addx(make_int4(s, z, y0, std::min(tlx, ylast + 1 - y0)));
  }
}

// device error bits
enum {
  ERRBIT_NONFINITE = 1,
  ERRBIT_SPECIES = 2,
  ERRBIT_J = 4,
  ERRBIT_PAIRCAP = 8,
  ERRBIT_SORT = 16,
  ERRBIT_TIMEOUT = 32,  // a bounded device wait ran out
};

// ---------------------------------------------------------------------------
// launchers (prep.cu)
cudaError_t launch_prepare_atoms(qeq_plan_s* P, const double* pos, const int32_t* species,
                                 const double* chi, const double* J, int need_pairs);
// launchers (matvec.cu)
cudaError_t launch_matvec(qeq_plan_s* P, int prec, const double* x, double* y, int with_J,
                          int use_active, int fuse_pAp, cudaEvent_t* ev /* QEQ_N_STAGES+1 or NULL */);
cudaError_t matvec_set_attributes();
// FP64 potential meshes of x (sorted order) in d_mesh, layout L0 (no gather)
cudaError_t launch_mesh_potential(qeq_plan_s* P, const double* x);
// the same in FP32 (x converted into d_x32; FP32 meshes in d_mesh, layout L0)
cudaError_t launch_mesh_potential32(qeq_plan_s* P, const double* x);
// strain-derivative sums of the reciprocal quadratic form of x (FP64): 8 doubles per x-pass
// unit in d_mesh2; *nsub_out = units per x item
cudaError_t launch_mesh_virial(qeq_plan_s* P, const double* x, int* nsub_out);
// launchers (forces.cu): force-trick forces and embedding potentials (input order in and out)
cudaError_t launch_forces(qeq_plan_s* P, const double* q, const double* lambda, double* F);
cudaError_t launch_embedding(qeq_plan_s* P, const double* q, double* Gamma);
// D[9 s + 3 a + b] = d/d eps_ab [(q/2 + lambda)^T E q] per structure (lambda may be NULL)
cudaError_t launch_stress(qeq_plan_s* P, const double* q, const double* lambda, double* D);
cudaError_t launch_precond_setup(qeq_plan_s* P);
// u = M^-1 r for the Fourier preconditioner; sum of u per structure into usum (slot 0) or w1sum (slot 1)
cudaError_t launch_precond(qeq_plan_s* P, const double* r, double* u, int slot, int use_active);
// launchers (mlp.cu)
cudaError_t launch_mlp_warm_start(qeq_plan_s* P, double* d_q_sorted);

// Deterministic block-wide sum of part[(first + i) * stride + k], i < count:
// thread t adds the entries i = t, t + blockDim, ... in order, each warp combines
// its lanes with a fixed shuffle tree and thread 0 adds the warp sums in order.
// Every thread must call it; the result is valid in thread 0.  red: blockDim.x/32
// doubles of shared memory.
__device__ __forceinline__ double ordered_block_sum(const double* part, int first, int count, int stride, int k,
                                                    double* red) {
  double a = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) a += ((const volatile double*)part)[(size_t)(first + i) * stride + k];
  // fixed shuffle tree inside each warp, then the warp sums in warp order
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
  __syncthreads();
  return tot;
}

inline void count_launch(qeq_plan_s* P, int n = 1) {
  if (P->capturing)
    P->graph_kernels += n;
  else
    P->launches += n;
}

#define QEQ_CUDA_TRY(expr)                  \
  do {                                      \
    cudaError_t e_ = (expr);                \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)
