// Internal declarations of libqeq: device tables, the plan object and the
// kernels' host launchers.  Not part of the public ABI (include/qeq.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qeq.h"

#define QEQ_MAX_SPECIES 8
#define QEQ_BIN 8          // mesh points per edge of an atom bin / spread-gather brick
#define QEQ_MAXP 8         // largest supported B-spline order
#define QEQ_MAX_STAGES 16  // radix stages of one FFT length
#define QEQ_CHUNK 2048     // atoms per reduction chunk (one CTA)

// ---------------------------------------------------------------------------
// Per-structure constants, built on the host by qeq_plan_create.
struct StructDev {
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
  int64_t mesh_off;       // complex-element offset of this structure's complex mesh 0
  int64_t atom_begin, atom_end;
  int bin_off;            // first global bin of this structure
  int fft_plan[3];        // FFT plan index per direction
  int bmod_off[3];        // offsets into the B-spline modulus table per direction
  int xpair_off;          // first entry of this structure in the x-pass line-pair table
  int pad_;
  double w2[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];     // reciprocal Gaussian width^2 w_st^2
  double corr[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES];   // G = 0 width term over r < r_cut (narrow pairs)
  double inv_sw[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES]; // 1/(sqrt2 w_st) (narrow pairs)
  double inv_sg[QEQ_MAX_SPECIES * QEQ_MAX_SPECIES]; // 1/(sqrt2 gamma_st) (narrow pairs)
  double self_s[QEQ_MAX_SPECIES];                   // k_e sqrt(2/pi)(1/gamma_ss - 1/w_ss)
  double diag_s[QEQ_MAX_SPECIES];                   // k_e/(sigma_s sqrt pi): Jacobi diagonal part
  uint32_t narrow[QEQ_MAX_SPECIES];                 // bit t set: pair (s,t) has a real-space term
};

struct FftPlanDev {
  int K;
  int nst;
  int radix[QEQ_MAX_STAGES];
  int tw_off;  // offset of exp(-2 pi i m / K), m < K, in the twiddle tables
  int pad_;
};

// Per-structure scalars of the PCG (device resident).
struct PcgScalars {
  double rz, rz_new, alpha, beta;
  double s0;          // sum_i 1/D_i
  double shift;       // (1^T D^-1 r)/(1^T D^-1 1)
  double qsum;
  double pAp;
  double r_sum, r_sq, r_max, r_min;   // residual statistics of the current r
  double tol_inf;     // stop threshold on max |P r|
  double tol_l2;      // optional stop threshold on ||P r||_2 (0 = off)
  double j_min;
  double q_tot;
  double chi_p2;      // ||P chi||_2^2
  double E_lin, E_quad, E_J;  // chi.q, q.Aq, q.Jq
  double xsum[QEQ_MAX_SPECIES];       // per-species sums of the matvec input
  int active;         // 1 while iterating
  int converged;      // 1 when the recursive residual meets the tolerance
  int iters;
  int restarts;
  int status;
  int n;
  int pad_[2];
};

// Atom-chunk for reductions: one CTA, atoms [begin, end) of one structure.
struct Chunk {
  int s;
  int last;     // 1 for the last chunk of its structure
  int64_t begin, end;
  int first;    // first chunk index of the structure
  int count;    // chunks of the structure
};

// ---------------------------------------------------------------------------
struct qeq_plan_s {
  qeq_plan_desc desc;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_struct = 0;
  int64_t n_atoms = 0;
  int precision = QEQ_FP64;
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
  int n_zitems = 0, n_yitems = 0, n_xitems = 0;
  int64_t workspace_bytes = 0;
  bool have_atoms = false;         // sorted atom data valid for profiling
  bool graph_ok = true;

  // device tables
  StructDev* d_st = nullptr;
  FftPlanDev* d_fft = nullptr;
  double2* d_tw64 = nullptr;
  float2* d_tw32 = nullptr;
  double* d_bmod = nullptr;
  float* d_bmod32 = nullptr;
  int max_ncm = 1;                 // largest complex-mesh count of any structure
  int ly = 8;                      // lines per y-pass item
  int64_t fft_smem_elems = 0;      // complex elements of shared memory per FFT CTA
  int4* d_zitems = nullptr;
  int4* d_yitems = nullptr;
  int4* d_xitems = nullptr;
  int2* d_xpairs = nullptr;
  int* d_bin_struct = nullptr;     // structure of each global bin
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
  // real-space pair list (CSR over sorted atoms)
  int64_t* d_row = nullptr;        // N+1
  int* d_row_cnt = nullptr;        // N
  int* d_col = nullptr;
  double* d_val64 = nullptr;
  float* d_val32 = nullptr;
  // vectors (sorted order)
  double *d_q = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_Ap = nullptr, *d_x = nullptr;
  // mesh (reinterpreted as float2 in mixed precision)
  double2* d_mesh = nullptr;
  // reductions
  double* d_part = nullptr;        // n_chunks * 16 partials
  int* d_counter = nullptr;        // n_struct counters for last-block reductions
  PcgScalars* d_sc = nullptr;
  int* d_err = nullptr;            // device error bits
  int* d_done = nullptr;           // all-structures-inactive flag
  int* h_done = nullptr;           // pinned mirror
  cudaEvent_t ev_done = nullptr;
  int64_t launches = 0;            // kernels launched by this plan (graph replays count their kernels)
  int64_t graph_kernels = 0;       // kernels inside the captured iteration graph
  bool capturing = false;
  cudaGraphExec_t graph_iter = nullptr;
  int graph_iter_prec = -1;
  int graph_iter_k = 0;
};

// device error bits
enum {
  ERRBIT_NONFINITE = 1,
  ERRBIT_SPECIES = 2,
  ERRBIT_J = 4,
  ERRBIT_PAIRCAP = 8,
  ERRBIT_SORT = 16,
};

// ---------------------------------------------------------------------------
// launchers (prep.cu)
cudaError_t launch_prepare_atoms(qeq_plan_s* P, const double* pos, const int32_t* species,
                                 const double* chi, const double* J, int need_pairs);
// launchers (matvec.cu)
cudaError_t launch_matvec(qeq_plan_s* P, int prec, const double* x, double* y, int with_J,
                          int use_active, int fuse_pAp, cudaEvent_t* ev /* QEQ_N_STAGES+1 or NULL */);
cudaError_t matvec_set_attributes();

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
