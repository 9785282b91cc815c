/*
 * qeq.h -- C ABI of libqeq.so, a B300 (sm_103a) periodic charge-equilibration
 * (QEq) solver for Gaussian charges.
 *
 * The operation (RuNNer 2.0 paper, Sec. 2.4 "Electrostatics and Charge
 * Equilibration"; SI "Fourth-Generation HDNNPs and Charge Equilibration"):
 * given per-atom electronegativities chi_i, hardnesses J_i > 0 and Gaussian
 * widths sigma_i of a periodic cell, find the charges q that minimise
 *
 *     E_QEq = 1/2 q^T (E + diag J) q + chi^T q        (eq. qeq_energy)
 *
 * subject to sum_i q_i = q_tot (the bordered system of eq. 4G_qeq_prime; SI
 * eq. qeq: (E + J) q = -chi + mu 1).  E is the Coulomb matrix of normalised
 * Gaussians (eq. elec_energy: E_ii = 1/(sigma_i sqrt pi), E_ij =
 * erf(r_ij/(sqrt2 gamma_ij))/r_ij, gamma_ij^2 = sigma_i^2 + sigma_j^2),
 * summed over periodic images with the G = 0 Fourier term of the charge
 * density dropped (the neutralising background implied by the plane-wave
 * kernel 4 pi/G^2 of eq. matvec).  Scaled by coulomb_k.
 *
 * The solve is a Jacobi-preconditioned conjugate gradient projected onto the
 * charge constraint, around the plane-wave matrix-vector product of eq.
 * (matvec) (Sec. 2.4 "Electrostatics Solvers"): an Ewald split (SI "Ewald
 * Summation") into a screened real-space pair term, B-spline charge
 * spreading, 3D FFT, a width-corrected Gaussian reciprocal multiply, inverse
 * FFT and B-spline interpolation back, plus self and width-correction terms.
 * A is never formed.
 *
 * Conventions
 *   units        eV, Angstrom, e (coulomb_k = 14.3996454784 eV A / e^2); any
 *                consistent system works (coulomb_k = 1 for atomic units).
 *   cells        row-major 3x3 per structure, rows are the lattice vectors
 *                a1, a2, a3; any non-singular (triclinic) cell.
 *   atoms        packed over structures: structure s owns atoms
 *                [atom_offsets[s], atom_offsets[s+1]).
 *   pointers     "h_" = host memory, "d_" = device memory of the plan's GPU.
 *                The caller owns every pointer; the library never keeps one
 *                after a call returns.  Device pointers may be PyTorch
 *                tensors' data_ptr().
 *   streams      all device work of a plan is enqueued on the stream given to
 *                qeq_plan_create; calls return after that stream has finished
 *                the call's work (the host reads per-structure results).
 *   allocation   qeq_plan_create allocates every device buffer the plan
 *                needs; qeq_solve, qeq_energy, qeq_matvec, qeq_forces,
 *                qeq_stress and qeq_embedding allocate nothing.
 *   errors       every call returns a qeq_status and never aborts the process;
 *                qeq_last_error gives a message.  Invalid input leaves outputs
 *                unspecified.
 *   threads      a plan is not thread-safe; distinct plans are independent.
 */
#ifndef QEQ_H
#define QEQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QEQ_OK = 0,
  QEQ_ERR_INVALID = 1,   /* bad argument, non-finite input, species out of range, singular cell */
  QEQ_ERR_NOT_PD = 2,    /* some J_i <= 0 or sigma <= 0: the QEq matrix is not positive definite */
  QEQ_ERR_NOCONV = 3,    /* PCG did not reach the tolerance within max_iter (best q returned) */
  QEQ_ERR_CUDA = 4,      /* a CUDA runtime call failed */
  QEQ_ERR_OOM = 5,       /* device allocation failed in qeq_plan_create */
  QEQ_ERR_TIMEOUT = 6,   /* a bounded device wait gave up */
  QEQ_ERR_CAPACITY = 7   /* real-space pair list larger than the plan's capacity */
} qeq_status;

enum { QEQ_FP64 = 0, QEQ_MIXED = 1 };
enum { QEQ_WARM_COLD = 0, QEQ_WARM_USER = 1, QEQ_WARM_MLP = 2 };
/* Plan flags.  NO_GRAPH: launch every PCG iteration from the host instead of CUDA graphs.
 * TEST_STALL (tests only): in the main mesh's x FFT pass, the first tile announces 16 more
 * bytes on its copy barrier than its bulk copies deliver, so its bounded wait (0.5 s on the
 * GPU's global timer) runs out; the kernel flags the timeout and returns, and the call
 * returns QEQ_ERR_TIMEOUT.  It exercises the timeout path without any fault.
 * TWO_RHS: the two-right-hand-side formulation of the iterative QEq that the paper compares
 * against (Sec. "LAMMPS MD Performance"): plain PCG on (E + diag J) t = 1 and on
 * (E + diag J) s = -chi without the charge constraint, then q = s + mu' t with
 * mu' = (q_tot - sum s) / sum t.  Each sub-solve stops at a quarter of the charge
 * threshold; the combined q gets the same FP64 projected-residual check as the default
 * solver, and qeq_info reports the two sub-solves' iterations together.  Cold start only
 * (another warm mode returns QEQ_ERR_INVALID).
 * SQNM: the stabilised quasi-Newton minimiser of the paper's solver comparison (SI solver
 * figure) instead of CG: steps on the constraint plane in Jacobi-scaled coordinates, a
 * Newton step in the significant subspace of the last 8 steps (symmetrised secant Hessian,
 * curvatures enlarged by their residues) and a steepest-descent step alpha in the
 * complement; a step that raises E_QEq is undone, alpha halved and the history cleared.
 * One matvec per step (mixed precision: FP64 A q1 at each round's start plus the FP32
 * product of the change); the same FP64 final check and restarts as the CG.  Host-paced;
 * the plan allocates its history (16 N doubles) at creation.  Warm starts as for CG.
 * CHECK_DD, CHECK_FP64 (QEQ_MIXED plans): the FP64-accurate products of a mixed plan (its
 * final checks, qeq_energy, qeq_matvec with force_fp64) run spread, gather and local terms
 * in FP64 and the FFT passes either in FP64 or in double-float arithmetic (pairs of FP32
 * values, ~2^-44 relative per operation, on the FP32 pipes); by default double-float when
 * some structure's mesh has 2^21 points or more and no structure has more than two
 * species (with more, the double-float x pass spills registers and FP64 stays the default).
 * The two flags force one or the other. */
enum {
  QEQ_FLAG_NO_GRAPH = 1,
  QEQ_FLAG_TEST_STALL = 2,
  QEQ_FLAG_TWO_RHS = 4,
  QEQ_FLAG_SQNM = 8,
  QEQ_FLAG_CHECK_DD = 16,
  QEQ_FLAG_CHECK_FP64 = 32
};
/* Preconditioners of the PCG.  JACOBI: D^-1, D_i = J_i + k_e/(sigma_i sqrt pi).
 * FOURIER: D^-1 - D^-1 T^T F^-1[h F(T D^-1 r)], the Woodbury inverse of D plus the
 * long-range Coulomb operator with the mesh operator T D^-1 T^T replaced by its
 * translation-invariant mean (T: cubic B-spline spreading on a coarse FP32 mesh,
 * h(m) = beta |b(m)|^2 g0 / (1 + s0 g0), g0 = k_e (4 pi/V) exp(-G^2 w^2/2)/G^2,
 * s0 = sum_i 1/D_i).  beta = 1 while x = s0 g0 of the smoothest mode is at most 150;
 * larger cells (x grows with the cell size squared) use precond_scale: beta < 1 keeps
 * the preconditioner positive definite when the mean differs from the real operator
 * by less than 1 - beta, where the correction nearly cancels D^-1 for smooth modes,
 * at the price of eigenvalues up to 1 + (1 - beta) x.  If r.z of a preconditioned residual is not positive
 * the structure continues with Jacobi.  It changes no result, only the iteration
 * count. */
enum { QEQ_PRECOND_JACOBI = 0, QEQ_PRECOND_FOURIER = 1 };

typedef struct qeq_plan_s* qeq_plan;

/* Plan description.  Zero / negative numeric fields select defaults. */
typedef struct {
  int32_t n_struct;             /* >= 1 structures solved together                          */
  const int64_t* atom_offsets;  /* h_, n_struct+1, CSR offsets into the packed atom arrays   */
  const double* cells;          /* h_, n_struct*9, rows a1 a2 a3 [A]                          */
  int32_t n_species;            /* species table width, 1..8                                 */
  const double* sigma;          /* h_, n_struct*n_species Gaussian widths [A], > 0; trailing  */
                                /* entries <= 0 mark species absent from that structure     */
  double coulomb_k;             /* default 14.3996454784                                      */
  double charge_tol;            /* stop: max-abs projected residual <= 0.5*charge_tol*J_min;  */
                                /* default 1e-5 e                                            */
  double ewald_tol;             /* relative accuracy of the matvec; default 1e-6              */
  double r_cut;                 /* real-space cutoff [A]; default 8                           */
  int32_t spline_order;         /* B-spline order p in {4,6,8}, one per plan; 0: autotuned    */
  double mesh_spacing;          /* target spacing between lattice planes [A]; <= 0: the      */
                                /* autotuner picks the cheapest mesh whose predicted matvec  */
                                /* error meets ewald_tol (mesh sizes are 2^a 3^b 5^c)        */
  int32_t precision;            /* QEQ_FP64 (all FP64) or QEQ_MIXED (FP32 mesh/FFT/pairs,    */
                                /* FP64 reductions, projection, multiplier, final check)     */
  int32_t max_iter;             /* PCG iterations per structure; default 1000                 */
  double residual_tol;          /* optional extra stop: ||P r||_2 <= residual_tol*||P chi||_2 */
  int32_t flags;                /* QEQ_FLAG_*                                                 */
  int32_t preconditioner;       /* QEQ_PRECOND_JACOBI (default) or QEQ_PRECOND_FOURIER        */
  double precond_spacing;       /* FOURIER: coarse mesh spacing [A]; <= 0: 2.0; a spacing so  */
                                /* fine that the coarse spread's tiles exceed 64 KB of shared */
                                /* memory: QEQ_ERR_INVALID                                    */
  double precond_width;         /* FOURIER: Gaussian width w [A]; <= 0: 3.0 for cells up to   */
                                /* 80 A wide, 4.5 above                                       */
  double precond_scale;         /* FOURIER: safety factor beta of large cells, 0 < beta <= 1;  */
                                /* <= 0: 0.98                                                 */
} qeq_plan_desc;

/* Per-structure result of qeq_solve. */
typedef struct {
  int32_t status;          /* qeq_status of this structure                                  */
  int32_t iterations;      /* PCG iterations (matvecs after the first residual)             */
  int32_t restarts;        /* residual replacements after a final check failed              */
  int32_t warm_used;       /* 1 when the warm start was kept, 0 when it fell back to cold   */
  double residual_inf;     /* final max-abs of P(Aq + chi) [eV/e], P = I - 11^T/N           */
  double residual_l2;      /* final ||P(Aq + chi)||_2 [eV/e]                                 */
  double error_bound_l2;   /* certified ||q - q*||_2 <= residual_l2 / J_min for the plan's   */
                           /* matrix (the mesh approximation of A is not included)          */
} qeq_info;

/* Mesh / split parameters the plan chose for one structure. */
typedef struct {
  int32_t mesh[3];         /* K1, K2, K3                                                     */
  int32_t spline_order;
  int32_t n_species;
  int32_t narrow_pairs;    /* species pairs carried partly in real space                     */
  double omega;            /* Ewald split width [A]                                          */
  double r_cut;            /* real-space cutoff [A]                                          */
  double volume;           /* [A^3]                                                          */
  int64_t n_atoms;
  int64_t pair_capacity;   /* real-space pair slots of the whole plan                        */
  int64_t workspace_bytes; /* device bytes held by the whole plan                            */
  int64_t kernel_launches; /* CUDA kernels this plan has launched so far (graph replays count  */
                           /* every kernel in the graph)                                     */
} qeq_plan_info;

/* Create a plan: validate the description, choose mesh, B-spline order and
 * Ewald split per structure, and allocate all device workspace on the current
 * CUDA device.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: QEQ_ERR_INVALID / QEQ_ERR_NOT_PD for bad descriptions (sigma <= 0,
 * singular cell, n_species out of range), QEQ_ERR_OOM. */
qeq_status qeq_plan_create(const qeq_plan_desc* desc, void* cuda_stream, qeq_plan* out);

/* Release a plan and its device memory (NULL is ignored). */
void qeq_plan_destroy(qeq_plan plan);

/* Per-structure parameters chosen by the plan. */
qeq_status qeq_plan_query(qeq_plan plan, int32_t s, qeq_plan_info* out);

/* Solve the QEq problem of every structure of the plan.
 *   d_pos      N x 3 Cartesian positions [A] (any image; wrapped internally)
 *   d_species  N species indices in [0, n_species)
 *   d_chi      N electronegativities [eV/e]
 *   d_J        N hardnesses [eV/e^2], all > 0 (else QEQ_ERR_NOT_PD)
 *   h_qtot     n_struct total charges [e]
 *   warm       QEQ_WARM_COLD: start from q_tot/N; QEQ_WARM_USER: start from
 *              d_q (projected onto the constraint); QEQ_WARM_MLP: start from
 *              the network attached with qeq_plan_set_warm_start (projected)
 *   d_q        N charges [e]: input for QEQ_WARM_USER, output always
 *   d_mu       n_struct Lagrange multipliers mu with (A + J) q + chi = mu 1
 *              (the bordered lambda of eq. 4G_qeq_prime is -mu); may be NULL
 *   h_info     n_struct qeq_info records; may be NULL
 * Returns the worst per-structure status (QEQ_ERR_NOCONV if any structure
 * stopped at max_iter). */
qeq_status qeq_solve(qeq_plan plan, const double* d_pos, const int32_t* d_species,
                     const double* d_chi, const double* d_J, const double* h_qtot,
                     int32_t warm, double* d_q, double* d_mu, qeq_info* h_info);

/* Energies of given charges: d_E_qeq[s] = chi.q + 1/2 q.(E + diag J) q
 * (eq. qeq_energy) and d_E_elec[s] = 1/2 q.E q (eq. elec_energy), per
 * structure, evaluated with the FP64 matvec.  Either output may be NULL. */
qeq_status qeq_energy(qeq_plan plan, const double* d_pos, const int32_t* d_species,
                      const double* d_chi, const double* d_J, const double* d_q,
                      double* d_E_qeq, double* d_E_elec);

/* One plane-wave matrix-vector product d_y = (E + diag J) d_x (eq. matvec),
 * in the plan's precision (QEQ_FP64 or QEQ_MIXED) or FP64 when force_fp64.
 * d_J may be NULL (then diag J is left out).  Same atom layout as qeq_solve. */
qeq_status qeq_matvec(qeq_plan plan, const double* d_pos, const int32_t* d_species,
                      const double* d_J, const double* d_x, double* d_y, int32_t force_fp64);

/* Electrostatic forces by the force trick (SI eq. 4g_force_trick).  For a
 * total energy E(q, R) whose charges solve the QEq system, the force on atom
 * k, with lambda solving (E + diag J) lambda = -dE/dq + nu 1, sum lambda = 0,
 * is
 *     F_k = -dE/dR_k|_q - lambda^T (dA/dR_k) q,
 * and this call returns the electrostatic part of it:
 *     d_F[k] = -(q_k + lambda_k) grad_k phi_q(k) - q_k grad_k phi_lambda(k),
 * phi_x(k) = sum_j E_kj x_j the potential of the charges x at atom k and
 * grad_k its gradient with respect to R_k at fixed x (the hardness and the
 * self terms do not depend on positions).  With d_lambda = NULL the lambda
 * terms are left out: d_F = -dE_elec/dR at fixed q (E_elec of eq.
 * elec_energy), the force when the charges minimise E_QEq itself.  lambda
 * comes from qeq_solve with chi := dE/dq and q_tot = 0.
 *
 * The potential gradients are taken through the plane-wave terms of eq.
 * (matvec): the potential meshes (spread, FFT, reciprocal multiply, inverse
 * FFT; FP64 in QEQ_FP64 plans, FP32 in QEQ_MIXED plans, whose meshes carry
 * ~3e-7 of the potentials' size) are interpolated with the derivative of the
 * B-spline weights
 * (dM_p(t)/dt = M_{p-1}(t) - M_{p-1}(t - 1)) and mapped to Cartesian
 * derivatives through the cell; the screened real-space pair term of the
 * Ewald split (SI "Ewald Summation") adds its analytic derivative in FP64.
 * The error is that of the matvec's interpolation (ewald_tol), plus FP32
 * rounding in mixed plans.  The cell
 * counterpart is qeq_stress.
 *
 *   d_pos, d_species   as in qeq_solve (device, input order)
 *   d_q                N charges (device), input order
 *   d_lambda           N Lagrange multipliers (device) or NULL
 *   d_F                N x 3 forces (device), input order, written
 * Errors: QEQ_ERR_INVALID (null pointer, non-finite position, species out of
 * range), QEQ_ERR_CUDA, QEQ_ERR_TIMEOUT. */
qeq_status qeq_forces(qeq_plan plan, const double* d_pos, const int32_t* d_species,
                      const double* d_q, const double* d_lambda, double* d_F);

/* Strain derivative of the same electrostatic terms (the cell counterpart of
 * qeq_forces, SI eq. 4g_force_trick): under the homogeneous deformation of a
 * structure's cell and positions r -> (1 + eps) r at fixed charges,
 *     d_D[9 s + 3 a + b] = d/d eps_ab [(q/2 + lambda)^T E q]
 * (E of eq. elec_energy; lambda = NULL: d/d eps of E_elec).  The stress of
 * these terms is D / V; D is symmetric.  Reciprocal part: the strain
 * derivative of the plane-wave kernel, dG^2/d eps_ab = -2 G_a G_b and
 * dV/d eps_ab = V delta_ab, summed over the forward-transformed charge
 * meshes in FP64 (two mesh passes with lambda, by polarisation of the
 * bilinear form; one without); real-space part: the pair-term derivative;
 * the G = 0 width term scales as 1/V.
 *
 *   d_pos, d_species   as in qeq_solve (device, input order)
 *   d_q                N charges (device), input order
 *   d_lambda           N Lagrange multipliers (device) or NULL
 *   d_D                n_struct x 9 (device), row-major 3x3 per structure, written
 * Errors: as qeq_forces. */
qeq_status qeq_stress(qeq_plan plan, const double* d_pos, const int32_t* d_species,
                      const double* d_q, const double* d_lambda, double* d_D);

/* Element-resolved electrostatic potentials of the ee4G embedding (Sec. 2.2,
 * Fig. 1c): d_Gamma[i * n_species + z] = sum over atoms j of element z of
 * E_ij q_j (E of eq. elec_energy, no hardness), the potential at atom i of
 * the charges of element z; summed over z it is (E q)_i.  One FP64 matvec of
 * eq. (matvec) per element; the descriptor built from it is the caller's.
 *
 *   d_pos, d_species   as in qeq_solve (device, input order)
 *   d_q                N charges (device), input order
 *   d_Gamma            N x n_species (device), input order, row-major, written
 * Errors: as qeq_matvec. */
qeq_status qeq_embedding(qeq_plan plan, const double* d_pos, const int32_t* d_species,
                         const double* d_q, double* d_Gamma);

/* Time each stage of the matvec with CUDA events on the plan's stream.
 * Runs n_rep matvecs of the plan's precision on the atoms of the last
 * qeq_solve / qeq_matvec call and writes the mean milliseconds per launch of
 * each stage to h_ms[0..QEQ_N_STAGES).  Stage order: species sums, spread,
 * FFT z, FFT y, FFT x + reciprocal multiply + inverse FFT x, inverse FFT y,
 * inverse FFT z, gather + real space + local terms. */
#define QEQ_N_STAGES 8
qeq_status qeq_profile_matvec(qeq_plan plan, int32_t n_rep, float* h_ms);

/* ------------------------------------------------------------------------
 * 4G charge training on cached dense matrices (Sec. "4G-HDNNP Charge
 * Training").  Training structures are small and their positions fixed while
 * the networks learn chi (and possibly J), so the Coulomb matrix E of each
 * structure (eq. elec_energy, periodic, G = 0 term dropped; no hardness) is
 * assembled once, the bordered matrix A' = [[E + diag J, 1], [1^T, 0]] of
 * eq. (4G_qeq_prime) is inverted whenever J changes, and the charges of a
 * training step are one matrix-vector product
 *     (q, lambda) = -A'^{-1} (chi, -q_tot),   mu = -lambda.
 * The backward pass uses the same inverse (A' is symmetric): with
 * (l, nu) = A'^{-1} (dL/dq, 0),  dL/dchi = -l  and  dL/dJ_i = -l_i q_i.
 *
 * E is assembled in FP64 by the Ewald split of SI "Ewald Summation" with one
 * width omega >= every gamma_ij per structure (chosen for the least work),
 * real-space and reciprocal sums truncated where their terms fall below
 * ewald_tol (default 1e-12 here); the inverse is FP64 (Cholesky of
 * E + diag J, triangular inverse, bordered by the Schur complement).
 *
 * Precision (desc.precision): QEQ_FP64 (default) caches the FP64 inverse and
 * charges are one FP64 matrix-vector product.  QEQ_MIXED inverts in FP32 (this
 * GPU's FP32 pipe is far wider than its FP64 pipe) and refines every result in
 * FP64 against the exact bordered matrix: x = K32 b, then twice
 * x += K32 (b - A' x); each step shrinks the error by about cond(A') eps_FP32,
 * so the charges and gradients reach FP64 accuracy for QEq matrices.
 *
 * Handle: qeq_dense_create takes a qeq_plan_desc (n_struct, atom_offsets,
 * cells, n_species, sigma, coulomb_k, ewald_tol, precision are read; the rest
 * is ignored) and the CUDA stream every call runs on; it allocates E, A'^{-1}
 * and a work matrix per structure (3 n^2 values) and nothing later.
 * Structures have at most QEQ_DENSE_MAX_ATOMS atoms (else QEQ_ERR_CAPACITY).
 * Atom arrays are packed by atom_offsets, device pointers, FP64 / int32.
 * Calls of one handle are ordered on its stream; inputs must be ready there.
 * ------------------------------------------------------------------------ */
#define QEQ_DENSE_MAX_ATOMS 1024
typedef struct qeq_dense_s* qeq_dense;

qeq_status qeq_dense_create(const qeq_plan_desc* desc, void* cuda_stream, qeq_dense* out);
void qeq_dense_destroy(qeq_dense dense);
const char* qeq_dense_last_error(qeq_dense dense);

/* E of every structure from the positions (N x 3) and species (N).
 * Errors: QEQ_ERR_INVALID (non-finite position, species out of range). */
qeq_status qeq_dense_assemble(qeq_dense dense, const double* d_pos, const int32_t* d_species);

/* A'^{-1} of every structure with hardness d_J (N, > 0), cached until the
 * next call.  Errors: QEQ_ERR_NOT_PD (E + diag J not positive definite),
 * QEQ_ERR_INVALID (qeq_dense_assemble not called). */
qeq_status qeq_dense_invert(qeq_dense dense, const double* d_J);

/* Charges d_q (N) and multipliers d_mu (n_struct, may be NULL) for the
 * electronegativities d_chi (N) and the total charges h_qtot (host,
 * n_struct; NULL: neutral). */
qeq_status qeq_dense_charges(qeq_dense dense, const double* d_chi, const double* h_qtot,
                             double* d_q, double* d_mu);

/* Backward pass of qeq_dense_charges for a loss gradient d_gq = dL/dq (N):
 * d_gchi = dL/dchi (N); d_gJ = dL/dJ (N, may be NULL; then d_q may be NULL). */
qeq_status qeq_dense_backward(qeq_dense dense, const double* d_q, const double* d_gq,
                              double* d_gchi, double* d_gJ);

/* Copy E (which = 0, n x n) or A'^{-1} (which = 1, (n+1) x (n+1); the FP32
 * inverse widened to FP64 under QEQ_MIXED) of structure s, row-major, to
 * d_out (device). */
qeq_status qeq_dense_matrix(qeq_dense dense, int32_t s, int32_t which, double* d_out);

/* The Ewald width and G-vector count chosen for structure s, and the kernels
 * launched by the handle so far (any pointer may be NULL). */
qeq_status qeq_dense_query(qeq_dense dense, int32_t s, double* h_omega, int32_t* h_ng,
                           int64_t* h_launches);

/* ------------------------------------------------------------------------
 * Learned warm start (the paper's atomic neural networks, SI "Feed-Forward
 * Neural Networks", applied here to predict starting charges for the solve).
 *
 * Descriptors of atom i (radial functions of Sec. 2.2 eq. g2 with the cosine
 * cutoff of SI "Cutoff Functions", cutoff QEQ_MLP_RCUT; the element-embracing
 * prefactor of SI "Element-Embracing ACSFs" with H_ij = chi_j), float32 x 32:
 *   [0..11]  sum_j exp(-2 (r_ij - R_mu)^2) f_c(r_ij),  R_mu = 0.5 + 0.5 mu A
 *   [12..23] the same weighted by chi_j
 *   [24..26] chi_i, J_i, sigma_i ; [27..31] zero
 * Network per species: 32 -> 64 -> 64 -> 1, tanh, tanh, linear, evaluated on
 * BF16 tensor cores (tcgen05 MMAs) with FP32 accumulation in tensor memory,
 * forward and, in training, backward; inputs scaled per species as
 * (G - mean) * inv_range (SI "Feature Scaling"), the scaled inputs, activations
 * and output-side derivatives rounded to BF16 as MMA operands.
 * Parameter block of one species (float32, QEQ_MLP_NPARAM entries):
 *   W1[64][32], b1[64], W2[64][64], b2[64], W3[64], b3, then padding.
 * Scaling block of one species: mean[32], inv_range[32].
 * Training minimises 1/(2n) sum (y_i - target_i)^2 with Adam (beta 0.9/0.999,
 * eps 1e-8, SI "Adam") on FP32 master weights. */
#define QEQ_MLP_NFEAT 32
#define QEQ_MLP_NHIDDEN 64
#define QEQ_MLP_NPARAM 6400
#define QEQ_MLP_RCUT 6.0f
typedef struct qeq_mlp_s* qeq_mlp;

/* Network for n_species species, zero-initialised (set parameters with
 * qeq_mlp_set_params), training batches of at most max_batch atoms; device
 * memory on the current device. */
qeq_status qeq_mlp_create(int32_t n_species, int64_t max_batch, qeq_mlp* out);
void qeq_mlp_destroy(qeq_mlp mlp);
/* h_params: n_species * QEQ_MLP_NPARAM floats (NULL = keep), h_scale:
 * n_species * 2 * QEQ_MLP_NFEAT floats (NULL = keep); new parameters reset Adam. */
qeq_status qeq_mlp_set_params(qeq_mlp mlp, const float* h_params, const float* h_scale);
/* Copies out parameters, scaling, Adam moments and step count (any may be NULL). */
qeq_status qeq_mlp_get_params(qeq_mlp mlp, float* h_params, float* h_scale, float* h_adam_m, float* h_adam_v,
                              int64_t* h_step);
/* Restores Adam moments and step count (checkpoint resume). */
qeq_status qeq_mlp_set_adam_state(qeq_mlp mlp, const float* h_adam_m, const float* h_adam_v, int64_t step);
/* d_out[i] = network output for atom i (d_feat n x 32 unscaled descriptors). */
qeq_status qeq_mlp_forward(qeq_mlp mlp, const float* d_feat, const int32_t* d_species, int64_t n, float* d_out,
                           void* cuda_stream);
/* One training step on a batch of n <= max_batch atoms: forward, backward, and,
 * when apply_update, an Adam update with learning rate lr.  d_grad_out (may be
 * NULL): the batch gradient, n_species * QEQ_MLP_NPARAM floats; h_loss (may be
 * NULL): the batch loss.  Gradients are summed per 64-atom tile and then over
 * tiles in a fixed order (deterministic). */
qeq_status qeq_mlp_train_step(qeq_mlp mlp, const float* d_feat, const int32_t* d_species, const float* d_target,
                              int64_t n, float lr, int32_t apply_update, float* d_grad_out, float* h_loss,
                              void* cuda_stream);
/* Descriptors (n_atoms x 32, the caller's atom order) of the plan's cells. */
qeq_status qeq_features(qeq_plan plan, const double* d_pos, const int32_t* d_species, const double* d_chi,
                        const double* d_J, float* d_feat);
/* Attach a network for QEQ_WARM_MLP solves (NULL detaches; the plan does not
 * own it).  The plan's first QEQ_WARM_MLP solve needs this call first; it
 * allocates the descriptor buffers.  In the solve the network's charges are
 * projected onto the charge constraint and kept only if their QEq energy is
 * below that of the uniform start q_tot/N (on the constraint plane
 * E(q) - E(q*) = 1/2 ||q - q*||_A^2, the error norm CG reduces); otherwise, or
 * if it is not finite, the solve restarts cold and reports warm_used = 0. */
qeq_status qeq_plan_set_warm_start(qeq_plan plan, qeq_mlp mlp);

/* ------------------------------------------------------------------------
 * qeq_matvec_static -- the FP64 matvec of qeq_matvec for ONE small cell,
 * with no device allocation at all.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (code running while
 * another component owns the device memory pool or a fixed arena, code that
 * must not trigger the implicit synchronisation of cudaMalloc/cudaFree, or an
 * embedding that only passes input and output buffers).
 *
 * Scratch lives in a file-scope __device__ array of QEQ_STATIC_SCRATCH_BYTES
 * that every GPU loading the library keeps until process exit.  Limits:
 * n_atoms <= QEQ_STATIC_MAX_ATOMS, n_species <= QEQ_STATIC_MAX_SPECIES, at
 * most QEQ_STATIC_MAX_MESH mesh points per direction (the mesh, B-spline order
 * and Ewald split are chosen exactly as qeq_plan_create does) and at most
 * QEQ_STATIC_MAX_PAIRS real-space pair slots.  The array holds every buffer
 * for inputs at all of these limits at once (checked at compile time).  Atom,
 * species and mesh limits are checked on the host before any GPU work and
 * return QEQ_ERR_CAPACITY; the estimated pair-slot count is checked on the host
 * too, and the actual pair count, known only after the neighbour search, is
 * checked on the device: a cell with more pairs than slots also returns
 * QEQ_ERR_CAPACITY (nothing is written past the slots).
 *   h_cell     9 doubles, rows a1 a2 a3 [A]     h_sigma  n_species widths [A]
 *   d_pos      n_atoms x 3 [A]    d_species  n_atoms indices
 *   d_J        n_atoms hardnesses or NULL (diag J left out)
 *   d_x, d_y   input / output vectors of n_atoms
 *   coulomb_k, ewald_tol, r_cut   as in qeq_plan_desc (<= 0: defaults)
 *   cuda_stream                   a cudaStream_t (NULL = legacy stream)
 * Each call reads the device's error bits back to the host and returns after
 * the stream has finished its work, so no call can be captured into a CUDA
 * graph.  All calls share the scratch array, which keeps the last call's
 * contents: calls that overlap on the GPU, or come from several host threads at
 * once, race.  The first call on a device also sets up that device (it looks up
 * the array's device address and the kernels' shared-memory limits). */
#define QEQ_STATIC_MAX_ATOMS 4096
#define QEQ_STATIC_MAX_SPECIES 4
#define QEQ_STATIC_MAX_MESH 64
#define QEQ_STATIC_MAX_PAIRS 1048576
#define QEQ_STATIC_SCRATCH_BYTES (40u * 1024u * 1024u)
qeq_status qeq_matvec_static(const double* h_cell, const double* h_sigma, int32_t n_species, int32_t n_atoms,
                             const double* d_pos, const int32_t* d_species, const double* d_J,
                             const double* d_x, double* d_y, double coulomb_k, double ewald_tol,
                             double r_cut, void* cuda_stream);

/* Static description of one status code. */
const char* qeq_status_str(qeq_status s);

/* Message of the last error of this plan (never NULL). */
const char* qeq_last_error(qeq_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* QEQ_H */
