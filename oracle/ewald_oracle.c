/*
 * Plain FP64 CPU pieces of the Gaussian-charge Coulomb matrix of a periodic
 * cell.  TEST INFRASTRUCTURE ONLY: the oracle that the CUDA path is checked
 * against.  Nothing in the product library links or calls this file.
 *
 * Conventions (k_e = 1; the caller scales):
 *   cell  row-major 3x3, rows are the lattice vectors a1, a2, a3
 *   pos   n x 3 Cartesian positions
 *   sigma n Gaussian widths (0 = point charge)
 *
 * The matrix is the periodic Coulomb kernel of normalised Gaussian charges
 * (Sec. 2.4, eq. elec_energy: E_ii = 1/(sigma_i sqrt(pi)), E_ij =
 * erf(r/(sqrt(2) gamma_ij))/r, gamma_ij = sqrt(sigma_i^2 + sigma_j^2)) with the
 * G = 0 term dropped, evaluated by the Ewald split of SI "Ewald Summation":
 *   real space    sum_n [erfc(r/(sqrt2 w)) - erfc(r/(sqrt2 gamma))]/r,  w = max(gamma, omega)
 *   reciprocal    (4 pi/V) sum_{G != 0} exp(-G^2 w^2/2) cos(G.r)/G^2
 *   self (i = j)  sqrt(2/pi) (1/gamma_ii - 1/w_ii)
 *   G = 0 width   -(2 pi/V)(w^2 - gamma^2)
 * For a point charge (gamma = 0) the 1/gamma self part is left out and the
 * erfc(r/(sqrt2 gamma)) term is zero, which is textbook point-charge Ewald.
 *
 * The reciprocal part of the dense matrix is assembled in numpy (a BLAS
 * rank-k update); this file supplies the real-space/self/width part of the
 * dense matrix, a full matrix-vector product for cells too large to store
 * the matrix, and the position gradient of that product's rows.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static double det3(const double* h) {
  return h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
         h[2] * (h[3] * h[7] - h[4] * h[6]);
}

/* inverse of the row-major 3x3 matrix h */
static void inv3(const double* h, double* hi) {
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

/* distance between the lattice planes spanned by the two other vectors */
static void plane_widths(const double* h, double* wd) {
  double V = fabs(det3(h));
  for (int d = 0; d < 3; ++d) {
    const double* a = h + 3 * ((d + 1) % 3);
    const double* b = h + 3 * ((d + 2) % 3);
    double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
    wd[d] = V / sqrt(cx * cx + cy * cy + cz * cz);
  }
}

/* fractional coordinates u = pos h^{-1} (row vectors) */
static void to_frac(int n, const double* hi, const double* pos, double* u) {
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d)
      u[3 * i + d] = pos[3 * i] * hi[d] + pos[3 * i + 1] * hi[3 + d] + pos[3 * i + 2] * hi[6 + d];
}

/* screened pair term for distance r > 0 */
static double pair_real(double r, double g, double w) {
  double v = erfc(r / (sqrt(2.0) * w));
  if (g > 0) v -= erfc(r / (sqrt(2.0) * g));
  return v / r;
}

/* r -> 0 limit of the pair term (also the self term) */
static double pair_zero(double g, double w) {
  return sqrt(2.0 / ORC_PI) * ((g > 0 ? 1.0 / g : 0.0) - 1.0 / w);
}

/*
 * A[i*n+j] += real-space image sum (|d| < r_cut, image (i,0) excluded)
 *           + self term (i = j) + G = 0 width correction, with k_e = 1.
 * Every image within r_cut is visited, so cells smaller than 2 r_cut are fine.
 */
int oracle_realspace_dense(int n, const double* cell, const double* pos, const double* sigma,
                           double omega, double r_cut, double* A) {
  double hi[9], wd[3];
  inv3(cell, hi);
  plane_widths(cell, wd);
  double V = fabs(det3(cell));
  double* u = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!u) return 1;
  to_frac(n, hi, pos, u);
  double rc2 = r_cut * r_cut;
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double si = sigma[i], sj = sigma[j];
      double g = sqrt(si * si + sj * sj);
      double w = g > omega ? g : omega;
      double acc = -(2.0 * ORC_PI / V) * (w * w - g * g);
      if (i == j) acc += pair_zero(g, w);
      if (w > g) {
        double f[3];
        int lo[3], hi_[3];
        for (int d = 0; d < 3; ++d) {
          f[d] = u[3 * j + d] - u[3 * i + d];
          f[d] -= floor(f[d] + 0.5);
          double ext = r_cut / wd[d];
          lo[d] = (int)ceil(-ext - f[d]);
          hi_[d] = (int)floor(ext - f[d]);
        }
        for (int n1 = lo[0]; n1 <= hi_[0]; ++n1)
          for (int n2 = lo[1]; n2 <= hi_[1]; ++n2)
            for (int n3 = lo[2]; n3 <= hi_[2]; ++n3) {
              double a = f[0] + n1, b = f[1] + n2, c = f[2] + n3;
              double dx = a * cell[0] + b * cell[3] + c * cell[6];
              double dy = a * cell[1] + b * cell[4] + c * cell[7];
              double dz = a * cell[2] + b * cell[5] + c * cell[8];
              double r2 = dx * dx + dy * dy + dz * dz;
              if (r2 >= rc2) continue;
              if (i == j && n1 == 0 && n2 == 0 && n3 == 0) continue;
              double r = sqrt(r2);
              acc += (r > 1e-12) ? pair_real(r, g, w) : pair_zero(g, w);
            }
      }
      A[(size_t)i * n + j] += acc;
    }
  }
  free(u);
  return 0;
}

/* d/dr of the screened pair term at r > 0 */
static double pair_real_deriv(double r, double g, double w) {
  const double c = 2.0 / sqrt(ORC_PI);
  double a = 1.0 / (sqrt(2.0) * w), v = -c * a * exp(-a * a * r * r);
  if (g > 0) {
    double b = 1.0 / (sqrt(2.0) * g);
    v += c * b * exp(-b * b * r * r);
  }
  return v / r - pair_real(r, g, w) / r;
}

/* cell list over the fractional coordinates u (wrapped to [0,1)) for a cutoff r_cut:
   nc cells per direction, R cells searched each way, atoms of cell c at
   cidx[cstart[c] .. cstart[c+1]), acell = cell of each atom */
typedef struct {
  int nc[3], R[3];
  int *cstart, *cidx, *acell;
} CellList;

static int cells_build(int n, const double* u, const double* wd, double r_cut, CellList* cl) {
  for (int d = 0; d < 3; ++d) {
    cl->nc[d] = (int)floor(wd[d] / r_cut);
    if (cl->nc[d] < 1) cl->nc[d] = 1;
    if (cl->nc[d] > 512) cl->nc[d] = 512;
    cl->R[d] = (int)ceil(r_cut * cl->nc[d] / wd[d]);
    if (cl->R[d] < 1) cl->R[d] = 1;
  }
  size_t ncell = (size_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
  cl->cstart = (int*)calloc(ncell + 1, sizeof(int));
  cl->cidx = (int*)malloc(sizeof(int) * (size_t)n);
  cl->acell = (int*)malloc(sizeof(int) * (size_t)n);
  if (!cl->cstart || !cl->cidx || !cl->acell) return 1;
  for (int i = 0; i < n; ++i) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      c[d] = (int)floor(u[3 * i + d] * cl->nc[d]);
      if (c[d] >= cl->nc[d]) c[d] = cl->nc[d] - 1;
      if (c[d] < 0) c[d] = 0;
    }
    cl->acell[i] = (c[0] * cl->nc[1] + c[1]) * cl->nc[2] + c[2];
    cl->cstart[cl->acell[i] + 1]++;
  }
  for (size_t c = 0; c < ncell; ++c) cl->cstart[c + 1] += cl->cstart[c];
  int* fill = (int*)malloc(sizeof(int) * ncell);
  if (!fill) return 1;
  for (size_t c = 0; c < ncell; ++c) fill[c] = cl->cstart[c];
  for (int i = 0; i < n; ++i) cl->cidx[fill[cl->acell[i]]++] = i;
  free(fill);
  return 0;
}

static void cells_free(CellList* cl) {
  free(cl->cstart);
  free(cl->cidx);
  free(cl->acell);
}

/* visit(j, d[3]) for every atom j and image within r_cut of atom i (d = r_j + n - r_i,
   Cartesian; the unshifted image of i itself is skipped) */
#define CELLS_FOR_NEIGHBOURS(cl, u, cell, i, rc2, BODY)                                          \
  do {                                                                                           \
    int ci_[3], c_ = (cl).acell[i];                                                              \
    ci_[2] = c_ % (cl).nc[2];                                                                    \
    ci_[1] = (c_ / (cl).nc[2]) % (cl).nc[1];                                                     \
    ci_[0] = c_ / ((cl).nc[1] * (cl).nc[2]);                                                     \
    for (int a_ = -(cl).R[0]; a_ <= (cl).R[0]; ++a_)                                             \
      for (int b_ = -(cl).R[1]; b_ <= (cl).R[1]; ++b_)                                           \
        for (int e_ = -(cl).R[2]; e_ <= (cl).R[2]; ++e_) {                                       \
          int cc_[3] = {ci_[0] + a_, ci_[1] + b_, ci_[2] + e_}, sh_[3];                          \
          for (int d_ = 0; d_ < 3; ++d_) {                                                       \
            sh_[d_] = (int)floor((double)cc_[d_] / (cl).nc[d_]);                                 \
            cc_[d_] -= sh_[d_] * (cl).nc[d_];                                                    \
          }                                                                                      \
          int cj_ = (cc_[0] * (cl).nc[1] + cc_[1]) * (cl).nc[2] + cc_[2];                        \
          for (int t_ = (cl).cstart[cj_]; t_ < (cl).cstart[cj_ + 1]; ++t_) {                     \
            int j = (cl).cidx[t_];                                                               \
            int self_image = (j == (i) && sh_[0] == 0 && sh_[1] == 0 && sh_[2] == 0);            \
            if (self_image) continue;                                                            \
            double fa_ = (u)[3 * j] + sh_[0] - (u)[3 * (i)];                                     \
            double fb_ = (u)[3 * j + 1] + sh_[1] - (u)[3 * (i) + 1];                             \
            double fc_ = (u)[3 * j + 2] + sh_[2] - (u)[3 * (i) + 2];                             \
            double d[3];                                                                         \
            d[0] = fa_ * (cell)[0] + fb_ * (cell)[3] + fc_ * (cell)[6];                          \
            d[1] = fa_ * (cell)[1] + fb_ * (cell)[4] + fc_ * (cell)[7];                          \
            d[2] = fa_ * (cell)[2] + fb_ * (cell)[5] + fc_ * (cell)[8];                          \
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];                                 \
            if (r2 >= (rc2)) continue;                                                           \
            BODY                                                                                 \
          }                                                                                      \
        }                                                                                        \
  } while (0)

/* G vectors of the half-space m = (m1,m2,m3) > 0 (lexicographic) with |G| <= g_cut:
   gm (3 per vector), gf = 2 (4 pi/V) exp(-G^2 omega^2/2)/G^2 (factor 2 for the -G
   partner), M = index range per direction.  Returns the count, -1 on failure. */
static long gvecs_build(const double* hi, const double* wd, double V, double omega, double g_cut, int* M,
                        int** gm_out, double** gf_out) {
  for (int d = 0; d < 3; ++d) {
    /* |G| >= 2 pi |m_d| / wd[d] bounds the range of m_d */
    M[d] = (int)floor(g_cut * wd[d] / (2.0 * ORC_PI)) + 1;
  }
  long ng = 0, cap = 1024;
  int* gm = (int*)malloc(sizeof(int) * 3 * cap);
  double* gf = (double*)malloc(sizeof(double) * cap);
  if (!gm || !gf) return -1;
  for (int m1 = 0; m1 <= M[0]; ++m1)
    for (int m2 = (m1 == 0 ? 0 : -M[1]); m2 <= M[1]; ++m2)
      for (int m3 = ((m1 == 0 && m2 == 0) ? 1 : -M[2]); m3 <= M[2]; ++m3) {
        /* G = 2 pi (m1 b1 + m2 b2 + m3 b3), b_k = k-th column of h^{-1} */
        double gx = 2 * ORC_PI * (m1 * hi[0] + m2 * hi[1] + m3 * hi[2]);
        double gy = 2 * ORC_PI * (m1 * hi[3] + m2 * hi[4] + m3 * hi[5]);
        double gz = 2 * ORC_PI * (m1 * hi[6] + m2 * hi[7] + m3 * hi[8]);
        double G2 = gx * gx + gy * gy + gz * gz;
        if (G2 > g_cut * g_cut) continue;
        if (ng == cap) {
          cap *= 2;
          gm = (int*)realloc(gm, sizeof(int) * 3 * cap);
          gf = (double*)realloc(gf, sizeof(double) * cap);
          if (!gm || !gf) return -1;
        }
        gm[3 * ng] = m1;
        gm[3 * ng + 1] = m2;
        gm[3 * ng + 2] = m3;
        gf[ng] = 2.0 * (4.0 * ORC_PI / V) * exp(-0.5 * G2 * omega * omega) / G2;
        ++ng;
      }
  *gm_out = gm;
  *gf_out = gf;
  return ng;
}

/* phase factors exp(i 2 pi m u_d), m = -M_d..M_d, of one atom: t[d][2 (m + M_d) + {0,1}] */
static void phases(const double* ui, const int* M, double* t, double** tc) {
  int W0 = 2 * M[0] + 1, W1 = 2 * M[1] + 1;
  tc[0] = t;
  tc[1] = t + 2 * W0;
  tc[2] = t + 2 * (W0 + W1);
  for (int d = 0; d < 3; ++d)
    for (int m = -M[d]; m <= M[d]; ++m) {
      double ph = 2 * ORC_PI * m * ui[d];
      tc[d][2 * (m + M[d])] = cos(ph);
      tc[d][2 * (m + M[d]) + 1] = sin(ph);
    }
}

/* exp(i G_k . r) from the separable phase factors */
static void phase_of(double* const* tc, const int* M, const int* gmk, double* er, double* ei) {
  const double* a = tc[0] + 2 * (gmk[0] + M[0]);
  const double* b = tc[1] + 2 * (gmk[1] + M[1]);
  const double* c = tc[2] + 2 * (gmk[2] + M[2]);
  double abr = a[0] * b[0] - a[1] * b[1], abi = a[0] * b[1] + a[1] * b[0];
  *er = abr * c[0] - abi * c[1];
  *ei = abr * c[1] + abi * c[0];
}

/* structure factor S(G) = sum_j q_j exp(i G.r_j); per-thread partials summed in thread order */
static int structure_factor(int n, const double* u, const double* q, const int* M, long ng, const int* gm,
                            double* Sre, double* Sim) {
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  double* part = (double*)calloc((size_t)nthr * 2 * ng, sizeof(double));
  if (!part) return 1;
  int W = 2 * (2 * M[0] + 1 + 2 * M[1] + 1 + 2 * M[2] + 1);
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* pr = part + (size_t)tid * 2 * ng;
    double* pi = pr + ng;
    double* t = (double*)malloc(sizeof(double) * W);
    double* tc[3];
#pragma omp for schedule(static)
    for (int j = 0; j < n; ++j) {
      phases(u + 3 * j, M, t, tc);
      for (long k = 0; k < ng; ++k) {
        double er, ei;
        phase_of(tc, M, gm + 3 * k, &er, &ei);
        pr[k] += q[j] * er;
        pi[k] += q[j] * ei;
      }
    }
    free(t);
  }
  for (long k = 0; k < ng; ++k) Sre[k] = Sim[k] = 0.0;
  for (int tt = 0; tt < nthr; ++tt)
    for (long k = 0; k < ng; ++k) {
      Sre[k] += part[(size_t)tt * 2 * ng + k];
      Sim[k] += part[(size_t)tt * 2 * ng + ng + k];
    }
  free(part);
  return 0;
}

/* sum_j x_j (w_ij^2 - gamma_ij^2) for atom i of width si, over the distinct widths */
typedef struct {
  int nd;
  double ds[64], dq[64];
} WidthSums;

static int width_sums(int n, const double* sigma, const double* x, WidthSums* ws) {
  ws->nd = 0;
  for (int j = 0; j < n; ++j) {
    int k = 0;
    while (k < ws->nd && ws->ds[k] != sigma[j]) ++k;
    if (k == ws->nd) {
      if (ws->nd == 64) return 2;
      ws->ds[ws->nd] = sigma[j];
      ws->dq[ws->nd] = 0.0;
      ++ws->nd;
    }
    ws->dq[k] += x[j];
  }
  return 0;
}

static double width_term(const WidthSums* ws, double si, double omega) {
  double acc = 0.0;
  for (int k = 0; k < ws->nd; ++k) {
    double g2 = si * si + ws->ds[k] * ws->ds[k];
    double w2 = g2 > omega * omega ? g2 : omega * omega;
    acc += ws->dq[k] * (w2 - g2);
  }
  return acc;
}

/*
 * y = A q for the Coulomb part (k_e = 1, no hardness) with a single Ewald
 * width omega >= every gamma_ij, so that every pair shares the reciprocal
 * Gaussian exp(-G^2 omega^2/2).  Real space by a cell list over all images
 * within r_cut; reciprocal space by explicit structure factors over the
 * half-space of G with |G| <= g_cut (separable phase factors per atom).
 * rows: if n_rows > 0, y is only evaluated for atoms rows[0..n_rows) and
 * written to y[0..n_rows); the structure factors still use every atom.
 * grad = 1: the position gradient of each row instead (oracle_ewald_potential_grad).
 */
static int ewald_rows(int n, const double* cell, const double* pos, const double* sigma, const double* q,
                      double omega, double r_cut, double g_cut, int n_rows, const int* rows, int grad,
                      double* y) {
  double hi[9], wd[3];
  inv3(cell, hi);
  plane_widths(cell, wd);
  double V = fabs(det3(cell));
  int nout = n_rows > 0 ? n_rows : n;
  double* u = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!u) return 1;
  to_frac(n, hi, pos, u);
  for (int i = 0; i < 3 * n; ++i) u[i] -= floor(u[i]);
  CellList cl;
  if (cells_build(n, u, wd, r_cut, &cl)) return 1;
  double rc2 = r_cut * r_cut;

  /* ---------------- real space */
#pragma omp parallel for schedule(dynamic, 64)
  for (int o = 0; o < nout; ++o) {
    int i = n_rows > 0 ? rows[o] : o;
    double si = sigma[i];
    double acc = 0.0, gr[3] = {0.0, 0.0, 0.0};
    CELLS_FOR_NEIGHBOURS(cl, u, cell, i, rc2, {
      if (grad && j == i) continue; /* the images of i move with i */
      double sj = sigma[j];
      double g = sqrt(si * si + sj * sj);
      double w = g > omega ? g : omega;
      double r = sqrt(r2);
      if (grad) {
        if (r > 1e-12) { /* coincident atoms exert no force on each other */
          double c = -q[j] * pair_real_deriv(r, g, w) / r;
          gr[0] += c * d[0];
          gr[1] += c * d[1];
          gr[2] += c * d[2];
        }
      } else {
        acc += q[j] * ((r > 1e-12) ? pair_real(r, g, w) : pair_zero(g, w));
      }
    });
    if (grad) {
      for (int e = 0; e < 3; ++e) y[3 * o + e] = gr[e];
    } else {
      double g = sqrt(2.0) * si;
      double w = g > omega ? g : omega;
      acc += q[i] * pair_zero(g, w);
      y[o] = acc;
    }
  }
  /* G = 0 width correction, O(n) per row over the distinct widths (no gradient) */
  if (!grad) {
    WidthSums ws;
    if (width_sums(n, sigma, q, &ws)) return 2;
    for (int o = 0; o < nout; ++o) {
      int i = n_rows > 0 ? rows[o] : o;
      y[o] -= (2.0 * ORC_PI / V) * width_term(&ws, sigma[i], omega);
    }
  }

  /* ---------------- reciprocal space: half-space of G, |G| <= g_cut */
  int M[3];
  int* gm;
  double* gf;
  long ng = gvecs_build(hi, wd, V, omega, g_cut, M, &gm, &gf);
  if (ng < 0) return 1;
  double* Sre = (double*)calloc((size_t)ng, sizeof(double));
  double* Sim = (double*)calloc((size_t)ng, sizeof(double));
  if (!Sre || !Sim || structure_factor(n, u, q, M, ng, gm, Sre, Sim)) return 1;
  int W = 2 * (2 * M[0] + 1 + 2 * M[1] + 1 + 2 * M[2] + 1);
  /* y_i += sum_G f(G) Re[exp(i G.r_i) conj(S(G))]; gradient: f G [S_im cos - S_re sin] */
#pragma omp parallel
  {
    double* t = (double*)malloc(sizeof(double) * W);
    double* tc[3];
#pragma omp for schedule(static)
    for (int o = 0; o < nout; ++o) {
      int i = n_rows > 0 ? rows[o] : o;
      phases(u + 3 * i, M, t, tc);
      double acc = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
      for (long k = 0; k < ng; ++k) {
        double er, ei;
        phase_of(tc, M, gm + 3 * k, &er, &ei);
        if (grad) {
          int m1 = gm[3 * k], m2 = gm[3 * k + 1], m3 = gm[3 * k + 2];
          double tt = gf[k] * (er * Sim[k] - ei * Sre[k]);
          gx += tt * 2 * ORC_PI * (m1 * hi[0] + m2 * hi[1] + m3 * hi[2]);
          gy += tt * 2 * ORC_PI * (m1 * hi[3] + m2 * hi[4] + m3 * hi[5]);
          gz += tt * 2 * ORC_PI * (m1 * hi[6] + m2 * hi[7] + m3 * hi[8]);
        } else {
          acc += gf[k] * (er * Sre[k] + ei * Sim[k]);
        }
      }
      if (grad) {
        y[3 * o] += gx;
        y[3 * o + 1] += gy;
        y[3 * o + 2] += gz;
      } else {
        y[o] += acc;
      }
    }
    free(t);
  }
  free(Sre);
  free(Sim);
  free(gm);
  free(gf);
  cells_free(&cl);
  free(u);
  return 0;
}

int oracle_ewald_matvec(int n, const double* cell, const double* pos, const double* sigma,
                        const double* q, double omega, double r_cut, double g_cut,
                        int n_rows, const int* rows, double* y) {
  return ewald_rows(n, cell, pos, sigma, q, omega, r_cut, g_cut, n_rows, rows, 0, y);
}

/*
 * g = the gradient, at atom i, of the potential of the charges q:
 *   g_i = d/dR_i sum_j A_ij q_j  (R_j, j != i, and q fixed; k_e = 1)
 * term by term from the same Ewald split (SI "Ewald Summation"):
 *   real space   sum_{j,n} q_j pair'(r) (R_i - R_j - n)/r   (j = i: the images of i
 *                itself do not move relative to i and drop out)
 *   reciprocal   sum_G f(G) G [S_im cos(G.r_i) - S_re sin(G.r_i)], S(G) = sum_j q_j e^{iG.r_j}
 *                (the j = i part of S cancels exactly)
 *   self, G = 0 width terms: independent of the positions.
 * These are the position derivatives that enter the force trick (SI eq.
 * 4g_force_trick).  Output g[3 o + c] for row o, like oracle_ewald_matvec.
 */
int oracle_ewald_potential_grad(int n, const double* cell, const double* pos, const double* sigma,
                                const double* q, double omega, double r_cut, double g_cut,
                                int n_rows, const int* rows, double* g) {
  return ewald_rows(n, cell, pos, sigma, q, omega, r_cut, g_cut, n_rows, rows, 1, g);
}

/*
 * Strain derivative of the bilinear form W = w^T A q (k_e = 1), A the Coulomb
 * matrix of oracle_ewald_matvec, under the homogeneous deformation of cell and
 * positions r -> (1 + eps) r:  D[3 a + b] = dW/d eps_ab.  Term by term from the
 * Ewald split (SI "Ewald Summation"), with a single width omega >= every gamma_ij:
 *   real space   sum_i w_i sum_{j,n} q_j pair'(r) d_a d_b / r,  d = r_j + n - r_i
 *                (the images of i itself included: their separation is strained too)
 *   reciprocal   sum_G f(G) Re[conj(S_w(G)) S_q(G)] (-delta_ab + G_a G_b (omega^2 + 2/G^2)),
 *                f(G) = (4 pi/V) exp(-G^2 omega^2/2)/G^2, since dG^2/d eps_ab = -2 G_a G_b
 *                and dV/d eps_ab = V delta_ab
 *   G = 0 width  +(2 pi/V) sum_ij w_i q_j (w_ij^2 - gamma_ij^2) delta_ab
 *   self terms   independent of the strain.
 * The stress of the form is D / V.  Sums over atoms and G run in a fixed order.
 */
int oracle_ewald_strain_derivative(int n, const double* cell, const double* pos, const double* sigma,
                                   const double* w, const double* q, double omega, double r_cut,
                                   double g_cut, double* D) {
  double hi[9], wd[3];
  inv3(cell, hi);
  plane_widths(cell, wd);
  double V = fabs(det3(cell));
  double* u = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  double* per = (double*)calloc((size_t)n * 9, sizeof(double));
  if (!u || !per) return 1;
  to_frac(n, hi, pos, u);
  for (int i = 0; i < 3 * n; ++i) u[i] -= floor(u[i]);
  CellList cl;
  if (cells_build(n, u, wd, r_cut, &cl)) return 1;
  double rc2 = r_cut * r_cut;
  for (int k = 0; k < 9; ++k) D[k] = 0.0;

  /* ---------------- real space, per atom, then summed in atom order */
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; ++i) {
    if (w[i] == 0.0) continue;
    double si = sigma[i];
    double* acc = per + 9 * (size_t)i;
    CELLS_FOR_NEIGHBOURS(cl, u, cell, i, rc2, {
      double sj = sigma[j];
      double g = sqrt(si * si + sj * sj);
      double wi = g > omega ? g : omega;
      double r = sqrt(r2);
      if (r > 1e-12) {
        double t = w[i] * q[j] * pair_real_deriv(r, g, wi) / r;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc[3 * a + b] += t * d[a] * d[b];
      }
    });
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 9; ++k) D[k] += per[9 * (size_t)i + k];
  free(per);

  /* ---------------- G = 0 width term */
  {
    WidthSums ws;
    if (width_sums(n, sigma, q, &ws)) return 2;
    double acc = 0.0;
    for (int i = 0; i < n; ++i)
      if (w[i] != 0.0) acc += w[i] * width_term(&ws, sigma[i], omega);
    for (int a = 0; a < 3; ++a) D[4 * a] += (2.0 * ORC_PI / V) * acc;
  }

  /* ---------------- reciprocal space over the half-space of G (gf holds the factor 2) */
  int M[3];
  int* gm;
  double* gf;
  long ng = gvecs_build(hi, wd, V, omega, g_cut, M, &gm, &gf);
  if (ng < 0) return 1;
  double* S = (double*)calloc((size_t)ng * 4, sizeof(double));
  if (!S || structure_factor(n, u, w, M, ng, gm, S, S + ng) ||
      structure_factor(n, u, q, M, ng, gm, S + 2 * ng, S + 3 * ng))
    return 1;
  for (long k = 0; k < ng; ++k) {
    double G[3];
    for (int e = 0; e < 3; ++e)
      G[e] = 2 * ORC_PI * (gm[3 * k] * hi[3 * e] + gm[3 * k + 1] * hi[3 * e + 1] + gm[3 * k + 2] * hi[3 * e + 2]);
    double G2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    double e = gf[k] * (S[k] * S[2 * ng + k] + S[ng + k] * S[3 * ng + k]);
    double k2 = omega * omega + 2.0 / G2;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) D[3 * a + b] += e * ((a == b ? -1.0 : 0.0) + G[a] * G[b] * k2);
  }
  free(S);
  free(gm);
  free(gf);
  cells_free(&cl);
  free(u);
  return 0;
}
