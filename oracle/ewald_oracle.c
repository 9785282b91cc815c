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
 * dense matrix and a full matrix-vector product for cells too large to store
 * the matrix.
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

/*
 * y = A q for the Coulomb part (k_e = 1, no hardness) with a single Ewald
 * width omega >= every gamma_ij, so that every pair shares the reciprocal
 * Gaussian exp(-G^2 omega^2/2).  Real space by a cell list over all images
 * within r_cut; reciprocal space by explicit structure factors over the
 * half-space of G with |G| <= g_cut (separable phase factors per atom).
 * rows: if n_rows > 0, y is only evaluated for atoms rows[0..n_rows) and
 * written to y[0..n_rows); the structure factors still use every atom.
 */
int oracle_ewald_matvec(int n, const double* cell, const double* pos, const double* sigma,
                        const double* q, double omega, double r_cut, double g_cut,
                        int n_rows, const int* rows, double* y) {
  double hi[9], wd[3];
  inv3(cell, hi);
  plane_widths(cell, wd);
  double V = fabs(det3(cell));
  int nout = n_rows > 0 ? n_rows : n;
  double* u = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!u) return 1;
  to_frac(n, hi, pos, u);
  for (int i = 0; i < 3 * n; ++i) u[i] -= floor(u[i]);

  /* ---------------- real space: cell list with image shifts */
  int nc[3], R[3];
  for (int d = 0; d < 3; ++d) {
    nc[d] = (int)floor(wd[d] / r_cut);
    if (nc[d] < 1) nc[d] = 1;
    if (nc[d] > 512) nc[d] = 512;
    R[d] = (int)ceil(r_cut * nc[d] / wd[d]);
    if (R[d] < 1) R[d] = 1;
  }
  size_t ncell = (size_t)nc[0] * nc[1] * nc[2];
  int* cstart = (int*)calloc(ncell + 1, sizeof(int));
  int* cidx = (int*)malloc(sizeof(int) * (size_t)n);
  int* acell = (int*)malloc(sizeof(int) * (size_t)n);
  if (!cstart || !cidx || !acell) return 1;
  for (int i = 0; i < n; ++i) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      c[d] = (int)floor(u[3 * i + d] * nc[d]);
      if (c[d] >= nc[d]) c[d] = nc[d] - 1;
      if (c[d] < 0) c[d] = 0;
    }
    acell[i] = (c[0] * nc[1] + c[1]) * nc[2] + c[2];
    cstart[acell[i] + 1]++;
  }
  for (size_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    int* fill = (int*)malloc(sizeof(int) * ncell);
    for (size_t c = 0; c < ncell; ++c) fill[c] = cstart[c];
    for (int i = 0; i < n; ++i) cidx[fill[acell[i]]++] = i;
    free(fill);
  }
  /* distinct widths for the G = 0 correction: sum_j (w_ij^2 - gamma_ij^2) q_j */
  double rc2 = r_cut * r_cut;

#pragma omp parallel for schedule(dynamic, 64)
  for (int o = 0; o < nout; ++o) {
    int i = n_rows > 0 ? rows[o] : o;
    int ci[3];
    int c = acell[i];
    ci[2] = c % nc[2];
    ci[1] = (c / nc[2]) % nc[1];
    ci[0] = c / (nc[1] * nc[2]);
    double si = sigma[i];
    double acc = 0.0;
    for (int a = -R[0]; a <= R[0]; ++a)
      for (int b = -R[1]; b <= R[1]; ++b)
        for (int e = -R[2]; e <= R[2]; ++e) {
          int cc[3] = {ci[0] + a, ci[1] + b, ci[2] + e}, sh[3];
          for (int d = 0; d < 3; ++d) {
            sh[d] = (int)floor((double)cc[d] / nc[d]);
            cc[d] -= sh[d] * nc[d];
          }
          int cj = (cc[0] * nc[1] + cc[1]) * nc[2] + cc[2];
          for (int t = cstart[cj]; t < cstart[cj + 1]; ++t) {
            int j = cidx[t];
            if (j == i && sh[0] == 0 && sh[1] == 0 && sh[2] == 0) continue;
            double fa = u[3 * j] + sh[0] - u[3 * i];
            double fb = u[3 * j + 1] + sh[1] - u[3 * i + 1];
            double fc = u[3 * j + 2] + sh[2] - u[3 * i + 2];
            double dx = fa * cell[0] + fb * cell[3] + fc * cell[6];
            double dy = fa * cell[1] + fb * cell[4] + fc * cell[7];
            double dz = fa * cell[2] + fb * cell[5] + fc * cell[8];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= rc2) continue;
            double sj = sigma[j];
            double g = sqrt(si * si + sj * sj);
            double w = g > omega ? g : omega;
            double r = sqrt(r2);
            acc += q[j] * ((r > 1e-12) ? pair_real(r, g, w) : pair_zero(g, w));
          }
        }
    {
      double g = sqrt(2.0) * si;
      double w = g > omega ? g : omega;
      acc += q[i] * pair_zero(g, w);
    }
    y[o] = acc;
  }
  /* G = 0 width correction, O(n) per row over the distinct widths */
  {
    int nd = 0;
    double ds[64], dq[64];
    for (int j = 0; j < n; ++j) {
      int k = 0;
      while (k < nd && ds[k] != sigma[j]) ++k;
      if (k == nd) {
        if (nd == 64) return 2;
        ds[nd] = sigma[j];
        dq[nd] = 0.0;
        ++nd;
      }
      dq[k] += q[j];
    }
    for (int o = 0; o < nout; ++o) {
      int i = n_rows > 0 ? rows[o] : o;
      double si = sigma[i], acc = 0.0;
      for (int k = 0; k < nd; ++k) {
        double g2 = si * si + ds[k] * ds[k];
        double w2 = g2 > omega * omega ? g2 : omega * omega;
        acc += dq[k] * (w2 - g2);
      }
      y[o] -= (2.0 * ORC_PI / V) * acc;
    }
  }

  /* ---------------- reciprocal space: half-space of G, |G| <= g_cut */
  int M[3];
  for (int d = 0; d < 3; ++d) {
    /* |G| >= 2 pi |m_d| / wd[d] bounds the range of m_d */
    M[d] = (int)floor(g_cut * wd[d] / (2.0 * ORC_PI)) + 1;
  }
  /* enumerate G vectors: m = (m1,m2,m3) > 0 lexicographically */
  long ng = 0, cap = 1024;
  int* gm = (int*)malloc(sizeof(int) * 3 * cap);
  double* gf = (double*)malloc(sizeof(double) * cap);
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
        }
        gm[3 * ng] = m1;
        gm[3 * ng + 1] = m2;
        gm[3 * ng + 2] = m3;
        /* factor 2 for the -G partner */
        gf[ng] = 2.0 * (4.0 * ORC_PI / V) * exp(-0.5 * G2 * omega * omega) / G2;
        ++ng;
      }
  double* Sre = (double*)calloc((size_t)ng, sizeof(double));
  double* Sim = (double*)calloc((size_t)ng, sizeof(double));
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  /* structure factors S(G) = sum_j q_j exp(i G.r_j); per-thread partials summed in thread order */
  double* part = (double*)calloc((size_t)nthr * 2 * ng, sizeof(double));
  int W0 = 2 * M[0] + 1, W1 = 2 * M[1] + 1, W2 = 2 * M[2] + 1;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* pr = part + (size_t)tid * 2 * ng;
    double* pi = pr + ng;
    double* t = (double*)malloc(sizeof(double) * 2 * (W0 + W1 + W2));
#pragma omp for schedule(static)
    for (int j = 0; j < n; ++j) {
      double* tc[3] = {t, t + 2 * W0, t + 2 * (W0 + W1)};
      int Mm[3] = {M[0], M[1], M[2]};
      for (int d = 0; d < 3; ++d)
        for (int m = -Mm[d]; m <= Mm[d]; ++m) {
          double ph = 2 * ORC_PI * m * u[3 * j + d];
          tc[d][2 * (m + Mm[d])] = cos(ph);
          tc[d][2 * (m + Mm[d]) + 1] = sin(ph);
        }
      for (long k = 0; k < ng; ++k) {
        const double* a = tc[0] + 2 * (gm[3 * k] + M[0]);
        const double* b = tc[1] + 2 * (gm[3 * k + 1] + M[1]);
        const double* c = tc[2] + 2 * (gm[3 * k + 2] + M[2]);
        double abr = a[0] * b[0] - a[1] * b[1], abi = a[0] * b[1] + a[1] * b[0];
        pr[k] += q[j] * (abr * c[0] - abi * c[1]);
        pi[k] += q[j] * (abr * c[1] + abi * c[0]);
      }
    }
    free(t);
  }
  for (int tt = 0; tt < nthr; ++tt)
    for (long k = 0; k < ng; ++k) {
      Sre[k] += part[(size_t)tt * 2 * ng + k];
      Sim[k] += part[(size_t)tt * 2 * ng + ng + k];
    }
  free(part);
  /* y_i += sum_G f(G) Re[exp(i G.r_i) conj(S(G))] */
#pragma omp parallel
  {
    double* t = (double*)malloc(sizeof(double) * 2 * (W0 + W1 + W2));
#pragma omp for schedule(static)
    for (int o = 0; o < nout; ++o) {
      int i = n_rows > 0 ? rows[o] : o;
      double* tc[3] = {t, t + 2 * W0, t + 2 * (W0 + W1)};
      int Mm[3] = {M[0], M[1], M[2]};
      for (int d = 0; d < 3; ++d)
        for (int m = -Mm[d]; m <= Mm[d]; ++m) {
          double ph = 2 * ORC_PI * m * u[3 * i + d];
          tc[d][2 * (m + Mm[d])] = cos(ph);
          tc[d][2 * (m + Mm[d]) + 1] = sin(ph);
        }
      double acc = 0.0;
      for (long k = 0; k < ng; ++k) {
        const double* a = tc[0] + 2 * (gm[3 * k] + M[0]);
        const double* b = tc[1] + 2 * (gm[3 * k + 1] + M[1]);
        const double* c = tc[2] + 2 * (gm[3 * k + 2] + M[2]);
        double abr = a[0] * b[0] - a[1] * b[1], abi = a[0] * b[1] + a[1] * b[0];
        double er = abr * c[0] - abi * c[1], ei = abr * c[1] + abi * c[0];
        acc += gf[k] * (er * Sre[k] + ei * Sim[k]);
      }
      y[o] += acc;
    }
    free(t);
  }
  free(Sre);
  free(Sim);
  free(gm);
  free(gf);
  free(cstart);
  free(cidx);
  free(acell);
  free(u);
  return 0;
}
