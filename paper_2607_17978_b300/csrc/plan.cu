// Plan creation: per-structure Ewald split, mesh and B-spline choice, FFT
// radix plans and work lists, and all device workspace (qeq_solve allocates
// nothing).  Parameter choice follows the paper's particle-mesh solver (SI
// "Particle-Particle-Particle-Mesh Method": the split width is tied to the
// Gaussian widths and the mesh resolves the narrowest reciprocal Gaussian) and
// SI "Ewald Summation" (real-space cutoff from the target accuracy).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "qeq_internal.cuh"

namespace {

const double kPi = 3.14159265358979323846;

bool smooth235(int n) {
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

int next_smooth(int n) {
  while (!smooth235(n)) ++n;
  return n;
}

// cardinal B-spline M_p at the integers 0..p-1 (same order recursion as prep.cu, at w = 0)
void bspline_at_integers(int p, double* out) {
  double a[QEQ_MAXP + 1] = {0};
  a[0] = 0.0;
  a[1] = 1.0;
  for (int n = 2; n < p; ++n) {
    a[n] = 0.0;
    for (int j = n; j >= 0; --j) {
      double x = j;
      double left = a[j], right = (j > 0) ? a[j - 1] : 0.0;
      a[j] = (x * left + (n + 1 - x) * right) / n;
    }
  }
  for (int j = 0; j < p; ++j) out[j] = a[j];
}

// |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K)|^2  (smooth PME moduli)
void bspline_moduli(int K, int p, double* out) {
  double M[QEQ_MAXP];
  bspline_at_integers(p, M);
  for (int m = 0; m < K; ++m) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= p - 2; ++k) {
      double ph = 2.0 * kPi * (double)m * k / K;
      re += M[k + 1] * cos(ph);
      im += M[k + 1] * sin(ph);
    }
    double d = re * re + im * im;
    out[m] = d > 1e-30 ? 1.0 / d : 0.0;
  }
}

template <typename T>
cudaError_t dalloc(qeq_plan_s* P, T** ptr, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e == cudaSuccess) P->workspace_bytes += bytes;
  return e;
}

template <typename T>
cudaError_t upload(qeq_plan_s* P, T** ptr, const std::vector<T>& v) {
  QEQ_CUDA_TRY(dalloc(P, ptr, v.size()));
  if (!v.empty()) QEQ_CUDA_TRY(cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return cudaSuccess;
}

// int_0^rc r erfc(r/a) dr = a^2/4 - [(a^2/4 - rc^2/2) erfc(rc/a) + a rc/(2 sqrt pi) exp(-rc^2/a^2)]
double sphere_int(double a, double rc) {
  double tail = (0.25 * a * a - 0.5 * rc * rc) * erfc(rc / a) + a * rc / (2.0 * sqrt(kPi)) * exp(-rc * rc / (a * a));
  return 0.25 * a * a - tail;
}

// Ewald split width from the real-space cutoff: erfc(r_cut / (sqrt2 omega)) = ewald_tol / 10
double split_width(const qeq_plan_desc& D) { return D.r_cut / (sqrt(2.0) * erfc_inv(0.1 * D.ewald_tol)); }

// narrowest reciprocal Gaussian width w_st = max(gamma_st, omega) of a structure
double narrowest_width(const double* sig, int S, double omega) {
  double wmin = 1e300;
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b) {
      if (!(sig[a] > 0.0) || !(sig[b] > 0.0)) continue;
      double g = sqrt(sig[a] * sig[a] + sig[b] * sig[b]);
      wmin = std::min(wmin, g < 0.999 * omega ? omega : g);
    }
  return wmin;
}

// Mesh for B-spline order pp.  An explicit mesh_spacing is honoured; otherwise
// the spacing comes from an error model fitted to measured smooth-PME errors
// of the matvec on equilibrium (solution) charge vectors against the dense
// Ewald matrix: rel. error ~ max(10^(a_p + b_p h / w_min), floor_p), h the
// spacing between lattice planes.  Returns false if no mesh of at most 1000
// points per direction is predicted to reach ewald_tol / 2.
// cost ~ mesh traffic + spline work per atom.
bool choose_mesh(const double* h, double V, double wmin, double n_atoms, int pp, const qeq_plan_desc& D, int* K,
                 double* cost) {
  double a = (pp == 4) ? -7.0 : (pp == 6 ? -9.5 : -11.5);
  double b = (pp == 4) ? 10.0 : (pp == 6 ? 10.8 : 12.6);
  double floor_p = (pp == 4) ? 1e-5 : (pp == 6 ? 7e-7 : 2e-8);
  double target = 0.5 * D.ewald_tol;
  double hsp;
  if (D.mesh_spacing > 0) {
    hsp = D.mesh_spacing;
  } else {
    if (floor_p > target) return false;
    hsp = (log10(target) - a) / b * wmin;
  }
  if (!(hsp > 0)) return false;
  double wd[3];
  plane_widths(h, V, wd);
  for (int d = 0; d < 3; ++d) {
    int k = (int)ceil(wd[d] / hsp - 1e-9);
    k = next_smooth(std::max(k, std::max(2 * pp, 12)));
    if (k > 1000) return false;
    K[d] = k;
  }
  double M = (double)K[0] * K[1] * K[2];
  *cost = M * (14.0 + 0.2 * log2(M)) + n_atoms * pp * pp * pp * 0.25;
  return true;
}


}  // namespace

static qeq_status fail(qeq_plan_s* P, qeq_status st, const std::string& msg) {
  if (P) P->last_error = msg;
  return st;
}

static void free_plan(qeq_plan_s* P) {
  if (!P) return;
  void* ptrs[] = {P->d_st,     P->d_fft,     P->d_tw64,    P->d_tw32,     P->d_bmod,    P->d_bmod32,   P->d_bmod_dd,
                  P->d_zitems, P->d_yitems,  P->d_xitems,  P->d_yiitems,  P->d_bin_struct, P->d_atom_struct, P->d_brick_struct, P->d_brick_cand,
                  P->d_chunks, P->d_key,     P->d_bin_count, P->d_bin_start, P->d_bin_fill, P->d_perm,
                  P->d_scan_tmp, P->d_base,  P->d_wts,     P->d_wts32,    P->d_spec,    P->d_J,
                  P->d_chi,    P->d_dinv,    P->d_posc,    P->d_row,      P->d_row_cnt, P->d_col,
                  P->d_val64,  P->d_val32,   P->d_q,       P->d_r,        P->d_z,       P->d_p,
                  P->d_Ap,     P->d_x,       P->d_mesh,    P->d_mesh2,   P->d_part,     P->d_counter, P->d_sc,
                  P->d_err,    P->d_done,    P->d_stp,     P->d_pzitems,  P->d_pyitems, P->d_pxitems, P->d_pyiitems, P->d_fft_tabs,
                  P->d_pmesh,  P->d_pmesh2,  P->d_w1,      P->d_u,        P->d_pbase,   P->d_pw,     P->d_pre_tiles,
                  P->d_x32,    P->d_posc32,  P->d_q1,      P->d_r1,       P->d_reject,  P->d_xitem_off, P->d_stress_part,
                  P->d_sqnm_dx, P->d_sqnm_dg, P->d_sqnm_g, P->d_sqnm_part, P->d_sqnm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (P->h_done) cudaFreeHost(P->h_done);
  if (P->d_feat) cudaFree(P->d_feat);
  if (P->d_pred) cudaFree(P->d_pred);
  if (P->ev_done) cudaEventDestroy(P->ev_done);
  if (P->graph_solve) cudaGraphExecDestroy(P->graph_solve);
  if (P->d_ctl) cudaFree(P->d_ctl);
}

extern "C" const char* qeq_status_str(qeq_status s) {
  switch (s) {
    case QEQ_OK: return "ok";
    case QEQ_ERR_INVALID: return "invalid argument or input";
    case QEQ_ERR_NOT_PD: return "QEq matrix not positive definite (J <= 0 or sigma <= 0)";
    case QEQ_ERR_NOCONV: return "PCG did not converge within max_iter";
    case QEQ_ERR_CUDA: return "CUDA runtime error";
    case QEQ_ERR_OOM: return "device allocation failed";
    case QEQ_ERR_TIMEOUT: return "bounded device wait timed out";
    case QEQ_ERR_CAPACITY: return "real-space pair list exceeds the plan's capacity";
  }
  return "unknown status";
}

extern "C" const char* qeq_last_error(qeq_plan plan) {
  if (!plan) return "null plan";
  return plan->last_error.c_str();
}

extern "C" void qeq_plan_destroy(qeq_plan plan) {
  if (!plan) return;
  free_plan(plan);
  delete plan;
}

extern "C" qeq_status qeq_plan_query(qeq_plan P, int32_t s, qeq_plan_info* out) {
  if (!P || !out) return QEQ_ERR_INVALID;
  if (s < 0 || s >= P->n_struct) return fail(P, QEQ_ERR_INVALID, "structure index out of range");
  const StructDev& S = P->hs[s];
  for (int d = 0; d < 3; ++d) out->mesh[d] = S.K[d];
  out->spline_order = S.p;
  out->n_species = S.S;
  int nn = 0;
  for (int a = 0; a < S.S; ++a)
    for (int b = a; b < S.S; ++b) nn += (S.narrow[a] >> b) & 1u;
  out->narrow_pairs = nn;
  out->omega = S.omega;
  out->r_cut = S.r_cut;
  out->volume = S.V;
  out->n_atoms = S.atom_end - S.atom_begin;
  out->pair_capacity = P->pair_cap;
  out->workspace_bytes = P->workspace_bytes;
  out->kernel_launches = P->launches;
  return QEQ_OK;
}

static qeq_status build_plan(qeq_plan_s* P) {
  qeq_plan_desc& D = P->desc;
  const int ns = D.n_struct;
  const int S = D.n_species;
  const int p = D.spline_order;
  P->n_struct = ns;
  P->offsets.assign(D.atom_offsets, D.atom_offsets + ns + 1);
  P->n_atoms = P->offsets[ns];
  P->precision = D.precision;
  P->max_p = 0;
  P->max_S = S;
  P->max_ncm = (S + 1) / 2;

  std::vector<StructDev> hs(ns);
  std::map<int, int> fft_index;
  std::vector<FftPlanDev> fplans;
  std::vector<double2> tw64;
  std::vector<float2> tw32;
  std::vector<double> bmod;
  std::vector<float> bmod32;
  std::vector<int> tabs;
  std::vector<int4> zit, yit, yiit, xit;
  std::vector<int> bin_struct, brick_struct, brick_cand;
  std::vector<Chunk> chunks;
  int64_t mesh_off = 0;
  int bin_off = 0;
  int64_t pair_cap = 0;


  // B-spline order: one per plan (the kernels are specialised on it); when not
  // given, the order with the smallest summed cost over all structures
  int pbest = p;
  if (pbest == 0) {
    const double omega = split_width(D);
    double best = 1e300;
    for (int pp : {4, 6, 8}) {
      double tot = 0.0;
      bool ok = true;
      for (int s = 0; s < ns && ok; ++s) {
        const double* h = D.cells + 9 * s;
        double V = fabs(det3(h)), c = 0;
        int K[3];
        ok = V > 1e-9 && choose_mesh(h, V, narrowest_width(D.sigma + (size_t)S * s, S, omega),
                                     (double)(P->offsets[s + 1] - P->offsets[s]), pp, D, K, &c);
        tot += c;
      }
      if (ok && tot < best) {
        best = tot;
        pbest = pp;
      }
    }
    if (pbest == 0) return fail(P, QEQ_ERR_INVALID, "no mesh meets ewald_tol within 1000 points per direction");
  }
  P->max_p = pbest;
  // three plans per FFT length: FP32 stages (radices up to 24), FP64 stages (up to 16), and the
  // FP64 stages with double-float twiddles
  auto fft_plan_for = [&](int K) {
    auto it = fft_index.find(K);
    if (it != fft_index.end()) return it->second;
    const int idx = (int)fplans.size();
    for (int maxR : {QEQ_MAXR32, QEQ_MAXR64}) {
      FftPlanDev f;
      memset(&f, 0, sizeof(f));
      f.tw_off = (int)tw64.size();
      f.tab_off = (int)tabs.size();
      const int padK = K + (K & 1);  // keeps every twiddle table 16-byte aligned
      tw64.resize(tw64.size() + padK);
      tw32.resize(tw32.size() + padK);
      tabs.resize(tabs.size() + 3 * (size_t)((K + 3) & ~3));
      if (!fft_plan_fill(K, f, tw64.data() + f.tw_off, tw32.data() + f.tw_off, tabs.data() + f.tab_off, maxR))
        return -1;
      fplans.push_back(f);
    }
    {  // third plan: the FP64 stages with double-float twiddles (hi, lo of cos, then of sin) in
       // 16-byte slots of the FP64 array
      FftPlanDev f = fplans[idx + 1];
      const int padK = K + (K & 1);
      const int off64 = f.tw_off;
      f.tw_off = (int)tw64.size();
      tw64.resize(tw64.size() + padK);
      tw32.resize(tw32.size() + padK);
      for (int m = 0; m < padK; ++m) {
        const double2 t = tw64[off64 + m];
        float q[4];
        q[0] = (float)t.x;
        q[1] = (float)(t.x - (double)q[0]);
        q[2] = (float)t.y;
        q[3] = (float)(t.y - (double)q[2]);
        memcpy(&tw64[f.tw_off + m], q, sizeof(q));
      }
      fplans.push_back(f);
    }
    fft_index[K] = idx;
    return idx;
  };
  int maxK[3] = {1, 1, 1};
  int max_s = 1;

  for (int s = 0; s < ns; ++s) {
    StructDev& T = hs[s];
    memset(&T, 0, sizeof(T));
    const double* h = D.cells + 9 * s;
    for (int k = 0; k < 9; ++k) {
      if (!std::isfinite(h[k])) return fail(P, QEQ_ERR_INVALID, "non-finite cell");
      T.h[k] = h[k];
    }
    double V = fabs(det3(h));
    if (!(V > 1e-9)) return fail(P, QEQ_ERR_INVALID, "singular cell");
    inv3(h, T.hinv);
    T.V = V;
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) T.B[3 * d + c] = 2.0 * kPi * T.hinv[3 * c + d];
    T.green_pref = D.coulomb_k * 4.0 * kPi / V;
    // species of this structure: the table width minus trailing entries with sigma <= 0
    int Ss = S;
    while (Ss > 1 && !(D.sigma[(size_t)S * s + Ss - 1] > 0.0)) --Ss;
    T.S = Ss;
    T.ncm = (Ss + 1) / 2;
    max_s = std::max(max_s, Ss);
    T.p = pbest;
    T.atom_begin = P->offsets[s];
    T.atom_end = P->offsets[s + 1];
    if (T.atom_end <= T.atom_begin) return fail(P, QEQ_ERR_INVALID, "structure without atoms");
    const double* sig = D.sigma + (size_t)S * s;
    for (int a = 0; a < Ss; ++a)
      if (!(sig[a] > 0.0) || !std::isfinite(sig[a])) return fail(P, QEQ_ERR_NOT_PD, "sigma must be finite and > 0");
    // --- Ewald split: omega from the real-space cutoff and the target accuracy
    double rc = D.r_cut;
    double omega = split_width(D);
    T.r_cut = rc;
    T.omega = omega;
    double wmin = 1e300;
    int any = 0;
    for (int a = 0; a < Ss; ++a) {
      for (int b = 0; b < Ss; ++b) {
        double g = sqrt(sig[a] * sig[a] + sig[b] * sig[b]);
        bool narrow = g < 0.999 * omega;
        double w = narrow ? omega : g;
        int k = a * QEQ_MAX_SPECIES + b;
        T.w2[k] = w * w;
        // G = 0 width term restricted to the real-space sphere r < r_cut, the same
        // region the pair sum covers: k_e (4 pi / V) int_0^rc r [erfc(r/(sqrt2 w)) - erfc(r/(sqrt2 g))] dr.
        // With rc -> infinity this is k_e (2 pi / V)(w^2 - g^2); truncating both
        // consistently leaves only the charge fluctuations beyond r_cut unaccounted.
        T.corr[k] = narrow ? D.coulomb_k * (4.0 * kPi / V) * (sphere_int(sqrt(2.0) * w, rc) - sphere_int(sqrt(2.0) * g, rc))
                           : 0.0;
        T.inv_sw[k] = 1.0 / (sqrt(2.0) * w);
        T.inv_sg[k] = 1.0 / (sqrt(2.0) * g);
        if (narrow) {
          T.narrow[a] |= 1u << b;
          any = 1;
        }
        wmin = std::min(wmin, w);
      }
      double g = sqrt(2.0) * sig[a];
      double w = (g < 0.999 * omega) ? omega : g;
      T.self_s[a] = D.coulomb_k * sqrt(2.0 / kPi) * (1.0 / g - 1.0 / w);
      T.sigma_s[a] = sig[a];
      T.diag_s[a] = D.coulomb_k / (sig[a] * sqrt(kPi));
    }
    T.any_narrow = any;
    // --- mesh for the plan's B-spline order
    double wd[3];
    plane_widths(h, V, wd);
    for (int d = 0; d < 3; ++d)  // periodic images are indexed with 8 bits
      if (std::max(rc, (double)QEQ_MLP_RCUT) > 100.0 * wd[d])
        return fail(P, QEQ_ERR_INVALID, "cell narrower than 1/100 of the real-space cutoff");
    int Kbest[3];
    double cst;
    if (!choose_mesh(h, V, wmin, (double)(T.atom_end - T.atom_begin), pbest, D, Kbest, &cst))
      return fail(P, QEQ_ERR_INVALID, "no mesh meets ewald_tol within 1000 points per direction");
    for (int d = 0; d < 3; ++d) {
      int K = Kbest[d];
      T.K[d] = K;
      (void)cst;
      T.nb[d] = (K + QEQ_BIN - 1) / QEQ_BIN;
      T.nbr[d] = (K + (d == 2 ? QEQ_BRICK_Z : QEQ_BRICK_XY) - 1) / (d == 2 ? QEQ_BRICK_Z : QEQ_BRICK_XY);
      // bins that can hold an atom within r_cut (plus one for a ragged last bin)
      double l = rc / wd[d] * K / QEQ_BIN;
      int R = (int)ceil(l + 1.0 / QEQ_BIN) + ((K % QEQ_BIN) ? 1 : 0);
      T.rs_range[d] = std::max(1, R);
      double lf = QEQ_MLP_RCUT / wd[d] * K / QEQ_BIN;
      T.feat_range[d] = std::max(1, (int)ceil(lf + 1.0 / QEQ_BIN) + ((K % QEQ_BIN) ? 1 : 0));
    }
    mesh_layout(T);
    T.mesh_off = mesh_off;
    mesh_off += T.Mp * T.ncm;
    for (int d = 0; d < 3; ++d) maxK[d] = std::max(maxK[d], T.K[d]);
    T.bin_off = bin_off;
    int nbins = T.nb[0] * T.nb[1] * T.nb[2];
    for (int b = 0; b < nbins; ++b) bin_struct.push_back(s);
    bin_off += nbins;
    T.brick_off = (int)brick_struct.size();
    for (int b = 0; b < T.nbr[0] * T.nbr[1] * T.nbr[2]; ++b) {
      brick_struct.push_back(s);
      const int bc[3] = {b / (T.nbr[2] * T.nbr[1]), (b / T.nbr[2]) % T.nbr[1], b % T.nbr[2]};
      int c[QEQ_BRICK_CAND];
      brick_candidates(T, pbest, bc, c);
      brick_cand.insert(brick_cand.end(), c, c + QEQ_BRICK_CAND);
    }
    for (int d = 0; d < 3; ++d) {
      T.fft_plan[d] = fft_plan_for(T.K[d]);
      if (T.fft_plan[d] < 0) return fail(P, QEQ_ERR_INVALID, "mesh size without an FFT plan");
      T.bmod_off[d] = (int)bmod.size();
      std::vector<double> bm(T.K[d]);
      bspline_moduli(T.K[d], T.p, bm.data());
      for (double v : bm) {
        bmod.push_back(v);
        bmod32.push_back((float)v);
      }
    }
    // --- real-space pair capacity: local density bound with margin
    if (any) {
      int64_t n = T.atom_end - T.atom_begin;
      double per = (double)n / V * (4.0 / 3.0) * kPi * rc * rc * rc;
      pair_cap += n * (int64_t)ceil(1.5 * per + 16.0);
    }
    // --- reduction chunks
    int first = (int)chunks.size();
    int64_t nat = T.atom_end - T.atom_begin;
    int cnt = (int)((nat + QEQ_CHUNK - 1) / QEQ_CHUNK);
    for (int c = 0; c < cnt; ++c) {
      Chunk ch;
      ch.s = s;
      ch.begin = T.atom_begin + (int64_t)c * QEQ_CHUNK;
      ch.end = std::min<int64_t>(T.atom_end, ch.begin + QEQ_CHUNK);
      ch.first = first;
      ch.count = cnt;
      ch.last = (c == cnt - 1);
      chunks.push_back(ch);
    }
  }
  // --- FFT tile sizes from the largest mesh of the plan, then the work lists
  P->geo = fft_geometry(maxK, (max_s + 1) / 2);
  std::vector<int> xoff(1, 0);
  for (int s = 0; s < ns; ++s) {
    fft_work_lists(hs[s], s, P->geo.tl, P->geo.tlx, [&](int4 v) { zit.push_back(v); },
                   [&](int4 v) { yit.push_back(v); }, [&](int4 v) { yiit.push_back(v); },
                   [&](int4 v) { xit.push_back(v); });
    xoff.push_back((int)xit.size());
  }
  // --- Fourier preconditioner: a coarse mesh per structure (spacing ~2 A, cubic B-splines)
  std::vector<StructDev> hsp;
  std::vector<int4> pzit, pyit, pyiit, pxit;
  int64_t pmesh_off = 0;
  if (D.preconditioner == QEQ_PRECOND_FOURIER) {
    const double kPreSpacing = D.precond_spacing;
    int maxKp[3] = {8, 8, 8};
    for (int s = 0; s < ns; ++s) {
      StructDev Tp = hs[s];
      double wd[3];
      plane_widths(Tp.h, Tp.V, wd);
      for (int d = 0; d < 3; ++d) {
        Tp.K[d] = next_smooth(std::max(8, (int)ceil(wd[d] / kPreSpacing - 1e-9)));
        maxKp[d] = std::max(maxKp[d], Tp.K[d]);
      }
      hsp.push_back(Tp);
    }
    P->pgeo = fft_geometry(maxKp, 1);
    for (int d = 0; d < 3; ++d) P->pfft_kmax[d] = maxKp[d];
    for (int s = 0; s < ns; ++s) {
      StructDev& Tp = hsp[s];
      Tp.S = 1;
      Tp.ncm = 1;
      Tp.p = 4;
      mesh_layout(Tp);
      Tp.mesh_off = pmesh_off;
      pmesh_off += Tp.Mp;
      // Gaussian width of the long-range part it inverts: as given, else 3 A for cells up to
      // 80 A wide and 4.5 A above (measured: 17 against 21 iterations at 68 A; at 135 A,
      // sheared, 3 A left the preconditioner close to Jacobi; at 282 A both gave ~105)
      double pwd[3];
      plane_widths(Tp.h, Tp.V, pwd);
      const double kPreWidth =
          D.precond_width > 0 ? D.precond_width : (std::min(pwd[0], std::min(pwd[1], pwd[2])) <= 80.0 ? 3.0 : 4.5);
      for (int k = 0; k < QEQ_MAX_SPECIES * QEQ_MAX_SPECIES; ++k) Tp.w2[k] = kPreWidth * kPreWidth;
      Tp.green_pref = hs[s].green_pref;
      Tp.omega = D.precond_scale;  // the coarse mesh carries beta in the otherwise unused split width
      {  // g0 at the smallest nonzero reciprocal vector (small integer combinations of the basis)
        double g2min = 1e300;
        for (int m0 = -2; m0 <= 2; ++m0)
          for (int m1 = -2; m1 <= 2; ++m1)
            for (int m2 = -2; m2 <= 2; ++m2) {
              if (!m0 && !m1 && !m2) continue;
              double g2 = 0.0;
              for (int c = 0; c < 3; ++c) {
                double gc = m0 * Tp.B[c] + m1 * Tp.B[3 + c] + m2 * Tp.B[6 + c];
                g2 += gc * gc;
              }
              g2min = std::min(g2min, g2);
            }
        Tp.pre_g0max = Tp.green_pref * exp(-0.5 * g2min * kPreWidth * kPreWidth) / g2min;
      }
      for (int d = 0; d < 3; ++d) {
        Tp.fft_plan[d] = fft_plan_for(Tp.K[d]);
        if (Tp.fft_plan[d] < 0) return fail(P, QEQ_ERR_INVALID, "mesh size without an FFT plan");
        Tp.bmod_off[d] = (int)bmod.size();
        std::vector<double> bm(Tp.K[d]);
        bspline_moduli(Tp.K[d], 4, bm.data());
        for (double v : bm) {
          bmod.push_back(v);
          bmod32.push_back((float)v);
        }
      }
      fft_work_lists(Tp, s, P->pgeo.tl, P->pgeo.tlx, [&](int4 v) { pzit.push_back(v); },
                     [&](int4 v) { pyit.push_back(v); }, [&](int4 v) { pyiit.push_back(v); },
                     [&](int4 v) { pxit.push_back(v); });
    }
  }
  // tile groups of the coarse spread: QEQ_PRE_TILE_G x QEQ_PRE_TILE_G fine bin columns and
  // gz bins in z, gz as large as keeps the largest tile (8-byte points) within 64 KB
  std::vector<int4> ptiles;
  if (D.preconditioner == QEQ_PRECOND_FOURIER) {
    const int G = QEQ_PRE_TILE_G;
    auto tile_bytes = [&](int gz) {
      int mx = 0;
      for (int s = 0; s < ns; ++s) {
        const StructDev& F = hs[s];
        const StructDev& C = hsp[s];
        int e[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d) {
          const int g = (d == 2) ? gz : G;
          for (int b0 = 0; b0 < F.nb[d]; b0 += g) {
            int o, ext;
            pre_tile_range(b0, g, F.nb[d], C.K[d], F.K[d], o, ext);
            e[d] = std::max(e[d], ext);
          }
        }
        mx = std::max(mx, e[0] * e[1] * e[2] * 8);
      }
      return mx;
    };
    int max_nbz = 1;
    for (int s = 0; s < ns; ++s) max_nbz = std::max(max_nbz, hs[s].nb[2]);
    int gz = max_nbz;
    while (gz > 1 && tile_bytes(gz) > 64 * 1024) gz = (gz + 1) / 2;
    P->pre_tile_gz = gz;
    P->pre_tile_smem = tile_bytes(gz);
    // the coarse spread launches with at most 64 KB of tile (its function attribute): a
    // coarse mesh so fine that a single-bin tile exceeds that is refused here
    if (P->pre_tile_smem > 64 * 1024)
      return fail(P, QEQ_ERR_INVALID, "preconditioner mesh too fine for its shared-memory tiles (raise precond_spacing)");
    for (int s = 0; s < ns; ++s)
      for (int bx = 0; bx < hs[s].nb[0]; bx += G)
        for (int by = 0; by < hs[s].nb[1]; by += G)
          for (int bz = 0; bz < hs[s].nb[2]; bz += gz) ptiles.push_back(make_int4(s, bx, by, bz));
    P->n_pre_tiles = (int)ptiles.size();
  }
  P->precond = D.preconditioner;
  P->hsp = hsp;
  P->n_pz = (int)pzit.size();
  P->n_py = (int)pyit.size();
  P->n_px = (int)pxit.size();
  P->n_pyi = (int)pyiit.size();
  P->total_pmesh = pmesh_off;
  P->hs = hs;
  P->hfft = fplans;
  P->total_bins = bin_off;
  P->total_bricks = (int)brick_struct.size();
  // the FP64-accurate products of a mixed plan (final checks) run their FFT passes in
  // double-float arithmetic when some structure's mesh has 2^21 points or more (measured:
  // 980,000 atoms on 480^3, check matvec 66 -> 41 ms; on small meshes of a batch the FP64
  // passes were faster) and no structure has more than two species: the x pass of up to
  // eight species keeps four complex meshes per line in registers and, in double-float,
  // spills ~2 KB per thread (its FP64 form does not), so there the FP64 passes stay
  if (max_s <= 2)
    for (int s = 0; s < ns; ++s)
      if ((int64_t)hs[s].K[0] * hs[s].K[1] * hs[s].K[2] >= (int64_t(1) << 21)) P->dd_check = 1;
  if (D.flags & QEQ_FLAG_CHECK_DD) P->dd_check = 1;
  if (D.flags & QEQ_FLAG_CHECK_FP64) P->dd_check = 0;
  P->total_mesh = mesh_off;
  P->pair_cap = pair_cap;
  P->n_chunks = (int)chunks.size();
  P->max_species = max_s;
  // gather CTAs: runs of at most 64 atoms (8 per chunk), shorter runs when chunks
  // are too few to fill the GPU (about 16 CTAs per SM of a 148-SM part)
  P->gather_split = std::max(8, std::min(QEQ_GATHER_SPLIT_MAX, (2368 + P->n_chunks - 1) / std::max(1, P->n_chunks)));
  P->n_zitems = (int)zit.size();
  P->n_yitems = (int)yit.size();
  P->n_xitems = (int)xit.size();
  P->n_yiitems = (int)yiit.size();
  P->max_ncm = (max_s + 1) / 2;
  for (int d = 0; d < 3; ++d) P->fft_kmax[d] = maxK[d];
  {
    const FftGeom& g = P->geo;
    const int hx = max_s <= 2 ? 1 : QEQ_MAX_SPECIES / 2;
    size_t big = 0;
    for (int e : {8, 16}) {  // FP32, FP64 complex elements
      const int sub = e == 8 ? g.sub32 : g.sub64, subx = e == 8 ? g.subx32 : g.subx64;
      const int ldz = e == 8 ? g.ldz32 : g.ldz64, ldy = e == 8 ? g.ldy32 : g.ldy64, ldx = e == 8 ? g.ldx32 : g.ldx64;
      big = std::max(big, (size_t)fft_buf(maxK[2], ldz, sub, e, 1, 0).bytes);
      big = std::max(big, (size_t)fft_buf(maxK[1], ldy, sub, e, 1, 0).bytes);
      big = std::max(big, (size_t)fft_buf(maxK[0], ldx, 2 * hx * subx, e, 2, fft_x_extra(subx, hx, e / 2)).bytes);
    }
    if (128 + 2 * big > 227 * 1024 - 1024) return fail(P, QEQ_ERR_INVALID, "FFT tile exceeds shared memory");
  }
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  if (P->num_sms < 1) P->num_sms = 1;

  // atom -> structure (input order)
  std::vector<int> atom_struct(P->n_atoms);
  for (int s = 0; s < ns; ++s)
    for (int64_t a = P->offsets[s]; a < P->offsets[s + 1]; ++a) atom_struct[a] = s;

  cudaError_t e = cudaSuccess;
#define ALLOC(expr)                                                                       \
  do {                                                                                    \
    e = (expr);                                                                           \
    if (e != cudaSuccess) return fail(P, e == cudaErrorMemoryAllocation ? QEQ_ERR_OOM : QEQ_ERR_CUDA, \
                                      std::string("plan allocation: ") + cudaGetErrorString(e));     \
  } while (0)
  ALLOC(upload(P, &P->d_st, hs));
  ALLOC(upload(P, &P->d_fft, fplans));
  ALLOC(upload(P, &P->d_tw64, tw64));
  ALLOC(upload(P, &P->d_tw32, tw32));
  ALLOC(upload(P, &P->d_bmod, bmod));
  ALLOC(upload(P, &P->d_bmod32, bmod32));
  {  // double-float copy (hi, lo) for the final-check passes of mixed-precision plans
    std::vector<float> bdd(2 * bmod.size());
    for (size_t i = 0; i < bmod.size(); ++i) {
      bdd[2 * i] = (float)bmod[i];
      bdd[2 * i + 1] = (float)(bmod[i] - (double)bdd[2 * i]);
    }
    ALLOC(upload(P, &P->d_bmod_dd, bdd));
  }
  ALLOC(upload(P, &P->d_zitems, zit));
  ALLOC(upload(P, &P->d_yitems, yit));
  ALLOC(upload(P, &P->d_xitems, xit));
  ALLOC(upload(P, &P->d_xitem_off, xoff));
  ALLOC(upload(P, &P->d_yiitems, yiit));
  ALLOC(upload(P, &P->d_fft_tabs, tabs));
  ALLOC(upload(P, &P->d_bin_struct, bin_struct));
  ALLOC(upload(P, &P->d_brick_struct, brick_struct));
  ALLOC(upload(P, &P->d_brick_cand, brick_cand));
  ALLOC(upload(P, &P->d_atom_struct, atom_struct));
  ALLOC(upload(P, &P->d_chunks, chunks));
  const int64_t N = P->n_atoms;
  ALLOC(dalloc(P, &P->d_key, N));
  ALLOC(dalloc(P, &P->d_bin_count, P->total_bins + 1));
  ALLOC(dalloc(P, &P->d_bin_start, P->total_bins + 1));
  ALLOC(dalloc(P, &P->d_bin_fill, P->total_bins + 1));
  ALLOC(dalloc(P, &P->d_perm, N));
  // scan scratch: per-1024 block sums of either scan (int64 for the pair rows)
  ALLOC(dalloc(P, (int64_t**)&P->d_scan_tmp, (size_t)(std::max<int64_t>(N, P->total_bins) / 1024 + 8)));
  ALLOC(dalloc(P, &P->d_base, N));
  ALLOC(dalloc(P, &P->d_wts, (size_t)N * 3 * QEQ_MAXP));
  ALLOC(dalloc(P, &P->d_wts32, (size_t)N * 3 * QEQ_MAXP));
  ALLOC(dalloc(P, &P->d_spec, N));
  ALLOC(dalloc(P, &P->d_J, N));
  ALLOC(dalloc(P, &P->d_chi, N));
  ALLOC(dalloc(P, &P->d_dinv, N));
  ALLOC(dalloc(P, &P->d_posc, (size_t)N * 3));
  ALLOC(dalloc(P, &P->d_posc32, (size_t)N));
  ALLOC(dalloc(P, &P->d_row, N + 1));
  ALLOC(dalloc(P, &P->d_row_cnt, N));
  ALLOC(dalloc(P, &P->d_col, pair_cap));
  ALLOC(dalloc(P, &P->d_val64, pair_cap));
  ALLOC(dalloc(P, &P->d_val32, pair_cap));
  for (double** v : {&P->d_q, &P->d_r, &P->d_z, &P->d_p, &P->d_Ap, &P->d_x, &P->d_q1, &P->d_r1})
    ALLOC(dalloc(P, v, N));
  ALLOC(dalloc(P, &P->d_x32, N));
  ALLOC(dalloc(P, &P->d_mesh, (size_t)P->total_mesh));
  ALLOC(dalloc(P, &P->d_mesh2, (size_t)P->total_mesh));
  // partials: species sums (8 per chunk), gather x.y (split per chunk, or bins), PCG reductions (8 per chunk)
  ALLOC(dalloc(P, &P->d_part, (size_t)P->n_chunks * QEQ_MAX_SPECIES * 2 +
                                  std::max<size_t>((size_t)P->total_bins, (size_t)P->n_chunks * QEQ_GATHER_SPLIT_MAX) + 64));
  ALLOC(dalloc(P, &P->d_counter, (size_t)ns * 4));
  ALLOC(dalloc(P, &P->d_stress_part, (size_t)P->n_chunks * (6 + 2 * QEQ_MAX_SPECIES)));
  if (D.flags & QEQ_FLAG_SQNM) {
    ALLOC(dalloc(P, &P->d_sqnm_dx, (size_t)N * QEQ_SQNM_HISTORY));
    ALLOC(dalloc(P, &P->d_sqnm_dg, (size_t)N * QEQ_SQNM_HISTORY));
    ALLOC(dalloc(P, &P->d_sqnm_g, (size_t)N));
    ALLOC(dalloc(P, &P->d_sqnm_part, (size_t)P->n_chunks * (QEQ_SQNM_NDOT + 7)));
    ALLOC(dalloc(P, &P->d_sqnm, (size_t)ns));
  }
  ALLOC(cudaMemset(P->d_counter, 0, sizeof(int) * ns * 4));
  ALLOC(dalloc(P, &P->d_sc, ns));
  ALLOC(cudaMemset(P->d_sc, 0, sizeof(PcgScalars) * ns));
  ALLOC(dalloc(P, &P->d_err, 4));
  ALLOC(cudaMemset(P->d_err, 0, sizeof(int) * 4));
  ALLOC(dalloc(P, &P->d_done, 4));
  ALLOC(dalloc(P, &P->d_reject, ns));
  ALLOC(dalloc(P, &P->d_ctl, 1));
  ALLOC(cudaMemset(P->d_reject, 0, sizeof(int) * ns));
  ALLOC(cudaHostAlloc((void**)&P->h_done, sizeof(int) * 8, cudaHostAllocDefault));
  ALLOC(cudaEventCreateWithFlags(&P->ev_done, cudaEventDisableTiming));
  if (P->precond == QEQ_PRECOND_FOURIER) {
    ALLOC(upload(P, &P->d_stp, hsp));
    ALLOC(upload(P, &P->d_pzitems, pzit));
    ALLOC(upload(P, &P->d_pyitems, pyit));
    ALLOC(upload(P, &P->d_pxitems, pxit));
    ALLOC(upload(P, &P->d_pyiitems, pyiit));
    ALLOC(dalloc(P, &P->d_pmesh, (size_t)P->total_pmesh));
    ALLOC(dalloc(P, &P->d_pmesh2, (size_t)P->total_pmesh));
    ALLOC(dalloc(P, &P->d_w1, N));
    ALLOC(dalloc(P, &P->d_u, N));
    ALLOC(dalloc(P, &P->d_pbase, N));
    ALLOC(dalloc(P, &P->d_pw, (size_t)N * 12));
    ALLOC(upload(P, &P->d_pre_tiles, ptiles));
  }
  ALLOC(matvec_set_attributes());
#undef ALLOC
  return QEQ_OK;
}

extern "C" qeq_status qeq_plan_create(const qeq_plan_desc* desc, void* cuda_stream, qeq_plan* out) {
  if (!desc || !out) return QEQ_ERR_INVALID;
  *out = nullptr;
  if (desc->n_struct < 1 || !desc->atom_offsets || !desc->cells || !desc->sigma) return QEQ_ERR_INVALID;
  if (desc->n_species < 1 || desc->n_species > QEQ_MAX_SPECIES) return QEQ_ERR_INVALID;
  if (desc->atom_offsets[0] != 0) return QEQ_ERR_INVALID;
  for (int s = 0; s < desc->n_struct; ++s)
    if (desc->atom_offsets[s + 1] <= desc->atom_offsets[s]) return QEQ_ERR_INVALID;
  if (desc->atom_offsets[desc->n_struct] > (int64_t)INT32_MAX / 4) return QEQ_ERR_INVALID;
  qeq_plan_s* P = new qeq_plan_s();
  P->desc = *desc;
  qeq_plan_desc& D = P->desc;
  if (!(D.coulomb_k > 0)) D.coulomb_k = 14.3996454784;
  if (!(D.charge_tol > 0)) D.charge_tol = 1e-5;
  if (!(D.ewald_tol > 0)) D.ewald_tol = 1e-6;
  if (!(D.r_cut > 0)) D.r_cut = 8.0;
  if (D.max_iter <= 0) D.max_iter = 1000;
  if (!(D.precond_spacing > 0)) D.precond_spacing = 2.0;
  if (!(D.precond_width > 0)) D.precond_width = 0.0;  // 0: chosen per cell size
  if (!(D.precond_scale > 0) || D.precond_scale > 1.0) D.precond_scale = 0.98;
  if (D.spline_order != 0 && D.spline_order != 4 && D.spline_order != 6 && D.spline_order != 8) {
    delete P;
    return QEQ_ERR_INVALID;
  }
  if (D.preconditioner != QEQ_PRECOND_JACOBI && D.preconditioner != QEQ_PRECOND_FOURIER) {
    delete P;
    return QEQ_ERR_INVALID;
  }
  if (D.precision != QEQ_FP64 && D.precision != QEQ_MIXED) {
    delete P;
    return QEQ_ERR_INVALID;
  }
  P->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&P->device);
  P->graph_ok = (P->stream != nullptr) && !(D.flags & QEQ_FLAG_NO_GRAPH);
  P->test_stall = (D.flags & QEQ_FLAG_TEST_STALL) ? 1 : 0;
  qeq_status st = build_plan(P);
  // the caller's description arrays are not kept
  D.atom_offsets = nullptr;
  D.cells = nullptr;
  D.sigma = nullptr;
  if (st != QEQ_OK) {
    free_plan(P);
    delete P;
    return st;
  }
  *out = P;
  return QEQ_OK;
}
