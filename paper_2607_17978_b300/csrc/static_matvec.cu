// qeq_matvec_static: the FP64 plane-wave matrix-vector product of one small
// periodic cell without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- for example code that
// runs while another component owns the device memory pool (a fixed arena, a
// memory-capped context), code that must not synchronise the device the way
// cudaMalloc/cudaFree can, or an embedding that only hands out input and
// output buffers.  qeq_plan_create allocates its workspace; this entry point
// instead uses the file-scope device array below, sized for one cell of at
// most QEQ_STATIC_MAX_ATOMS atoms, QEQ_STATIC_MAX_SPECIES species and
// QEQ_STATIC_MAX_MESH mesh points per direction.  Every GPU that loads the
// library holds this array until the process exits.
//
// The caller passes inputs and outputs only; the mesh, the sorted atom data,
// the real-space pair list and the small tables live in the static array.  All
// calls share it and it keeps the previous call's contents, so calls that
// overlap on the GPU (different streams or threads without ordering) race and
// give wrong results.  Counters that must start at zero are cleared every call.
// The host-side tables are staged in file-scope host arrays, so concurrent
// host threads must serialise their calls as well.
//
// The first call on a device does a one-time set-up there: it looks up the
// device address of the array with cudaGetSymbolAddress and raises the
// kernels' dynamic shared-memory limit.  Make that first call before any
// stream capture on the device.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "qeq_internal.cuh"

namespace {

const double kPiS = 3.14159265358979323846;
const int kMaxDev = 64;

// File-scope scratch: every buffer of one matvec, carved at 256-byte offsets.
static __device__ __align__(256) unsigned char g_static_scratch[QEQ_STATIC_SCRATCH_BYTES];

void* g_scratch_dev[kMaxDev] = {nullptr};
bool g_attr_done[kMaxDev] = {false};

// ---------------------------------------------------------------- host staging (no heap)
constexpr int kSM = QEQ_STATIC_MAX_MESH;
constexpr int kSNcm = QEQ_STATIC_MAX_SPECIES / 2;
struct Staging {
  StructDev st;
  FftPlanDev fft[6];       // per direction: FP32 stages, then FP64 stages
  double2 tw64[6 * kSM];
  float2 tw32[6 * kSM];
  int tabs[6 * 3 * kSM];
  double bmod[3 * kSM];
  float bmod32[3 * kSM];
  int4 zit[kSM * kSM * kSNcm];
  int4 yit[kSM * kSM * kSNcm];
  int4 yiit[kSM * kSM * kSNcm];
  int4 xit[(kSM / 2 + 1) * kSM];
  int bin_struct[(kSM / QEQ_BIN) * (kSM / QEQ_BIN) * (kSM / QEQ_BIN)];
  int brick_cand[(kSM / QEQ_BRICK_XY) * (kSM / QEQ_BRICK_XY) * (kSM / QEQ_BRICK_Z) * QEQ_BRICK_CAND];
  int atom_struct[QEQ_STATIC_MAX_ATOMS];
  Chunk chunks[(QEQ_STATIC_MAX_ATOMS + QEQ_CHUNK - 1) / QEQ_CHUNK];
};
Staging g_stage;

// Worst case of the carve below at the stated limits (every piece rounded up to 256
// bytes, as Carver does): the scratch array must hold it.
constexpr size_t carve_bytes(size_t count, size_t elem) { return ((count ? count : 1) * elem + 255) & ~(size_t)255; }
constexpr size_t kStaticWorstCase() {
  const size_t N = QEQ_STATIC_MAX_ATOMS, M = (size_t)kSM * kSM * kSM, cap = QEQ_STATIC_MAX_PAIRS;
  const size_t nbins = (kSM / QEQ_BIN) * (kSM / QEQ_BIN) * (kSM / QEQ_BIN);
  const size_t nch = (N + QEQ_CHUNK - 1) / QEQ_CHUNK;
  return carve_bytes(1, sizeof(StructDev)) + carve_bytes(6, sizeof(FftPlanDev)) + carve_bytes(6 * kSM, 16) +
         carve_bytes(6 * kSM, 8) + carve_bytes(18 * kSM, 4) + carve_bytes(3 * kSM, 8) + carve_bytes(3 * kSM, 4) +
         3 * carve_bytes((size_t)kSM * kSM * kSNcm, 16) + carve_bytes((kSM / 2 + 1) * kSM, 16) +
         carve_bytes(nbins, 4) + carve_bytes(nbins, 4) + carve_bytes(nbins * QEQ_BRICK_CAND, 4) + carve_bytes(N, 4) +
         carve_bytes(nch, sizeof(Chunk)) +
         carve_bytes(N, 4) + 3 * carve_bytes(nbins + 1, 4) + carve_bytes(N, 4) + carve_bytes(N / 1024 + 8, 8) +
         carve_bytes(N, 4) + carve_bytes(N * 3 * QEQ_MAXP, 8) + carve_bytes(N * 3 * QEQ_MAXP, 4) +
         carve_bytes(N, 4) + 3 * carve_bytes(N, 8) + carve_bytes(3 * N, 8) + carve_bytes(N, 16) +
         carve_bytes(N + 1, 8) + carve_bytes(N, 4) + carve_bytes(cap, 4) + carve_bytes(cap, 8) +
         carve_bytes(cap, 4) + 2 * carve_bytes(N, 8) + 2 * carve_bytes(M * kSNcm, 16) +
         carve_bytes(nch * QEQ_MAX_SPECIES * 2 + (nbins > nch * QEQ_GATHER_SPLIT_MAX ? nbins : nch * QEQ_GATHER_SPLIT_MAX) + 64, 8) +
         carve_bytes(4, 4) + carve_bytes(1, sizeof(PcgScalars)) + carve_bytes(4, 4);
}
static_assert(kStaticWorstCase() <= QEQ_STATIC_SCRATCH_BYTES, "static scratch smaller than the worst case of the limits");

int next_smooth_s(int n) {
  for (;; ++n) {
    int m = n;
    for (int f : {2, 3, 5})
      while (m % f == 0) m /= f;
    if (m == 1) return n;
  }
}

double sphere_int_s(double a, double rc) {
  double tail = (0.25 * a * a - 0.5 * rc * rc) * erfc(rc / a) + a * rc / (2.0 * sqrt(kPiS)) * exp(-rc * rc / (a * a));
  return 0.25 * a * a - tail;
}

void bspline_int_s(int p, double* out) {
  double a[QEQ_MAXP + 1] = {0};
  a[1] = 1.0;
  for (int n = 2; n < p; ++n) {
    a[n] = 0.0;
    for (int j = n; j >= 0; --j) {
      double x = j, left = a[j], right = (j > 0) ? a[j - 1] : 0.0;
      a[j] = (x * left + (n + 1 - x) * right) / n;
    }
  }
  for (int j = 0; j < p; ++j) out[j] = a[j];
}

// The same parameter choice as qeq_plan_create for one structure (split width
// from r_cut and ewald_tol, error-model mesh, cheapest B-spline order).
bool choose_mesh_s(const double* wd, double wmin, double n_atoms, int pp, double ewald_tol, int* K, double* cost) {
  double a = (pp == 4) ? -7.0 : (pp == 6 ? -9.5 : -11.5);
  double b = (pp == 4) ? 10.0 : (pp == 6 ? 10.8 : 12.6);
  double floor_p = (pp == 4) ? 1e-5 : (pp == 6 ? 7e-7 : 2e-8);
  double target = 0.5 * ewald_tol;
  if (floor_p > target) return false;
  double hsp = (log10(target) - a) / b * wmin;
  if (!(hsp > 0)) return false;
  for (int d = 0; d < 3; ++d) {
    int k = (int)ceil(wd[d] / hsp - 1e-9);
    k = next_smooth_s(std::max(k, std::max(2 * pp, 12)));
    if (k > 1000) return false;
    K[d] = k;
  }
  double M = (double)K[0] * K[1] * K[2];
  *cost = M * (14.0 + 0.2 * log2(M)) + n_atoms * pp * pp * pp * 0.25;
  return true;
}

__global__ void k_static_sort_in(const int* __restrict__ perm, int n, const double* __restrict__ src,
                                 double* __restrict__ dst) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) dst[a] = src[perm[a]];
}

__global__ void k_static_unsort(const int* __restrict__ perm, int n, const double* __restrict__ src,
                                double* __restrict__ dst) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) dst[perm[a]] = src[a];
}

struct Carver {
  unsigned char* base;
  size_t off, cap;
  bool ok = true;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
    if (off + bytes > cap) {
      ok = false;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

}  // namespace

extern "C" qeq_status qeq_matvec_static(const double* h_cell, const double* h_sigma, int32_t n_species,
                                        int32_t n_atoms, const double* d_pos, const int32_t* d_species,
                                        const double* d_J, const double* d_x, double* d_y, double coulomb_k,
                                        double ewald_tol, double r_cut, void* cuda_stream) {
  if (!h_cell || !h_sigma || !d_pos || !d_species || !d_x || !d_y) return QEQ_ERR_INVALID;
  if (n_atoms < 1 || n_atoms > QEQ_STATIC_MAX_ATOMS) return QEQ_ERR_CAPACITY;
  if (n_species < 1 || n_species > QEQ_STATIC_MAX_SPECIES) return QEQ_ERR_CAPACITY;
  if (!(coulomb_k > 0)) coulomb_k = 14.3996454784;
  if (!(ewald_tol > 0)) ewald_tol = 1e-6;
  if (!(r_cut > 0)) r_cut = 8.0;
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(h_cell[k])) return QEQ_ERR_INVALID;
  for (int a = 0; a < n_species; ++a)
    if (!(h_sigma[a] > 0.0) || !std::isfinite(h_sigma[a])) return QEQ_ERR_NOT_PD;
  const double V = fabs(det3(h_cell));
  if (!(V > 1e-9)) return QEQ_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // ---- one-time set-up on this device: device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return QEQ_ERR_CUDA;
  if (!g_scratch_dev[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return QEQ_ERR_CUDA;
    g_scratch_dev[dev] = ptr;
  }
  if (!g_attr_done[dev]) {
    if (matvec_set_attributes() != cudaSuccess) return QEQ_ERR_CUDA;
    g_attr_done[dev] = true;
  }

  // ---- host tables for this cell (the same choices as qeq_plan_create)
  Staging& G = g_stage;
  StructDev& T = G.st;
  memset(&T, 0, sizeof(T));
  const int S = n_species;
  for (int k = 0; k < 9; ++k) T.h[k] = h_cell[k];
  inv3(h_cell, T.hinv);
  T.V = V;
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) T.B[3 * d + c] = 2.0 * kPiS * T.hinv[3 * c + d];
  T.green_pref = coulomb_k * 4.0 * kPiS / V;
  T.S = S;
  T.ncm = (S + 1) / 2;
  T.atom_begin = 0;
  T.atom_end = n_atoms;
  const double omega = r_cut / (sqrt(2.0) * erfc_inv(0.1 * ewald_tol));
  T.r_cut = r_cut;
  T.omega = omega;
  double wmin = 1e300;
  int any = 0;
  for (int a = 0; a < S; ++a) {
    for (int b = 0; b < S; ++b) {
      double g = sqrt(h_sigma[a] * h_sigma[a] + h_sigma[b] * h_sigma[b]);
      bool narrow = g < 0.999 * omega;
      double w = narrow ? omega : g;
      int k = a * QEQ_MAX_SPECIES + b;
      T.w2[k] = w * w;
      T.corr[k] = narrow ? coulomb_k * (4.0 * kPiS / V) * (sphere_int_s(sqrt(2.0) * w, r_cut) -
                                                           sphere_int_s(sqrt(2.0) * g, r_cut))
                         : 0.0;
      T.inv_sw[k] = 1.0 / (sqrt(2.0) * w);
      T.inv_sg[k] = 1.0 / (sqrt(2.0) * g);
      if (narrow) {
        T.narrow[a] |= 1u << b;
        any = 1;
      }
      wmin = std::min(wmin, w);
    }
    double g = sqrt(2.0) * h_sigma[a];
    double w = (g < 0.999 * omega) ? omega : g;
    T.self_s[a] = coulomb_k * sqrt(2.0 / kPiS) * (1.0 / g - 1.0 / w);
    T.sigma_s[a] = h_sigma[a];
    T.diag_s[a] = coulomb_k / (h_sigma[a] * sqrt(kPiS));
  }
  T.any_narrow = any;
  double wd[3];
  for (int d = 0; d < 3; ++d) {
    const double* a1 = h_cell + 3 * ((d + 1) % 3);
    const double* a2 = h_cell + 3 * ((d + 2) % 3);
    double cx = a1[1] * a2[2] - a1[2] * a2[1], cy = a1[2] * a2[0] - a1[0] * a2[2], cz = a1[0] * a2[1] - a1[1] * a2[0];
    wd[d] = V / sqrt(cx * cx + cy * cy + cz * cz);
  }
  int pbest = 0, Kb[3] = {0, 0, 0};
  double best = 1e300;
  for (int pp : {4, 6, 8}) {
    int K[3];
    double c;
    if (choose_mesh_s(wd, wmin, n_atoms, pp, ewald_tol, K, &c) && c < best) {
      best = c;
      pbest = pp;
      for (int d = 0; d < 3; ++d) Kb[d] = K[d];
    }
  }
  if (pbest == 0) return QEQ_ERR_INVALID;
  for (int d = 0; d < 3; ++d)
    if (Kb[d] > QEQ_STATIC_MAX_MESH) return QEQ_ERR_CAPACITY;
  T.p = pbest;
  for (int d = 0; d < 3; ++d) {
    int K = Kb[d];
    T.K[d] = K;
    T.nb[d] = (K + QEQ_BIN - 1) / QEQ_BIN;
    T.nbr[d] = (K + (d == 2 ? QEQ_BRICK_Z : QEQ_BRICK_XY) - 1) / (d == 2 ? QEQ_BRICK_Z : QEQ_BRICK_XY);
    double l = r_cut / wd[d] * K / QEQ_BIN;
    int R = (int)ceil(l + 1.0 / QEQ_BIN) + ((K % QEQ_BIN) ? 1 : 0);
    T.rs_range[d] = std::max(1, R);
  }
  mesh_layout(T);
  T.mesh_off = 0;
  T.bin_off = 0;
  const int nbins = T.nb[0] * T.nb[1] * T.nb[2];
  for (int b = 0; b < nbins; ++b) G.bin_struct[b] = 0;
  T.brick_off = 0;
  const int nbricks = T.nbr[0] * T.nbr[1] * T.nbr[2];
  for (int b = 0; b < nbricks; ++b) {
    const int bc[3] = {b / (T.nbr[2] * T.nbr[1]), (b / T.nbr[2]) % T.nbr[1], b % T.nbr[2]};
    brick_candidates(T, T.p, bc, G.brick_cand + (size_t)b * QEQ_BRICK_CAND);
  }
  double Mp[QEQ_MAXP];
  bspline_int_s(T.p, Mp);
  for (int d = 0; d < 3; ++d) {
    const int K = T.K[d];
    for (int h = 0; h < 2; ++h) {
      FftPlanDev& f = G.fft[2 * d + h];
      memset(&f, 0, sizeof(f));
      f.tw_off = (2 * d + h) * kSM;
      f.tab_off = (2 * d + h) * 3 * kSM;
      if (!fft_plan_fill(K, f, G.tw64 + f.tw_off, G.tw32 + f.tw_off, G.tabs + f.tab_off,
                         h ? QEQ_MAXR64 : QEQ_MAXR32))
        return QEQ_ERR_INVALID;
    }
    T.fft_plan[d] = 2 * d;
    T.bmod_off[d] = d * kSM;
    for (int m = 0; m < K; ++m) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k <= T.p - 2; ++k) {
        double ph = 2.0 * kPiS * (double)m * k / K;
        re += Mp[k + 1] * cos(ph);
        im += Mp[k + 1] * sin(ph);
      }
      double den = re * re + im * im;
      double v = den > 1e-30 ? 1.0 / den : 0.0;
      G.bmod[d * kSM + m] = v;
      G.bmod32[d * kSM + m] = (float)v;
    }
  }
  // FFT work lists (transposing passes)
  int nz = 0, ny = 0, nyi = 0, nx = 0;
  const FftGeom geo = fft_geometry(T.K, T.ncm);
  fft_work_lists(
      T, 0, geo.tl, geo.tlx, [&](int4 v) { G.zit[nz++] = v; }, [&](int4 v) { G.yit[ny++] = v; },
      [&](int4 v) { G.yiit[nyi++] = v; }, [&](int4 v) { G.xit[nx++] = v; });
  int64_t pair_cap = 0;
  if (any) {
    double per = (double)n_atoms / V * (4.0 / 3.0) * kPiS * r_cut * r_cut * r_cut;
    pair_cap = (int64_t)n_atoms * (int64_t)ceil(1.5 * per + 16.0);
    if (pair_cap > QEQ_STATIC_MAX_PAIRS) return QEQ_ERR_CAPACITY;
  }
  const int nchunks = (n_atoms + QEQ_CHUNK - 1) / QEQ_CHUNK;
  for (int c = 0; c < nchunks; ++c) {
    Chunk& ch = G.chunks[c];
    ch.s = 0;
    ch.begin = (int64_t)c * QEQ_CHUNK;
    ch.end = std::min<int64_t>(n_atoms, ch.begin + QEQ_CHUNK);
    ch.first = 0;
    ch.count = nchunks;
    ch.last = (c == nchunks - 1);
  }
  for (int a = 0; a < n_atoms; ++a) G.atom_struct[a] = 0;

  // ---- carve the static array
  qeq_plan_s P;
  P.stream = s;
  P.device = dev;
  P.n_struct = 1;
  P.n_atoms = n_atoms;
  P.precision = QEQ_FP64;
  P.max_S = S;
  P.max_p = T.p;
  P.max_ncm = T.ncm;
  P.geo = geo;
  for (int d = 0; d < 3; ++d) P.fft_kmax[d] = T.K[d];
  if (cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QEQ_ERR_CUDA;
  P.total_bins = nbins;
  P.total_bricks = nbricks;
  P.total_mesh = T.Mp * T.ncm;
  P.pair_cap = pair_cap;
  P.n_chunks = nchunks;
  P.max_species = S;
  P.n_zitems = nz;
  P.n_yitems = ny;
  P.n_xitems = nx;
  P.n_yiitems = nyi;
  P.desc.coulomb_k = coulomb_k;
  Carver cv{reinterpret_cast<unsigned char*>(g_scratch_dev[dev]), 0, (size_t)QEQ_STATIC_SCRATCH_BYTES};
  const int N = n_atoms;
  P.d_st = cv.take<StructDev>(1);
  P.d_fft = cv.take<FftPlanDev>(6);
  P.d_tw64 = cv.take<double2>(6 * kSM);
  P.d_tw32 = cv.take<float2>(6 * kSM);
  P.d_fft_tabs = cv.take<int>(6 * 3 * kSM);
  P.d_bmod = cv.take<double>(3 * kSM);
  P.d_bmod32 = cv.take<float>(3 * kSM);
  P.d_zitems = cv.take<int4>(nz);
  P.d_yitems = cv.take<int4>(ny);
  P.d_yiitems = cv.take<int4>(nyi);
  P.d_xitems = cv.take<int4>(nx);
  P.d_bin_struct = cv.take<int>(nbins);
  P.d_brick_struct = cv.take<int>(nbricks);
  P.d_brick_cand = cv.take<int>((size_t)nbricks * QEQ_BRICK_CAND);
  P.d_atom_struct = cv.take<int>(N);
  P.d_chunks = cv.take<Chunk>(nchunks);
  P.d_key = cv.take<int>(N);
  P.d_bin_count = cv.take<int>(nbins + 1);
  P.d_bin_start = cv.take<int>(nbins + 1);
  P.d_bin_fill = cv.take<int>(nbins + 1);
  P.d_perm = cv.take<int>(N);
  P.d_scan_tmp = reinterpret_cast<int*>(cv.take<int64_t>(std::max(N, nbins) / 1024 + 8));
  P.d_base = cv.take<int>(N);
  P.d_wts = cv.take<double>((size_t)N * 3 * QEQ_MAXP);
  P.d_wts32 = cv.take<float>((size_t)N * 3 * QEQ_MAXP);
  P.d_spec = cv.take<int>(N);
  P.d_J = cv.take<double>(N);
  P.d_chi = cv.take<double>(N);
  P.d_dinv = cv.take<double>(N);
  P.d_posc = cv.take<double>((size_t)N * 3);
  P.d_posc32 = cv.take<float4>(N);
  P.d_row = cv.take<int64_t>(N + 1);
  P.d_row_cnt = cv.take<int>(N);
  P.d_col = cv.take<int>(pair_cap);
  P.d_val64 = cv.take<double>(pair_cap);
  P.d_val32 = cv.take<float>(pair_cap);
  P.d_x = cv.take<double>(N);
  P.d_Ap = cv.take<double>(N);
  P.d_mesh = cv.take<double2>((size_t)P.total_mesh);
  P.d_mesh2 = cv.take<double2>((size_t)P.total_mesh);
  P.gather_split = std::max(8, std::min(QEQ_GATHER_SPLIT_MAX, (2368 + nchunks - 1) / nchunks));
  P.d_part = cv.take<double>((size_t)nchunks * QEQ_MAX_SPECIES * 2 + std::max(nbins, nchunks * QEQ_GATHER_SPLIT_MAX) + 64);
  P.d_counter = cv.take<int>(4);
  P.d_sc = cv.take<PcgScalars>(1);
  P.d_err = cv.take<int>(4);
  if (!cv.ok) return QEQ_ERR_CAPACITY;

  // ---- upload tables, clear what must start at zero
#define SCOPY(dst, src, bytes)                                                          \
  do {                                                                                  \
    if ((bytes) > 0 && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) \
      return QEQ_ERR_CUDA;                                                              \
  } while (0)
  SCOPY(P.d_st, &T, sizeof(StructDev));
  SCOPY(P.d_fft, G.fft, sizeof(G.fft));
  SCOPY(P.d_tw64, G.tw64, sizeof(G.tw64));
  SCOPY(P.d_tw32, G.tw32, sizeof(G.tw32));
  SCOPY(P.d_bmod, G.bmod, sizeof(G.bmod));
  SCOPY(P.d_bmod32, G.bmod32, sizeof(G.bmod32));
  SCOPY(P.d_fft_tabs, G.tabs, sizeof(G.tabs));
  SCOPY(P.d_zitems, G.zit, sizeof(int4) * nz);
  SCOPY(P.d_yitems, G.yit, sizeof(int4) * ny);
  SCOPY(P.d_yiitems, G.yiit, sizeof(int4) * nyi);
  SCOPY(P.d_xitems, G.xit, sizeof(int4) * nx);
  SCOPY(P.d_bin_struct, G.bin_struct, sizeof(int) * nbins);
  SCOPY(P.d_brick_struct, G.bin_struct, sizeof(int) * nbricks);
  SCOPY(P.d_brick_cand, G.brick_cand, sizeof(int) * nbricks * QEQ_BRICK_CAND);
  SCOPY(P.d_atom_struct, G.atom_struct, sizeof(int) * N);
  SCOPY(P.d_chunks, G.chunks, sizeof(Chunk) * nchunks);
#undef SCOPY
  if (cudaMemsetAsync(P.d_counter, 0, sizeof(int) * 4, s) != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaMemsetAsync(P.d_err, 0, sizeof(int) * 4, s) != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaMemsetAsync(P.d_sc, 0, sizeof(PcgScalars), s) != cudaSuccess) return QEQ_ERR_CUDA;

  // ---- atoms, matvec (FP64), back to the caller's order
  if (launch_prepare_atoms(&P, d_pos, d_species, nullptr, d_J, pair_cap > 0) != cudaSuccess) return QEQ_ERR_CUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QEQ_ERR_CUDA;
  if (err & ERRBIT_J) return QEQ_ERR_NOT_PD;
  if (err & ERRBIT_PAIRCAP) return QEQ_ERR_CAPACITY;
  if (err) return QEQ_ERR_INVALID;
  const int nb = (N + 255) / 256;
  k_static_sort_in<<<nb, 256, 0, s>>>(P.d_perm, N, d_x, P.d_x);
  if (cudaGetLastError() != cudaSuccess) return QEQ_ERR_CUDA;
  if (launch_matvec(&P, QEQ_FP64, P.d_x, P.d_Ap, d_J ? 1 : 0, 0, 0, nullptr) != cudaSuccess) return QEQ_ERR_CUDA;
  k_static_unsort<<<nb, 256, 0, s>>>(P.d_perm, N, P.d_Ap, d_y);
  if (cudaGetLastError() != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QEQ_ERR_CUDA;
  return QEQ_OK;
}
