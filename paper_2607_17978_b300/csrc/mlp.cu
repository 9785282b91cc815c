// Learned warm start for the QEq solve: radial descriptors and a small per-species
// network that predicts starting charges; inference and the training step's forward
// and backward products on the tcgen05 tensor cores (BF16 operands in shared memory,
// FP32 accumulators in tensor memory), Adam on FP32 master weights.
//
// Descriptors (Sec. 2.2 eq. g2 radial functions with the cosine cutoff of SI
// "Cutoff Functions"; element-embracing prefactor of SI "Element-Embracing
// ACSFs" with H_ij = chi_j): for atom i, neighbours j within R_C = 6 A,
//   G_mu       = sum_j exp(-eta (r_ij - R_mu)^2) f_c(r_ij)          mu = 0..11
//   G_{12+mu}  = sum_j chi_j exp(-eta (r_ij - R_mu)^2) f_c(r_ij)
//   G_24..26   = chi_i, J_i, sigma_i ;  G_27..31 = 0
// with R_mu = 0.5 + 0.5 mu A, eta = 2 A^-2, f_c(r) = (cos(pi r / R_C) + 1) / 2.
// Scaling (SI "Feature Scaling"): (G - mean) * inv_range per species.
// Network (SI "Feed-Forward Neural Networks"): 32 -> 64 -> 64 -> 1 per species,
// tanh hidden layers, linear output.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "neighbors.cuh"
#include "qeq_internal.cuh"

namespace {

constexpr int NF = QEQ_MLP_NFEAT;  // 32
constexpr int NH = QEQ_MLP_NHIDDEN;  // 64
constexpr int P_W1 = 0, P_B1 = P_W1 + NH * NF, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH,
              P_B3 = P_W3 + NH;
static_assert(P_B3 + 1 <= QEQ_MLP_NPARAM, "parameter block");

// ---------------------------------------------------------------- descriptors
// One warp per atom: the lanes take the candidate neighbours of the walk, each
// accumulates its share of the 24 radial sums, and a fixed shuffle tree adds the
// lanes' shares (deterministic).
template <bool SORTED>
__global__ void __launch_bounds__(256) k_features(const StructDev* __restrict__ st,
                                                  const int* __restrict__ sorted_struct,
                                                  const int* __restrict__ bin_start, const int* __restrict__ base,
                                                  const int* __restrict__ spec, const float4* __restrict__ posc32,
                                                  const double* __restrict__ chis, const double* __restrict__ Js,
                                                  const int* __restrict__ perm, int64_t n, float* __restrict__ feat) {
  __shared__ NbrWarpSmem ws[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a = (int64_t)blockIdx.x * 8 + w;
  if (a >= n) return;  // whole warp
  const StructDev& S = st[sorted_struct[a]];
  const float RC = QEQ_MLP_RCUT, ETA = 2.0f;
  float G[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) G[k] = 0.f;
  const int bs = base[a];
  const int bb[3] = {(bs & 1023) / QEQ_BIN, ((bs >> 10) & 1023) / QEQ_BIN, ((bs >> 20) & 1023) / QEQ_BIN};
  // FP32 distances: the descriptors are FP32 and vanish smoothly at the cutoff
  const float4 pa = posc32[a];
  const float rc2 = RC * RC;
  warp_neighbour_walk(S, bb, S.feat_range, bin_start, ws[w],
                      [&](bool valid, int t, const double*, const float* sh, bool zero, int) {
    if (!valid || (zero && t == a)) return;
    const float4 pt = posc32[t];
    const float dx = pt.x + sh[0] - pa.x, dy = pt.y + sh[1] - pa.y, dz = pt.z + sh[2] - pa.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2) return;
    const float r = sqrtf(r2);
    const float fc = 0.5f * (cospif(r / RC) + 1.0f);
    const float cj = (float)chis[t];
#pragma unroll
    for (int mu = 0; mu < 12; ++mu) {
      const float dr = r - (0.5f + 0.5f * mu);
      const float g = __expf(-ETA * dr * dr) * fc;
      G[mu] += g;
      G[12 + mu] += cj * g;
    }
  });
#pragma unroll
  for (int k = 0; k < 24; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) G[k] += __shfl_xor_sync(0xffffffffu, G[k], o);
  const int64_t o = SORTED ? a : perm[a];
  float* f = feat + o * NF;
  float v = 0.f;
#pragma unroll
  for (int k = 0; k < 24; ++k)
    if (lane == k) v = G[k];
  if (lane == 24) v = (float)chis[a];
  if (lane == 25) v = (float)Js[a];
  if (lane == 26) v = (float)S.sigma_s[spec[a]];
  if (lane < NF) f[lane] = v;
}

// ---------------------------------------------------------------- network forward on tcgen05
// Inference: one CTA = 4 warps = 128 atoms.  Both layers are M = 128 (atoms) x N = 64
// (neurons) products on the fifth-generation tensor cores: BF16 operands staged in
// shared memory in the canonical K-major layout without swizzle (8 x 16-byte core
// matrices, 128 bytes each: row r, column k of an operand with Kt columns at element
// ((r / 8) (Kt / 8) + k / 8) 64 + (r % 8) 8 + k % 8; neighbours along K 128 bytes apart,
// along M or N Kt 16 bytes apart), FP32 accumulators in tensor memory (lane = atom,
// column = neuron; layer 1 in columns 0-63, layer 2 in 64-127), one elected thread
// issuing the MMAs, a commit to an mbarrier signalling their completion, and each warp
// reading its 32 atoms' rows back with tcgen05.ld.  Every thread then owns one atom's
// row: bias and tanh, the next layer's operand, and the output dot product stay in
// registers.  For every species present in the tile its weights are staged and the
// tile is run through that network; atoms of other species keep their earlier result.
constexpr int TC_TILE = 128;
struct MlpTcSmem {
  alignas(128) __nv_bfloat16 X[TC_TILE * NF];    // A of layer 1 (K = NF)
  alignas(128) __nv_bfloat16 H1[TC_TILE * NH];   // A of layer 2 (K = NH)
  alignas(128) __nv_bfloat16 W1[NH * NF];        // B of layer 1: W1[n][k], K-major
  alignas(128) __nv_bfloat16 W2[NH * NH];        // B of layer 2
  float b1[NH], b2[NH], W3[NH], b3;
  int sp[TC_TILE];
  alignas(8) uint64_t bar;
  uint32_t tmem;
};

__device__ __forceinline__ int kmaj_off(int r, int k, int Kt) {
  return ((r >> 3) * (Kt >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
// shared-memory matrix descriptor of a K-major operand without swizzle (start, leading =
// K-neighbour core matrix, stride = M/N-neighbour core matrix, all in 16-byte units;
// descriptor version 1)
__device__ __forceinline__ uint64_t kmaj_desc(const void* p, int Kt) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  const uint64_t lbo = 128 >> 4, sbo = (uint64_t)(Kt * 16) >> 4;
  return (uint64_t)((a >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 accumulator, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(bar))
               : "memory");
}
__device__ __forceinline__ bool tc_bar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (0.5 s of the global timer) for the MMAs behind a commit
__device__ __forceinline__ bool tc_bar_wait(uint64_t* bar, uint32_t parity) {
  if (tc_bar_test(bar, parity)) return true;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (tc_bar_test(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 500000000ull) return false;
  }
}
// this warp's 32 tensor-memory lanes, 64 consecutive columns from column c, into v
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t* u = reinterpret_cast<uint32_t*>(v);
#define QEQ_R8(i) "=r"(u[i]), "=r"(u[i + 1]), "=r"(u[i + 2]), "=r"(u[i + 3]), "=r"(u[i + 4]), "=r"(u[i + 5]), \
                  "=r"(u[i + 6]), "=r"(u[i + 7])
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, "
      "%36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, "
      "%57, %58, %59, %60, %61, %62, %63}, [%64];"
      : QEQ_R8(0), QEQ_R8(8), QEQ_R8(16), QEQ_R8(24), QEQ_R8(32), QEQ_R8(40), QEQ_R8(48), QEQ_R8(56)
      : "r"(taddr));
#undef QEQ_R8
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128) k_mlp_fwd_tc(const float* __restrict__ feat, const int* __restrict__ species,
                                                    int64_t n, int n_species, const float* __restrict__ params,
                                                    const float* __restrict__ scale, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // operand tiles on a 1024-byte boundary of the shared window (1024 bytes reserved for it)
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
  MlpTcSmem& M = *reinterpret_cast<MlpTcSmem*>(smem_raw + (((base + 1023u) & ~1023u) - base));
  const int tid = threadIdx.x, w = tid >> 5;
  const int64_t a0 = (int64_t)blockIdx.x * TC_TILE, a = a0 + tid;
  M.sp[tid] = (a < n) ? species[a] : -1;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&M.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {  // 128 tensor-memory columns: layer 1 in 0-63, layer 2 in 64-127
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&M.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = M.tmem;
  const uint32_t lane_base = (uint32_t)(w * 32) << 16;
  unsigned present = 0;
  for (int i = 0; i < TC_TILE; ++i)
    if (M.sp[i] >= 0 && M.sp[i] < n_species) present |= 1u << M.sp[i];
  const int my_sp = M.sp[tid];
  float y = 0.f;
  uint32_t phase = 0;
  bool ok = true;
  for (int s = 0; s < n_species && ok; ++s) {
    if (!((present >> s) & 1u)) continue;
    const float* P = params + (size_t)s * QEQ_MLP_NPARAM;
    const float* mean = scale + (size_t)s * 2 * NF;
    const float* inv = mean + NF;
    // weights in the K-major layout (W[n][k]: neuron n, input k)
    for (int i = tid; i < NH * NF; i += blockDim.x) {
      const int nn = i / NF, k = i - nn * NF;
      M.W1[kmaj_off(nn, k, NF)] = __float2bfloat16(P[P_W1 + i]);
    }
    for (int i = tid; i < NH * NH; i += blockDim.x) {
      const int nn = i / NH, k = i - nn * NH;
      M.W2[kmaj_off(nn, k, NH)] = __float2bfloat16(P[P_W2 + i]);
    }
    for (int i = tid; i < NH; i += blockDim.x) {
      M.b1[i] = P[P_B1 + i];
      M.b2[i] = P[P_B2 + i];
      M.W3[i] = P[P_W3 + i];
    }
    if (tid == 0) M.b3 = P[P_B3];
    // this thread's atom: its scaled features as row tid of X
    {
      __align__(16) __nv_bfloat16 xr[NF];
#pragma unroll
      for (int k = 0; k < NF; ++k) xr[k] = __float2bfloat16((a < n) ? (feat[a * NF + k] - mean[k]) * inv[k] : 0.f);
#pragma unroll
      for (int kg = 0; kg < NF / 8; ++kg)
        *reinterpret_cast<uint4*>(&M.X[kmaj_off(tid, kg * 8, NF)]) = *reinterpret_cast<const uint4*>(&xr[kg * 8]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the operands, to the tensor cores
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 1: H1 = X W1^T (K = 32: two K = 16 steps of two core matrices)
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < NF / 16; ++j)
        tc_mma(tmem, kmaj_desc(&M.X[j * 16 * 8], NF), kmaj_desc(&M.W1[j * 16 * 8], NF), tc_idesc(TC_TILE, NH), j);
      tc_commit(&M.bar);
    }
    ok = __syncthreads_and(tc_bar_wait(&M.bar, phase)) != 0;  // the same outcome on every thread
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float v[NH];
    tc_ld64(tmem + lane_base, v);
    {
      __align__(16) __nv_bfloat16 hr[NH];
#pragma unroll
      for (int k = 0; k < NH; ++k) hr[k] = __float2bfloat16(tanhf(v[k] + M.b1[k]));
#pragma unroll
      for (int kg = 0; kg < NH / 8; ++kg)
        *reinterpret_cast<uint4*>(&M.H1[kmaj_off(tid, kg * 8, NH)]) = *reinterpret_cast<const uint4*>(&hr[kg * 8]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 2: H2 = tanh(H1 W2^T + b2) (K = 64: four steps), y = H2 . W3 + b3
    if (tid == 0 && ok) {
#pragma unroll
      for (int j = 0; j < NH / 16; ++j)
        tc_mma(tmem + NH, kmaj_desc(&M.H1[j * 16 * 8], NH), kmaj_desc(&M.W2[j * 16 * 8], NH), tc_idesc(TC_TILE, NH),
               j);
      tc_commit(&M.bar);
    }
    ok = __syncthreads_and(ok && tc_bar_wait(&M.bar, phase)) != 0;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc_ld64(tmem + lane_base + NH, v);
    float ys = M.b3;
#pragma unroll
    for (int k = 0; k < NH; ++k) ys += tanhf(v[k] + M.b2[k]) * M.W3[k];
    if (my_sp == s) y = ys;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the staged operands and tensor memory are reused by the next species
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (a < n) out[a] = ok ? y : __int_as_float(0x7fc00000);  // a timed-out MMA wait: NaN (rejected start)
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// this warp's 32 tensor-memory lanes, 32 consecutive columns from column c, into v
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t* u = reinterpret_cast<uint32_t*>(v);
#define QEQ_R8(i) "=r"(u[i]), "=r"(u[i + 1]), "=r"(u[i + 2]), "=r"(u[i + 3]), "=r"(u[i + 4]), "=r"(u[i + 5]), \
                  "=r"(u[i + 6]), "=r"(u[i + 7])
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : QEQ_R8(0), QEQ_R8(8), QEQ_R8(16), QEQ_R8(24)
      : "r"(taddr));
#undef QEQ_R8
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- network training step on tcgen05
// One CTA = 4 warps = 128 atoms, the loss 1/(2n) sum (y - t)^2 and its gradient for every
// species present in the tile, written to the tile's own partial block.  All five products
// run on the tensor cores with both operands K-major (the transposed operands are written
// transposed into shared memory): forward H1 = X W1^T, H2 = H1 W2^T (M = atoms); backward
// dW2 = D2^T H1 and dW1 = D1^T X (M = output neurons padded to 128 with zero rows, K =
// atoms), dZ1 = D2 W2 (M = atoms).  Tensor memory: columns 0-63 layer 1 (later dW1),
// 64-127 layer 2, 128-191 dW2, 192-255 dZ1.  Bias and output-layer gradients are column
// sums over the tile's atoms in a fixed order.
struct MlpTrainSmem {
  alignas(128) __nv_bfloat16 X[TC_TILE * NF];    // [atom][k]        A of layer 1
  alignas(128) __nv_bfloat16 XT[NF * TC_TILE];   // [k][atom]        B of dW1
  alignas(128) __nv_bfloat16 H1[TC_TILE * NH];   // [atom][f]        A of layer 2
  alignas(128) __nv_bfloat16 H1T[NH * TC_TILE];  // [f][atom]        B of dW2
  alignas(128) __nv_bfloat16 D2[TC_TILE * NH];   // [atom][f]        A of dZ1
  alignas(128) __nv_bfloat16 DT[128 * TC_TILE];  // [f][atom], rows >= NH zero: A of dW2, then of dW1
  alignas(128) __nv_bfloat16 W1[NH * NF];        // [n][k]           B of layer 1
  alignas(128) __nv_bfloat16 W2[NH * NH];        // [n][k]           B of layer 2
  alignas(128) __nv_bfloat16 W2T[NH * NH];       // [k][n]           B of dZ1
  float red[TC_TILE][NH + 1];                    // per-atom values of column sums
  float dyv[TC_TILE];
  float b1[NH], b2[NH], W3[NH], b3;
  int sp[TC_TILE];
  float lw[4];
  alignas(8) uint64_t bar;
  uint32_t tmem;
};

__global__ void __launch_bounds__(128) k_mlp_train_tc(const float* __restrict__ feat,
                                                      const int* __restrict__ species, int64_t n, int n_species,
                                                      const float* __restrict__ params,
                                                      const float* __restrict__ scale,
                                                      const float* __restrict__ target, float inv_batch,
                                                      float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
  MlpTrainSmem& M = *reinterpret_cast<MlpTrainSmem*>(smem_raw + (((base + 1023u) & ~1023u) - base));
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t a0 = (int64_t)blockIdx.x * TC_TILE, a = a0 + tid;
  M.sp[tid] = (a < n) ? species[a] : -1;
  for (int i = tid; i < (128 - NH) * TC_TILE; i += blockDim.x) M.DT[NH * TC_TILE + i] = __float2bfloat16(0.f);
  float* gp = gpart + (size_t)blockIdx.x * n_species * QEQ_MLP_NPARAM;
  for (int i = tid; i < n_species * QEQ_MLP_NPARAM; i += blockDim.x) gp[i] = 0.f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&M.bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&M.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = M.tmem, lane_base = (uint32_t)(w * 32) << 16;
  unsigned present = 0;
  for (int i = 0; i < TC_TILE; ++i)
    if (M.sp[i] >= 0 && M.sp[i] < n_species) present |= 1u << M.sp[i];
  const int my_sp = M.sp[tid];
  float loss = 0.f;
  uint32_t phase = 0;
  bool ok = true;
  // all threads: operands written by threads -> tensor cores; tcgen05 ops ordered by the barrier
  auto sync_operands = [&]() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  };
  auto wait_mma = [&]() {  // the commit issued by thread 0 (CTA-uniform outcome)
    ok = __syncthreads_and(ok && tc_bar_wait(&M.bar, phase)) != 0;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  };
  for (int s = 0; s < n_species && ok; ++s) {
    if (!((present >> s) & 1u)) continue;
    const float* P = params + (size_t)s * QEQ_MLP_NPARAM;
    float* G = gp + (size_t)s * QEQ_MLP_NPARAM;
    const float* mean = scale + (size_t)s * 2 * NF;
    const float* inv = mean + NF;
    for (int i = tid; i < NH * NF; i += blockDim.x) {
      const int nn = i / NF, k = i - nn * NF;
      M.W1[kmaj_off(nn, k, NF)] = __float2bfloat16(P[P_W1 + i]);
    }
    for (int i = tid; i < NH * NH; i += blockDim.x) {
      const int nn = i / NH, k = i - nn * NH;
      const __nv_bfloat16 v = __float2bfloat16(P[P_W2 + i]);
      M.W2[kmaj_off(nn, k, NH)] = v;
      M.W2T[kmaj_off(k, nn, NH)] = v;
    }
    for (int i = tid; i < NH; i += blockDim.x) {
      M.b1[i] = P[P_B1 + i];
      M.b2[i] = P[P_B2 + i];
      M.W3[i] = P[P_W3 + i];
    }
    if (tid == 0) M.b3 = P[P_B3];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const __nv_bfloat16 v = __float2bfloat16((a < n) ? (feat[a * NF + k] - mean[k]) * inv[k] : 0.f);
      M.X[kmaj_off(tid, k, NF)] = v;
      M.XT[kmaj_off(k, tid, TC_TILE)] = v;
    }
    sync_operands();
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < NF / 16; ++j)
        tc_mma(tmem, kmaj_desc(&M.X[j * 128], NF), kmaj_desc(&M.W1[j * 128], NF), tc_idesc(TC_TILE, NH), j);
      tc_commit(&M.bar);
    }
    wait_mma();
    float v[NH];
    tc_ld64(tmem + lane_base, v);
#pragma unroll
    for (int f = 0; f < NH; ++f) {
      const __nv_bfloat16 h = __float2bfloat16(tanhf(v[f] + M.b1[f]));
      M.H1[kmaj_off(tid, f, NH)] = h;
      M.H1T[kmaj_off(f, tid, TC_TILE)] = h;
    }
    sync_operands();
    if (tid == 0 && ok) {
#pragma unroll
      for (int j = 0; j < NH / 16; ++j)
        tc_mma(tmem + 64, kmaj_desc(&M.H1[j * 128], NH), kmaj_desc(&M.W2[j * 128], NH), tc_idesc(TC_TILE, NH), j);
      tc_commit(&M.bar);
    }
    wait_mma();
    tc_ld64(tmem + lane_base + 64, v);
    float y = M.b3;
#pragma unroll
    for (int f = 0; f < NH; ++f) {
      v[f] = tanhf(v[f] + M.b2[f]);  // h2
      y += v[f] * M.W3[f];
    }
    float dy = 0.f;
    if (a < n && my_sp == s) {
      const float e = y - target[a];
      dy = e * inv_batch;
      loss += 0.5f * e * e * inv_batch;
    }
    M.dyv[tid] = dy;
    // dZ2 = dy W3 (1 - h2^2): rows of D2, columns of DT; dy h2 for dW3
#pragma unroll
    for (int f = 0; f < NH; ++f) {
      M.red[tid][f] = dy * v[f];
      const __nv_bfloat16 d = __float2bfloat16(dy * M.W3[f] * (1.f - v[f] * v[f]));
      M.D2[kmaj_off(tid, f, NH)] = d;
      M.DT[kmaj_off(f, tid, TC_TILE)] = d;
    }
    sync_operands();
    if (tid == 0 && ok) {
      // dW2 (rows 0-63 of a 128-row product) and dZ1 = D2 W2, one commit
#pragma unroll
      for (int j = 0; j < TC_TILE / 16; ++j)
        tc_mma(tmem + 128, kmaj_desc(&M.DT[j * 128], TC_TILE), kmaj_desc(&M.H1T[j * 128], TC_TILE),
               tc_idesc(128, NH), j);
#pragma unroll
      for (int j = 0; j < NH / 16; ++j)
        tc_mma(tmem + 192, kmaj_desc(&M.D2[j * 128], NH), kmaj_desc(&M.W2T[j * 128], NH), tc_idesc(TC_TILE, NH), j);
      tc_commit(&M.bar);
    }
    if (tid < NH) {  // dW3, fixed order over the tile's atoms
      float acc = 0.f;
      for (int r = 0; r < TC_TILE; ++r) acc += M.red[r][tid];
      G[P_W3 + tid] = acc;
    } else if (tid == NH) {
      float acc = 0.f;
      for (int r = 0; r < TC_TILE; ++r) acc += M.dyv[r];
      G[P_B3] = acc;
    }
    __syncthreads();  // red is rewritten below
#pragma unroll
    for (int f = 0; f < NH; ++f) M.red[tid][f] = __bfloat162float(M.D2[kmaj_off(tid, f, NH)]);
    __syncthreads();
    if (tid < NH) {  // db2
      float acc = 0.f;
      for (int r = 0; r < TC_TILE; ++r) acc += M.red[r][tid];
      G[P_B2 + tid] = acc;
    }
    wait_mma();
    // dZ1 (1 - h1^2) -> D1, transposed into DT (dW2 has been read by the MMA)
    tc_ld64(tmem + lane_base + 192, v);
    __syncthreads();  // db2 has read red
#pragma unroll
    for (int f = 0; f < NH; ++f) {
      const float h = __bfloat162float(M.H1[kmaj_off(tid, f, NH)]);
      const __nv_bfloat16 d = __float2bfloat16(v[f] * (1.f - h * h));
      M.DT[kmaj_off(f, tid, TC_TILE)] = d;
      M.red[tid][f] = __bfloat162float(d);
    }
    if (w < 2) {  // dW2: rows 0-63 live in the lanes of warps 0 and 1
      tc_ld64(tmem + lane_base + 128, v);
#pragma unroll
      for (int f = 0; f < NH; ++f) G[P_W2 + tid * NH + f] = v[f];
    }
    sync_operands();
    if (tid == 0 && ok) {
#pragma unroll
      for (int j = 0; j < TC_TILE / 16; ++j)
        tc_mma(tmem, kmaj_desc(&M.DT[j * 128], TC_TILE), kmaj_desc(&M.XT[j * 128], TC_TILE), tc_idesc(128, NF), j);
      tc_commit(&M.bar);
    }
    if (tid < NH) {  // db1
      float acc = 0.f;
      for (int r = 0; r < TC_TILE; ++r) acc += M.red[r][tid];
      G[P_B1 + tid] = acc;
    }
    wait_mma();
    if (w < 2) {
      float u[NF];
      tc_ld32(tmem + lane_base, u);
#pragma unroll
      for (int k = 0; k < NF; ++k) G[P_W1 + tid * NF + k] = u[k];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // operands, red and tensor memory are reused by the next species
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // deterministic per-tile loss: warp sums, then the warps in order
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0) M.lw[w] = loss;
  __syncthreads();
  if (tid == 0) lpart[blockIdx.x] = ok ? (M.lw[0] + M.lw[1] + M.lw[2] + M.lw[3]) : __int_as_float(0x7fc00000);
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// sum of the per-tile gradient blocks in tile order, then Adam on the FP32 master weights
__global__ void k_adam(const float* __restrict__ gpart, int ntiles, int nparam, float* __restrict__ params,
                       float* __restrict__ m, float* __restrict__ v, float* __restrict__ grad_out, float lr,
                       float beta1, float beta2, float eps, float bc1, float bc2, int apply) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nparam) return;
  float gsum = 0.f;
  for (int k = 0; k < ntiles; ++k) gsum += gpart[(size_t)k * nparam + i];
  if (grad_out) grad_out[i] = gsum;
  if (!apply) return;
  float mi = beta1 * m[i] + (1.f - beta1) * gsum;
  float vi = beta2 * v[i] + (1.f - beta2) * gsum * gsum;
  m[i] = mi;
  v[i] = vi;
  params[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_sum_tiles(const float* __restrict__ lpart, int ntiles, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float s = 0.f;
  for (int k = 0; k < ntiles; ++k) s += lpart[k];
  *loss = s;
}

// warm start: prediction (sorted order) -> FP64 starting charges
__global__ void k_pred_to_q(const float* __restrict__ pred, int64_t n, double* __restrict__ q) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) q[a] = (double)pred[a];
}

}  // namespace

// ---------------------------------------------------------------- host side
struct qeq_mlp_s {
  int n_species = 0;
  int64_t max_batch = 0;
  int device = 0;
  float* d_params = nullptr;  // FP32 master weights, n_species * QEQ_MLP_NPARAM
  float* d_scale = nullptr;   // n_species * 2 * NF: mean, inv_range
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_gpart = nullptr;   // per-tile gradient blocks
  float* d_lpart = nullptr;
  float* d_loss = nullptr;
  float* h_loss = nullptr;
  int64_t step = 0;
  std::string err;
};

static size_t mlp_tc_smem() { return sizeof(MlpTcSmem) + 1024; }  // + alignment of the operand tiles
static size_t mlp_train_smem() { return sizeof(MlpTrainSmem) + 1024; }

extern "C" qeq_status qeq_mlp_create(int32_t n_species, int64_t max_batch, qeq_mlp* out) {
  if (!out || n_species < 1 || n_species > QEQ_MAX_SPECIES || max_batch < 1) return QEQ_ERR_INVALID;
  *out = nullptr;
  qeq_mlp_s* m = new qeq_mlp_s();
  m->n_species = n_species;
  m->max_batch = max_batch;
  cudaGetDevice(&m->device);
  size_t np = (size_t)n_species * QEQ_MLP_NPARAM;
  int64_t ntiles = (max_batch + TC_TILE - 1) / TC_TILE;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&m->d_params, np * sizeof(float));
  e = e ? e : cudaMalloc(&m->d_scale, (size_t)n_species * 2 * NF * sizeof(float));
  e = e ? e : cudaMalloc(&m->d_m, np * sizeof(float));
  e = e ? e : cudaMalloc(&m->d_v, np * sizeof(float));
  e = e ? e : cudaMalloc(&m->d_gpart, (size_t)ntiles * np * sizeof(float));
  e = e ? e : cudaMalloc(&m->d_lpart, (size_t)ntiles * sizeof(float));
  e = e ? e : cudaMalloc(&m->d_loss, sizeof(float));
  e = e ? e : cudaHostAlloc(&m->h_loss, sizeof(float), cudaHostAllocDefault);
  e = e ? e : cudaMemset(m->d_params, 0, np * sizeof(float));
  e = e ? e : cudaMemset(m->d_m, 0, np * sizeof(float));
  e = e ? e : cudaMemset(m->d_v, 0, np * sizeof(float));
  e = e ? e : cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_tc_smem());
  e = e ? e : cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)mlp_train_smem());
  if (e != cudaSuccess) {
    qeq_mlp_destroy(m);
    return e == cudaErrorMemoryAllocation ? QEQ_ERR_OOM : QEQ_ERR_CUDA;
  }
  // identity scaling until set
  std::vector<float> sc((size_t)n_species * 2 * NF);
  for (int s = 0; s < n_species; ++s)
    for (int k = 0; k < NF; ++k) {
      sc[(size_t)s * 2 * NF + k] = 0.f;
      sc[(size_t)s * 2 * NF + NF + k] = 1.f;
    }
  cudaMemcpy(m->d_scale, sc.data(), sc.size() * sizeof(float), cudaMemcpyHostToDevice);
  *out = m;
  return QEQ_OK;
}

extern "C" void qeq_mlp_destroy(qeq_mlp m) {
  if (!m) return;
  for (void* p : {(void*)m->d_params, (void*)m->d_scale, (void*)m->d_m, (void*)m->d_v, (void*)m->d_gpart,
                  (void*)m->d_lpart, (void*)m->d_loss})
    if (p) cudaFree(p);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  delete m;
}

extern "C" qeq_status qeq_mlp_set_params(qeq_mlp m, const float* h_params, const float* h_scale) {
  if (!m) return QEQ_ERR_INVALID;
  size_t np = (size_t)m->n_species * QEQ_MLP_NPARAM;
  if (h_params && cudaMemcpy(m->d_params, h_params, np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return QEQ_ERR_CUDA;
  if (h_scale &&
      cudaMemcpy(m->d_scale, h_scale, (size_t)m->n_species * 2 * NF * sizeof(float), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return QEQ_ERR_CUDA;
  if (h_params) {
    cudaMemset(m->d_m, 0, np * sizeof(float));
    cudaMemset(m->d_v, 0, np * sizeof(float));
    m->step = 0;
  }
  return QEQ_OK;
}

extern "C" qeq_status qeq_mlp_get_params(qeq_mlp m, float* h_params, float* h_scale, float* h_adam_m,
                                         float* h_adam_v, int64_t* h_step) {
  if (!m) return QEQ_ERR_INVALID;
  size_t np = (size_t)m->n_species * QEQ_MLP_NPARAM;
  if (h_params && cudaMemcpy(h_params, m->d_params, np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return QEQ_ERR_CUDA;
  if (h_scale && cudaMemcpy(h_scale, m->d_scale, (size_t)m->n_species * 2 * NF * sizeof(float),
                            cudaMemcpyDeviceToHost) != cudaSuccess)
    return QEQ_ERR_CUDA;
  if (h_adam_m && cudaMemcpy(h_adam_m, m->d_m, np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return QEQ_ERR_CUDA;
  if (h_adam_v && cudaMemcpy(h_adam_v, m->d_v, np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return QEQ_ERR_CUDA;
  if (h_step) *h_step = m->step;
  return QEQ_OK;
}

extern "C" qeq_status qeq_mlp_set_adam_state(qeq_mlp m, const float* h_adam_m, const float* h_adam_v, int64_t step) {
  if (!m || !h_adam_m || !h_adam_v || step < 0) return QEQ_ERR_INVALID;
  size_t np = (size_t)m->n_species * QEQ_MLP_NPARAM;
  if (cudaMemcpy(m->d_m, h_adam_m, np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaMemcpy(m->d_v, h_adam_v, np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return QEQ_ERR_CUDA;
  m->step = step;
  return QEQ_OK;
}

extern "C" qeq_status qeq_mlp_forward(qeq_mlp m, const float* d_feat, const int32_t* d_species, int64_t n,
                                      float* d_out, void* cuda_stream) {
  if (!m || !d_feat || !d_species || !d_out || n < 0) return QEQ_ERR_INVALID;
  if (n == 0) return QEQ_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int ntiles = (int)((n + TC_TILE - 1) / TC_TILE);
  k_mlp_fwd_tc<<<ntiles, 128, mlp_tc_smem(), s>>>(d_feat, d_species, n, m->n_species, m->d_params, m->d_scale,
                                                  d_out);
  if (cudaGetLastError() != cudaSuccess) return QEQ_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? QEQ_OK : QEQ_ERR_CUDA;
}

extern "C" qeq_status qeq_mlp_train_step(qeq_mlp m, const float* d_feat, const int32_t* d_species,
                                         const float* d_target, int64_t n, float lr, int32_t apply_update,
                                         float* d_grad_out, float* h_loss, void* cuda_stream) {
  if (!m || !d_feat || !d_species || !d_target || n < 1) return QEQ_ERR_INVALID;
  if (n > m->max_batch) return QEQ_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int ntiles = (int)((n + TC_TILE - 1) / TC_TILE);
  int np = m->n_species * QEQ_MLP_NPARAM;
  k_mlp_train_tc<<<ntiles, 128, mlp_train_smem(), s>>>(d_feat, d_species, n, m->n_species, m->d_params, m->d_scale,
                                                       d_target, 1.0f / (float)n, m->d_gpart, m->d_lpart);
  if (apply_update) m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float bc1 = 1.f - powf(b1, (float)std::max<int64_t>(m->step, 1));
  float bc2 = 1.f - powf(b2, (float)std::max<int64_t>(m->step, 1));
  k_adam<<<(np + 255) / 256, 256, 0, s>>>(m->d_gpart, ntiles, np, m->d_params, m->d_m, m->d_v, d_grad_out, lr, b1, b2,
                                          1e-8f, bc1, bc2, apply_update);
  k_sum_tiles<<<1, 32, 0, s>>>(m->d_lpart, ntiles, m->d_loss);
  if (cudaGetLastError() != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaMemcpyAsync(m->h_loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QEQ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QEQ_ERR_CUDA;
  if (h_loss) *h_loss = *m->h_loss;
  return QEQ_OK;
}

// descriptors of every atom of a plan, in the caller's atom order
extern "C" qeq_status qeq_features(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_chi,
                                   const double* d_J, float* d_feat) {
  if (!P || !d_pos || !d_species || !d_chi || !d_J || !d_feat) return QEQ_ERR_INVALID;
  if (cudaSetDevice(P->device) != cudaSuccess) return QEQ_ERR_CUDA;
  if (launch_prepare_atoms(P, d_pos, d_species, d_chi, d_J, 0) != cudaSuccess) return QEQ_ERR_CUDA;
  int nb = (int)((P->n_atoms + 7) / 8);  // one warp per atom
  count_launch(P);
  k_features<false><<<nb, 256, 0, P->stream>>>(P->d_st, P->d_key, P->d_bin_start, P->d_base, P->d_spec, P->d_posc32,
                                                P->d_chi, P->d_J, P->d_perm, P->n_atoms, d_feat);
  if (cudaGetLastError() != cudaSuccess) return QEQ_ERR_CUDA;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEQ_ERR_CUDA;
  int err = 0;
  cudaMemcpy(&err, P->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (err) {
    cudaMemset(P->d_err, 0, sizeof(int));
    return (err & ERRBIT_J) ? QEQ_ERR_NOT_PD : QEQ_ERR_INVALID;
  }
  return QEQ_OK;
}

extern "C" qeq_status qeq_plan_set_warm_start(qeq_plan P, qeq_mlp m) {
  if (!P) return QEQ_ERR_INVALID;
  if (m && m->n_species < P->max_S) {
    P->last_error = "network has fewer species than the plan";
    return QEQ_ERR_INVALID;
  }
  P->mlp = m;
  if (m && !P->d_feat) {
    if (cudaMalloc(&P->d_feat, (size_t)P->n_atoms * NF * sizeof(float)) != cudaSuccess) return QEQ_ERR_OOM;
    if (cudaMalloc(&P->d_pred, (size_t)P->n_atoms * sizeof(float)) != cudaSuccess) return QEQ_ERR_OOM;
    P->workspace_bytes += (int64_t)P->n_atoms * (NF + 1) * sizeof(float);
  }
  return QEQ_OK;
}

// warm start inside qeq_solve: descriptors and network on the sorted atoms -> d_q (sorted)
cudaError_t launch_mlp_warm_start(qeq_plan_s* P, double* d_q_sorted) {
  qeq_mlp_s* m = P->mlp;
  cudaStream_t s = P->stream;
  int nb = (int)((P->n_atoms + 7) / 8);  // one warp per atom
  count_launch(P, 3);
  k_features<true><<<nb, 256, 0, s>>>(P->d_st, P->d_key, P->d_bin_start, P->d_base, P->d_spec, P->d_posc32, P->d_chi,
                                       P->d_J, P->d_perm, P->n_atoms, P->d_feat);
  int ntiles = (int)((P->n_atoms + TC_TILE - 1) / TC_TILE);
  k_mlp_fwd_tc<<<ntiles, 128, mlp_tc_smem(), s>>>(P->d_feat, P->d_spec, P->n_atoms, m->n_species, m->d_params,
                                                  m->d_scale, P->d_pred);
  k_pred_to_q<<<(int)((P->n_atoms + 255) / 256), 256, 0, s>>>(P->d_pred, P->n_atoms, d_q_sorted);
  return cudaGetLastError();
}
