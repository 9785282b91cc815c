// Learned warm start for the QEq solve: radial descriptors and a small per-species
// network that predicts starting charges; inference on the tcgen05 tensor cores
// (BF16 operands, FP32 accumulators in tensor memory), training forward and
// backward on warp-level BF16 MMAs (mma.sync m16n8k16, FP32 accumulate) and Adam
// on FP32 master weights.
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
constexpr int TILE = 64;           // atoms per CTA
constexpr int P_W1 = 0, P_B1 = P_W1 + NH * NF, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH,
              P_B3 = P_W3 + NH;
static_assert(P_B3 + 1 <= QEQ_MLP_NPARAM, "parameter block");

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
  __nv_bfloat162 v;
  v.x = *p0;
  v.y = *p1;
  return *reinterpret_cast<uint32_t*>(&v);
}

// c (16x8 FP32 accumulator fragment) += A (16 x K) * B (K x 8), BF16 operands in
// shared memory with A(m, k) = A[m*sam + k*sak] and B(k, n) = B[k*sbk + n*sbn].
// Fragment layout of mma.m16n8k16 (row.col): lane = 4*g + t;
//   A regs: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
//   B regs: (2t..2t+1, g), (2t+8..2t+9, g)
//   C regs: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
__device__ __forceinline__ void mma_16x8(float* c, const __nv_bfloat16* A, int sam, int sak, const __nv_bfloat16* B,
                                         int sbk, int sbn, int K) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + 2 * t;
    uint32_t a0 = pack2(A + g * sam + ka * sak, A + g * sam + (ka + 1) * sak);
    uint32_t a1 = pack2(A + (g + 8) * sam + ka * sak, A + (g + 8) * sam + (ka + 1) * sak);
    uint32_t a2 = pack2(A + g * sam + (ka + 8) * sak, A + g * sam + (ka + 9) * sak);
    uint32_t a3 = pack2(A + (g + 8) * sam + (ka + 8) * sak, A + (g + 8) * sam + (ka + 9) * sak);
    uint32_t b0 = pack2(B + ka * sbk + g * sbn, B + (ka + 1) * sbk + g * sbn);
    uint32_t b1 = pack2(B + (ka + 8) * sbk + g * sbn, B + (ka + 9) * sbk + g * sbn);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
}

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

// ---------------------------------------------------------------- network
// One CTA = 4 warps = 64 atoms (16 per warp).  For every species present in the
// tile the species' weights are staged in shared memory and the tile is run
// through that network; atoms of other species are masked.  TRAIN adds the
// backward pass and writes the tile's gradient to its own partial block.
struct MlpSmem {
  __nv_bfloat16 W1[NH * NF];
  __nv_bfloat16 W2[NH * NH];
  float b1[NH], b2[NH], W3[NH], b3;
  __nv_bfloat16 X[TILE * NF];
  __nv_bfloat16 H1[TILE * NH];
  __nv_bfloat16 H2[TILE * NH];
  __nv_bfloat16 D2[TILE * NH];   // dL/dz2
  __nv_bfloat16 D1[TILE * NH];   // dL/dz1
  float y[TILE];
  float dy[TILE];
  int sp[TILE];
};

template <bool TRAIN>
__global__ void __launch_bounds__(128) k_mlp(const float* __restrict__ feat, const int* __restrict__ species, int64_t n,
                                             int n_species, const float* __restrict__ params,
                                             const float* __restrict__ scale, const float* __restrict__ target,
                                             float inv_batch, float* __restrict__ out, float* __restrict__ gpart,
                                             float* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& M = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int64_t a0 = (int64_t)blockIdx.x * TILE;
  for (int i = tid; i < TILE; i += blockDim.x) {
    int64_t a = a0 + i;
    M.sp[i] = (a < n) ? species[a] : -1;
    M.y[i] = 0.f;
  }
  __syncthreads();
  unsigned present = 0;
  for (int i = 0; i < TILE; ++i)
    if (M.sp[i] >= 0 && M.sp[i] < n_species) present |= 1u << M.sp[i];
  float loss = 0.f;
  float* gp = TRAIN ? gpart + (size_t)blockIdx.x * n_species * QEQ_MLP_NPARAM : nullptr;
  if (TRAIN)
    for (int i = tid; i < n_species * QEQ_MLP_NPARAM; i += blockDim.x) gp[i] = 0.f;
  for (int s = 0; s < n_species; ++s) {
    if (!((present >> s) & 1u)) continue;
    const float* P = params + (size_t)s * QEQ_MLP_NPARAM;
    const float* mean = scale + (size_t)s * 2 * NF;
    const float* inv = mean + NF;
    __syncthreads();
    for (int i = tid; i < NH * NF; i += blockDim.x) M.W1[i] = __float2bfloat16(P[P_W1 + i]);
    for (int i = tid; i < NH * NH; i += blockDim.x) M.W2[i] = __float2bfloat16(P[P_W2 + i]);
    for (int i = tid; i < NH; i += blockDim.x) {
      M.b1[i] = P[P_B1 + i];
      M.b2[i] = P[P_B2 + i];
      M.W3[i] = P[P_W3 + i];
    }
    if (tid == 0) M.b3 = P[P_B3];
    for (int i = tid; i < TILE * NF; i += blockDim.x) {
      int r = i / NF, k = i - r * NF;
      int64_t a = a0 + r;
      float v = (a < n) ? (feat[a * NF + k] - mean[k]) * inv[k] : 0.f;
      M.X[i] = __float2bfloat16(v);
    }
    __syncthreads();
    const int r0 = w * 16;  // this warp's rows
    // layer 1: H1 = tanh(X W1^T + b1)
    for (int nt = 0; nt < NH / 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_16x8(c, M.X + r0 * NF, NF, 1, M.W1 + nt * 8 * NF, 1, NF, NF);
      int col = nt * 8 + 2 * t;
      M.H1[(r0 + g) * NH + col] = __float2bfloat16(tanhf(c[0] + M.b1[col]));
      M.H1[(r0 + g) * NH + col + 1] = __float2bfloat16(tanhf(c[1] + M.b1[col + 1]));
      M.H1[(r0 + g + 8) * NH + col] = __float2bfloat16(tanhf(c[2] + M.b1[col]));
      M.H1[(r0 + g + 8) * NH + col + 1] = __float2bfloat16(tanhf(c[3] + M.b1[col + 1]));
    }
    __syncwarp();
    // layer 2: H2 = tanh(H1 W2^T + b2); output y = H2 . W3 + b3
    float yg = 0.f, yg8 = 0.f;
    for (int nt = 0; nt < NH / 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_16x8(c, M.H1 + r0 * NH, NH, 1, M.W2 + nt * 8 * NH, 1, NH, NH);
      int col = nt * 8 + 2 * t;
      float h00 = tanhf(c[0] + M.b2[col]), h01 = tanhf(c[1] + M.b2[col + 1]);
      float h10 = tanhf(c[2] + M.b2[col]), h11 = tanhf(c[3] + M.b2[col + 1]);
      M.H2[(r0 + g) * NH + col] = __float2bfloat16(h00);
      M.H2[(r0 + g) * NH + col + 1] = __float2bfloat16(h01);
      M.H2[(r0 + g + 8) * NH + col] = __float2bfloat16(h10);
      M.H2[(r0 + g + 8) * NH + col + 1] = __float2bfloat16(h11);
      yg += h00 * M.W3[col] + h01 * M.W3[col + 1];
      yg8 += h10 * M.W3[col] + h11 * M.W3[col + 1];
    }
    yg += __shfl_xor_sync(0xffffffffu, yg, 1);
    yg += __shfl_xor_sync(0xffffffffu, yg, 2);
    yg8 += __shfl_xor_sync(0xffffffffu, yg8, 1);
    yg8 += __shfl_xor_sync(0xffffffffu, yg8, 2);
    if (t == 0) {
      if (M.sp[r0 + g] == s) M.y[r0 + g] = yg + M.b3;
      if (M.sp[r0 + g + 8] == s) M.y[r0 + g + 8] = yg8 + M.b3;
    }
    if (!TRAIN) continue;
    __syncthreads();
    // ---------------- backward (MSE 1/2 mean): dy = (y - target) / batch for atoms of species s
    for (int i = tid; i < TILE; i += blockDim.x) {
      int64_t a = a0 + i;
      float d = 0.f;
      if (a < n && M.sp[i] == s) {
        float e = M.y[i] - target[a];
        d = e * inv_batch;
        loss += 0.5f * e * e * inv_batch;
      }
      M.dy[i] = d;
    }
    __syncthreads();
    // dz2 = dy W3 (1 - h2^2);  grads of W3, b3
    for (int i = tid; i < TILE * NH; i += blockDim.x) {
      int r = i / NH, f = i - r * NH;
      float h = __bfloat162float(M.H2[i]);
      M.D2[i] = __float2bfloat16(M.dy[r] * M.W3[f] * (1.f - h * h));
    }
    for (int f = tid; f < NH; f += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < TILE; ++r) acc += M.dy[r] * __bfloat162float(M.H2[r * NH + f]);
      gp[s * QEQ_MLP_NPARAM + P_W3 + f] += acc;
    }
    if (tid == 0) {
      float acc = 0.f;
      for (int r = 0; r < TILE; ++r) acc += M.dy[r];
      gp[s * QEQ_MLP_NPARAM + P_B3] += acc;
    }
    __syncthreads();
    // dL/dW2 (64 x 64) = D2^T H1 over the tile's 64 atoms: 32 output fragments, 8 per warp
    for (int q = w; q < (NH / 16) * (NH / 8); q += 4) {
      int mt = q / (NH / 8), nt = q - mt * (NH / 8);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      // A(m = out feature, k = atom) = D2[atom][out], B(k = atom, n = in feature) = H1[atom][in]
      mma_16x8(c, M.D2 + mt * 16, 1, NH, M.H1 + nt * 8, NH, 1, TILE);
      int row = mt * 16 + g, col = nt * 8 + 2 * t;
      float* G2 = gp + s * QEQ_MLP_NPARAM + P_W2;
      G2[row * NH + col] += c[0];
      G2[row * NH + col + 1] += c[1];
      G2[(row + 8) * NH + col] += c[2];
      G2[(row + 8) * NH + col + 1] += c[3];
    }
    for (int f = tid; f < NH; f += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < TILE; ++r) acc += __bfloat162float(M.D2[r * NH + f]);
      gp[s * QEQ_MLP_NPARAM + P_B2 + f] += acc;
    }
    // dz1 = (D2 W2) (1 - h1^2), per warp rows
    for (int nt = 0; nt < NH / 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      // A(m = atom, k = out feature) = D2, B(k = out feature, n = in feature) = W2[out][in]
      mma_16x8(c, M.D2 + r0 * NH, NH, 1, M.W2 + nt * 8, NH, 1, NH);
      int col = nt * 8 + 2 * t;
      float h00 = __bfloat162float(M.H1[(r0 + g) * NH + col]), h01 = __bfloat162float(M.H1[(r0 + g) * NH + col + 1]);
      float h10 = __bfloat162float(M.H1[(r0 + g + 8) * NH + col]),
            h11 = __bfloat162float(M.H1[(r0 + g + 8) * NH + col + 1]);
      M.D1[(r0 + g) * NH + col] = __float2bfloat16(c[0] * (1.f - h00 * h00));
      M.D1[(r0 + g) * NH + col + 1] = __float2bfloat16(c[1] * (1.f - h01 * h01));
      M.D1[(r0 + g + 8) * NH + col] = __float2bfloat16(c[2] * (1.f - h10 * h10));
      M.D1[(r0 + g + 8) * NH + col + 1] = __float2bfloat16(c[3] * (1.f - h11 * h11));
    }
    __syncthreads();
    // dL/dW1 (64 x 32) = D1^T X over the tile: 16 output fragments, 4 per warp
    for (int q = w; q < (NH / 16) * (NF / 8); q += 4) {
      int mt = q / (NF / 8), nt = q - mt * (NF / 8);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_16x8(c, M.D1 + mt * 16, 1, NH, M.X + nt * 8, NF, 1, TILE);
      int row = mt * 16 + g, col = nt * 8 + 2 * t;
      float* G1 = gp + s * QEQ_MLP_NPARAM + P_W1;
      G1[row * NF + col] += c[0];
      G1[row * NF + col + 1] += c[1];
      G1[(row + 8) * NF + col] += c[2];
      G1[(row + 8) * NF + col + 1] += c[3];
    }
    for (int f = tid; f < NH; f += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < TILE; ++r) acc += __bfloat162float(M.D1[r * NH + f]);
      gp[s * QEQ_MLP_NPARAM + P_B1 + f] += acc;
    }
  }
  __syncthreads();
  if (out)
    for (int i = tid; i < TILE; i += blockDim.x)
      if (a0 + i < n) out[a0 + i] = M.y[i];
  if (TRAIN) {
    // deterministic per-tile loss: warp sums, then thread 0 in warp order
    __shared__ float wl[4];
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) wl[w] = loss;
    __syncthreads();
    if (tid == 0) lpart[blockIdx.x] = wl[0] + wl[1] + wl[2] + wl[3];
  }
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
    ok = __syncthreads_and(tc_bar_wait(&M.bar, phase)) != 0;  // the same verdict on every thread
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

static size_t mlp_smem() { return sizeof(MlpSmem); }
static size_t mlp_tc_smem() { return sizeof(MlpTcSmem) + 1024; }  // + alignment of the operand tiles

extern "C" qeq_status qeq_mlp_create(int32_t n_species, int64_t max_batch, qeq_mlp* out) {
  if (!out || n_species < 1 || n_species > QEQ_MAX_SPECIES || max_batch < 1) return QEQ_ERR_INVALID;
  *out = nullptr;
  qeq_mlp_s* m = new qeq_mlp_s();
  m->n_species = n_species;
  m->max_batch = max_batch;
  cudaGetDevice(&m->device);
  size_t np = (size_t)n_species * QEQ_MLP_NPARAM;
  int64_t ntiles = (max_batch + TILE - 1) / TILE;
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
  e = e ? e : cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem());
  e = e ? e : cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem());
  e = e ? e : cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_tc_smem());
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
  int ntiles = (int)((n + TILE - 1) / TILE);
  int np = m->n_species * QEQ_MLP_NPARAM;
  k_mlp<true><<<ntiles, 128, mlp_smem(), s>>>(d_feat, d_species, n, m->n_species, m->d_params, m->d_scale, d_target,
                                               1.0f / (float)n, nullptr, m->d_gpart, m->d_lpart);
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
