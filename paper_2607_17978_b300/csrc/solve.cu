// The QEq solve (Sec. 2.4, bordered system eq. 4G_qeq_prime; SI eq. qeq):
// Jacobi-preconditioned conjugate gradient restricted to the charge-constraint
// plane sum_i q_i = q_tot, around the plane-wave matvec of matvec.cu.
//
//   r = -chi - A q                       (A = E + diag J)
//   z = D^-1 (r - s 1),  s = (1^T D^-1 r)/(1^T D^-1 1)     so that 1^T z = 0
//   p = z + beta p,  alpha = r.z / p.Ap,  q += alpha p,  r -= alpha Ap
//
// Every search direction sums to zero, so q stays on the constraint plane.
// At convergence A q + chi = mu 1 with mu = -mean(r) (the bordered lambda is
// -mu).  All vector arithmetic, dot products, the projection and mu are FP64;
// in QEQ_MIXED the matvec inside the iteration is FP32, and a final FP64
// matvec recomputes the true residual; if that residual misses the tolerance
// the iteration restarts from it (residual replacement, i.e. iterative
// refinement).  Structures of a batch iterate together and drop out as they
// converge; a block of iterations is captured once in a CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "qeq_internal.cuh"

namespace {

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double wmin(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

enum { RED_SUM = 0, RED_MAX = 1, RED_MIN = 2 };

// Block reduction of NV values (op per value), written to part[chunk*8 + k];
// returns true in thread 0 of the last chunk of the structure, which then
// combines the chunk partials in chunk order (deterministic).
template <int NV>
__device__ bool chunk_reduce(double (&v)[NV], const int (&op)[NV], const Chunk& ch, double* part, int* counter,
                             double (&tot)[NV]) {
  __shared__ double red[NV][32];
  __shared__ double red2[256];
  __shared__ bool last;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = op[k] == RED_SUM ? wsum(v[k]) : (op[k] == RED_MAX ? wmax(v[k]) : wmin(v[k]));
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) {
      double x = red[k][0];
      for (int i = 1; i < nw; ++i)
        x = op[k] == RED_SUM ? x + red[k][i] : (op[k] == RED_MAX ? fmax(x, red[k][i]) : fmin(x, red[k][i]));
      part[(size_t)blockIdx.x * 8 + k] = x;
    }
    __threadfence();
    int prev = atomicAdd(counter + ch.s, 1);
    last = (prev == ch.count - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the structure's last chunk combines all its chunk partials in a fixed order
  for (int k = 0; k < NV; ++k) {
    double a = op[k] == RED_SUM ? 0.0 : (op[k] == RED_MAX ? -1e300 : 1e300);
    for (int i = threadIdx.x; i < ch.count; i += blockDim.x) {
      double y = ((volatile double*)part)[(size_t)(ch.first + i) * 8 + k];
      a = op[k] == RED_SUM ? a + y : (op[k] == RED_MAX ? fmax(a, y) : fmin(a, y));
    }
    a = op[k] == RED_SUM ? wsum(a) : (op[k] == RED_MAX ? wmax(a) : wmin(a));
    if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double x = red2[0];
      for (int i = 1; i < nw; ++i)
        x = op[k] == RED_SUM ? x + red2[i] : (op[k] == RED_MAX ? fmax(x, red2[i]) : fmin(x, red2[i]));
      tot[k] = x;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) counter[ch.s] = 0;
  return threadIdx.x == 0;
}

// q0: user charges (permuted to sorted order) or zero; sums for the projection.
// reject (MLP start only, may be NULL): structures whose network start was rejected start cold.
__global__ void k_init(const Chunk* __restrict__ chunks, const int* __restrict__ perm, const double* __restrict__ q_user,
                       int warm, const int* __restrict__ reject, const double* __restrict__ dinv,
                       const double* __restrict__ chi, const double* __restrict__ J, double* __restrict__ q,
                       PcgScalars* __restrict__ sc, double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  double v[6] = {0, 0, 0, 0, 1e300, 0};
  const int op[6] = {RED_SUM, RED_SUM, RED_SUM, RED_SUM, RED_MIN, RED_MAX};
  const bool mlp_kept = warm == QEQ_WARM_MLP && !(reject && reject[ch.s]);
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    double qa = (warm == QEQ_WARM_USER) ? q_user[perm[a]] : (mlp_kept ? q[a] : 0.0);
    if (!isfinite(qa)) qa = 0.0;
    q[a] = qa;
    v[0] += qa;
    v[1] += dinv[a];
    v[2] += chi[a];
    v[3] += chi[a] * chi[a];
    v[4] = fmin(v[4], J[a]);
    v[5] = fmax(v[5], dinv[a]);
  }
  double tot[6];
  if (chunk_reduce<6>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    double n = (double)c.n;
    c.qsum = tot[0];
    c.s0 = tot[1];
    c.chi_p2 = fmax(tot[3] - tot[2] * tot[2] / n, 0.0);
    c.chi_sum = tot[2];
    c.j_min = tot[4];
    c.dinv_max = tot[5];
  }
}

// project q onto the constraint plane: q += (q_tot - sum q)/n
__global__ void k_project(const Chunk* __restrict__ chunks, double* __restrict__ q, const PcgScalars* __restrict__ sc) {
  const Chunk ch = chunks[blockIdx.x];
  const PcgScalars& c = sc[ch.s];
  double d = (c.q_tot - c.qsum) / (double)c.n;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) q[a] += d;
}

// residual statistics -> convergence test (thread 0 of the last chunk).  tot[1], tot[2]
// are sums of r - ref and (r - ref)^2 about a reference ref close to the mean of r (the
// previous shift): r carries mu 1, and sums of r and r^2 themselves would lose the
// projected part, sum (r - mean)^2 = tot[2] - tot[1]^2 / n, to cancellation.
__device__ void residual_test(PcgScalars& c, const double* tot, double ref, int max_iter, int final_check) {
  double n = (double)c.n;
  const double dmean = tot[1] / n;
  c.r_sum = ref * n + tot[1];
  c.r_max = tot[3];
  c.r_min = tot[4];
  double pinf, pl2;
  if (c.unconstrained) {  // plain residual (the shift, and so ref, stay 0)
    c.shift = 0.0;
    pinf = fmax(fabs(c.r_max), fabs(c.r_min));
    pl2 = sqrt(fmax(tot[2] + ref * (2.0 * tot[1] + n * ref), 0.0));
  } else {
    c.shift = tot[0] / c.s0;
    const double mean = ref + dmean;
    pinf = fmax(c.r_max - mean, mean - c.r_min);
    pl2 = sqrt(fmax(tot[2] - tot[1] * dmean, 0.0));
  }
  c.r_l2 = pl2;
  // the iterations stop a margin below the threshold of the final check, so that
  // the drift of the recurrence residual (FP32 matvec) rarely forces a restart
  const double f = final_check ? 1.0 : c.inner;
  // a final check adds the bound on its residual's own error (0 when it is FP64)
  const double sl = final_check ? c.slack : 0.0;
  // FP32 rounds also end once the residual fell by `drop` below that of the round's check:
  // each FP32 product carries ~3e-7 of the mesh potentials' size as noise, so FP32 CG
  // stalls near 1e-6..1e-5 of the starting residual; the next check then restarts on the
  // correction, whose products are accurate relative to its own (small) size
  const double ti = final_check ? f * c.tol_inf : fmax(f * c.tol_inf, c.floor_inf);
  const double tl = final_check ? f * c.tol_l2 : fmax(f * c.tol_l2, c.floor_l2);
  bool ok = pinf + sl <= ti && (c.tol_l2 <= 0.0 || pl2 + sl * sqrt(n) <= tl);
  if (!isfinite(pinf)) ok = false;
  if (final_check) {
    c.converged = ok ? 1 : 0;
    c.floor_inf = c.drop * pinf;
    c.floor_l2 = c.drop * pl2;
  } else {
    if (ok) {
      c.converged = 1;
      c.active = 0;
    } else if (c.iters >= max_iter) {
      c.active = 0;
    }
  }
}

// r = -chi - Aq (true residual) + statistics
__global__ void k_resid(const Chunk* __restrict__ chunks, const double* __restrict__ chi, const double* __restrict__ Aq,
                        const double* __restrict__ dinv, double* __restrict__ r, PcgScalars* __restrict__ sc,
                        int only_flagged, double* part, int* counter, int max_iter) {
  const Chunk ch = chunks[blockIdx.x];
  const double ref = sc[ch.s].shift;
  double v[5] = {0, 0, 0, -1e300, 1e300};
  const int op[5] = {RED_SUM, RED_SUM, RED_SUM, RED_MAX, RED_MIN};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    double ra = -chi[a] - Aq[a];
    r[a] = ra;
    v[0] += dinv[a] * ra;
    v[1] += ra - ref;
    v[2] += (ra - ref) * (ra - ref);
    v[3] = fmax(v[3], ra);
    v[4] = fmin(v[4], ra);
  }
  double tot[5];
  if (chunk_reduce<5>(v, op, ch, part, counter, tot)) {
    sc[ch.s].slack = 0.0;
    residual_test(sc[ch.s], tot, ref, max_iter, 1);
  }
  (void)only_flagged;
}

// Mixed precision after an FP64 check at charges q1 with FP64 residual r1: the
// residual of q is r1 - A (q - q1).  The change d = q - q1 is small (the FP32
// iterations only correct the last FP32-limited digits), so A d in FP32 is
// accurate to far below the tolerance; the check adds the bound
// op_err (max|A d| + max D max|d|) on that error to the residual before
// comparing.  d into x, with max|d| and max D_i.
__global__ void k_delta(const Chunk* __restrict__ chunks, const double* __restrict__ q, const double* __restrict__ q1,
                        const double* __restrict__ dinv, double* __restrict__ x, PcgScalars* __restrict__ sc,
                        double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  double v[2] = {0.0, 0.0};
  const int op[2] = {RED_MAX, RED_MAX};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const double d = q[a] - q1[a];
    x[a] = d;
    v[0] = fmax(v[0], fabs(d));
    v[1] = fmax(v[1], 1.0 / dinv[a]);
  }
  double tot[2];
  if (chunk_reduce<2>(v, op, ch, part, counter, tot)) {
    sc[ch.s].dmax = tot[0];
    sc[ch.s].dmaxD = tot[1];
  }
}

// r = r1 - Ad (see k_delta), A q = -chi - r for the energies, statistics and the final test
__global__ void k_resid_delta(const Chunk* __restrict__ chunks, const double* __restrict__ chi,
                              const double* __restrict__ r1, double* __restrict__ Ad, const double* __restrict__ dinv,
                              double* __restrict__ r, PcgScalars* __restrict__ sc, double* part, int* counter,
                              int max_iter, double op_err) {
  const Chunk ch = chunks[blockIdx.x];
  const double ref = sc[ch.s].shift;
  double v[6] = {0, 0, 0, -1e300, 1e300, 0};
  const int op[6] = {RED_SUM, RED_SUM, RED_SUM, RED_MAX, RED_MIN, RED_MAX};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const double ad = Ad[a];
    const double ra = r1[a] - ad;
    r[a] = ra;
    Ad[a] = -chi[a] - ra;
    v[0] += dinv[a] * ra;
    v[1] += ra - ref;
    v[2] += (ra - ref) * (ra - ref);
    v[3] = fmax(v[3], ra);
    v[4] = fmin(v[4], ra);
    v[5] = fmax(v[5], fabs(ad));
  }
  double tot[6];
  if (chunk_reduce<6>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    c.slack = op_err * (tot[5] + c.dmaxD * c.dmax);
    residual_test(c, tot, ref, max_iter, 1);
  }
}

__global__ void k_copy2(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* __restrict__ a1,
                        double* __restrict__ b1) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    a1[i] = a[i];
    b1[i] = b[i];
  }
}

// q += alpha p ; r -= alpha Ap ; statistics of the new r
__global__ void k_update(const Chunk* __restrict__ chunks, const double* __restrict__ p, const double* __restrict__ Ap,
                         const double* __restrict__ dinv, double* __restrict__ q, double* __restrict__ r,
                         PcgScalars* __restrict__ sc, double* part, int* counter, int max_iter) {
  const Chunk ch = chunks[blockIdx.x];
  if (!sc[ch.s].active) return;
  const double alpha = sc[ch.s].alpha;
  const double ref = sc[ch.s].shift;
  double v[5] = {0, 0, 0, -1e300, 1e300};
  const int op[5] = {RED_SUM, RED_SUM, RED_SUM, RED_MAX, RED_MIN};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    q[a] += alpha * p[a];
    double ra = r[a] - alpha * Ap[a];
    r[a] = ra;
    v[0] += dinv[a] * ra;
    v[1] += ra - ref;
    v[2] += (ra - ref) * (ra - ref);
    v[3] = fmax(v[3], ra);
    v[4] = fmin(v[4], ra);
  }
  double tot[5];
  if (chunk_reduce<5>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    c.iters += 1;
    residual_test(c, tot, ref, max_iter, 0);
  }
}

// z = D^-1 (r - shift); rz_new = r.z; beta.  Since 1^T z = 0, r.z = (r - shift).z; the
// second form is the one summed: r itself carries mu 1 (several eV), and near convergence
// shift * sum z (rounding of order eps mu) would swamp the projected part of r.z, which
// then corrupts alpha and beta and lets q wander along A^-1 1, a direction the projected
// residual does not see.  As summed, r.z = sum D^-1 (r - shift)^2 >= 0.
__global__ void k_precond(const Chunk* __restrict__ chunks, const double* __restrict__ r, const double* __restrict__ dinv,
                          double* __restrict__ z, PcgScalars* __restrict__ sc, int restart, double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  if (!sc[ch.s].active) return;
  const double sh = sc[ch.s].shift;
  double v[1] = {0};
  const int op[1] = {RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const double rp = r[a] - sh;
    double za = dinv[a] * rp;
    z[a] = za;
    v[0] += rp * za;
  }
  double tot[1];
  if (chunk_reduce<1>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    c.beta = (restart || c.rz == 0.0) ? 0.0 : tot[0] / c.rz;
    c.rz = tot[0];
  }
}

// Fourier preconditioner: z = u - w1 (sum u / sum w1) (so that 1^T z = 0); rz_new = r.z; beta.
// The Jacobi direction zj = D^-1 (r - shift) is formed beside it: if r.z of the
// Fourier direction is not positive (the preconditioner lost definiteness) the
// structure continues with Jacobi for the rest of the solve.
__global__ void k_proj_rz(const Chunk* __restrict__ chunks, const double* __restrict__ r, const double* __restrict__ u,
                          const double* __restrict__ w1, const double* __restrict__ dinv, double* __restrict__ z,
                          double* __restrict__ zj, PcgScalars* __restrict__ sc, int restart, double* part,
                          int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  if (!sc[ch.s].active) return;
  const double f = sc[ch.s].unconstrained ? 0.0 : sc[ch.s].usum / sc[ch.s].w1sum;  // no projection without the constraint
  const double sh = sc[ch.s].shift;
  double v[2] = {0, 0};
  const int op[2] = {RED_SUM, RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const double rp = r[a] - sh;  // both directions sum to zero: dot with r - shift (see k_precond)
    double za = u[a] - f * w1[a];
    double zja = dinv[a] * rp;
    z[a] = za;
    zj[a] = zja;
    v[0] += rp * za;
    v[1] += rp * zja;
  }
  double tot[2];
  if (chunk_reduce<2>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    if (!c.jacobi && !(tot[0] > 0.0 && isfinite(tot[0]))) {
      c.jacobi = 1;
      restart = 1;
    }
    double rz = c.jacobi ? tot[1] : tot[0];
    c.beta = (restart || c.rz == 0.0) ? 0.0 : rz / c.rz;
    c.rz = rz;
  }
}

// p = z + beta p  (zj instead of z for a structure that fell back to Jacobi)
__global__ void k_direction(const Chunk* __restrict__ chunks, const double* __restrict__ z,
                            const double* __restrict__ zj, double* __restrict__ p, const PcgScalars* __restrict__ sc) {
  const Chunk ch = chunks[blockIdx.x];
  if (!sc[ch.s].active) return;
  const double beta = sc[ch.s].beta;
  const double* zz = (zj && sc[ch.s].jacobi) ? zj : z;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) p[a] = zz[a] + beta * p[a];
}

// all structures inactive?  A timed-out device wait (ERRBIT_TIMEOUT) stops every structure.
__global__ void k_done(PcgScalars* __restrict__ sc, int ns, const int* __restrict__ err, int* __restrict__ done) {
  __shared__ int any;
  const bool stop = (*((volatile const int*)err) & ERRBIT_TIMEOUT) != 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    if (stop) sc[s].active = 0;
    if (sc[s].active) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) *done = any ? 0 : 1;
}

// after a final check: restart the failing structures (bounded), settle the rest
__global__ void k_after_check(PcgScalars* __restrict__ sc, int ns, int max_restarts, int max_iter,
                              const int* __restrict__ err, int* __restrict__ done) {
  __shared__ int any;
  const bool stop = (*((volatile const int*)err) & ERRBIT_TIMEOUT) != 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    PcgScalars& c = sc[s];
    if (stop) {
      c.status = QEQ_ERR_TIMEOUT;
      c.active = 0;
    } else if (c.converged) {
      c.status = QEQ_OK;
      c.active = 0;
    } else if (c.restarts < max_restarts && c.iters < max_iter) {
      c.restarts += 1;
      c.active = 1;
      any = 1;
    } else {
      c.status = QEQ_ERR_NOCONV;
      c.active = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *done = any ? 0 : 1;
}

// ---------------------------------------------------------------- device-paced solve graph
// The conditions of the graph's WHILE / IF nodes are set on the device from the
// per-structure state, by thread 0 only (one writer per handle).

// start of a round: reset the round's replay count; iterate while some structure is active
__global__ void k_round_begin(LoopCtl* __restrict__ ctl, const PcgScalars* __restrict__ sc, int ns,
                              const int* __restrict__ err, cudaGraphConditionalHandle h_inner) {
  __shared__ int any;
  const bool stop = (*((volatile const int*)err) & ERRBIT_TIMEOUT) != 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x)
    if (sc[s].active) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->replays_round = 0;
    cudaGraphSetConditional(h_inner, (any && !stop) ? 1u : 0u);
  }
}

// end of a block of iterations: continue while some structure is active, no device wait
// ran out, and the round has not used its replays (a second guard besides max_iter)
__global__ void k_inner_cond(PcgScalars* __restrict__ sc, int ns, const int* __restrict__ err,
                             LoopCtl* __restrict__ ctl, int cap, cudaGraphConditionalHandle h_inner) {
  __shared__ int any;
  const bool stop = (*((volatile const int*)err) & ERRBIT_TIMEOUT) != 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    if (stop) sc[s].active = 0;
    if (sc[s].active) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->replays_round += 1;
    ctl->replays_total += 1;
    cudaGraphSetConditional(h_inner, (any && ctl->replays_round < cap) ? 1u : 0u);
  }
}

// mixed precision: the rounds after the first FP64 check and before the last allowed
// restart check from the FP64 residual plus the FP32 product of the change (IF branch);
// the others run the full FP64 check (ELSE branch)
__global__ void k_choose_check(const LoopCtl* __restrict__ ctl, int max_restarts, cudaGraphConditionalHandle h_check) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h_check, (ctl->outer > 0 && ctl->outer < max_restarts) ? 1u : 0u);
}

// after a final check: restart the failing structures (bounded), settle the rest; another
// round while some structure restarts
__global__ void k_round_end(PcgScalars* __restrict__ sc, int ns, int max_restarts, int max_iter,
                            const int* __restrict__ err, LoopCtl* __restrict__ ctl, cudaGraphConditionalHandle h_outer) {
  __shared__ int any;
  const bool stop = (*((volatile const int*)err) & ERRBIT_TIMEOUT) != 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    PcgScalars& c = sc[s];
    if (stop) {
      c.status = QEQ_ERR_TIMEOUT;
      c.active = 0;
    } else if (c.converged) {
      c.status = QEQ_OK;
      c.active = 0;
    } else if (c.restarts < max_restarts && c.iters < max_iter) {
      c.restarts += 1;
      c.active = 1;
      any = 1;
    } else {
      c.status = QEQ_ERR_NOCONV;
      c.active = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->outer += 1;
    cudaGraphSetConditional(h_outer, (any && ctl->outer <= max_restarts + 1) ? 1u : 0u);
  }
}

__global__ void k_energy(const Chunk* __restrict__ chunks, const double* __restrict__ q, const double* __restrict__ Aq,
                         const double* __restrict__ chi, const double* __restrict__ J, PcgScalars* __restrict__ sc,
                         double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  double v[3] = {0, 0, 0};
  const int op[3] = {RED_SUM, RED_SUM, RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    v[0] += chi[a] * q[a];
    v[1] += q[a] * Aq[a];
    v[2] += J[a] * q[a] * q[a];
  }
  double tot[3];
  if (chunk_reduce<3>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    c.E_lin = tot[0];
    c.E_quad = tot[1];
    c.E_J = tot[2];
  }
}

// E(q) = chi.q + 1/2 q.A q with A q = -chi - r:  E = 1/2 chi.q - 1/2 q.r  (per structure, into E_lin)
__global__ void k_start_energy(const Chunk* __restrict__ chunks, const double* __restrict__ q,
                               const double* __restrict__ r, const double* __restrict__ chi,
                               PcgScalars* __restrict__ sc, double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  double v[2] = {0, 0};
  const int op[2] = {RED_SUM, RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    v[0] += chi[a] * q[a];
    v[1] += q[a] * r[a];
  }
  double tot[2];
  if (chunk_reduce<2>(v, op, ch, part, counter, tot)) sc[ch.s].E_lin = 0.5 * tot[0] - 0.5 * tot[1];
}

// per-structure sums of a vector (into E_quad): used for 1^T A 1 of the uniform start
__global__ void k_vec_sum(const Chunk* __restrict__ chunks, const double* __restrict__ y, PcgScalars* __restrict__ sc,
                          double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  double v[1] = {0};
  const int op[1] = {RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) v[0] += y[a];
  double tot[1];
  if (chunk_reduce<1>(v, op, ch, part, counter, tot)) sc[ch.s].E_quad = tot[0];
}

__global__ void k_flip(int* __restrict__ f, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = f[i] ? 0 : 1;
}

__global__ void k_fill(double* __restrict__ x, int64_t n, double v) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) x[a] = v;
}

__global__ void k_unsort(const int* __restrict__ perm, int64_t n, const double* __restrict__ src, double* __restrict__ dst) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) dst[perm[a]] = src[a];
}

__global__ void k_sort_in(const int* __restrict__ perm, int64_t n, const double* __restrict__ src, double* __restrict__ dst) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) dst[a] = src[perm[a]];
}

__global__ void k_write_mu(const PcgScalars* __restrict__ sc, int ns, double* __restrict__ mu,
                           double* __restrict__ E_qeq, double* __restrict__ E_elec) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const PcgScalars& c = sc[s];
  if (mu) mu[s] = -c.r_sum / (double)c.n;
  if (E_qeq) E_qeq[s] = c.E_lin + 0.5 * c.E_quad;
  if (E_elec) E_elec[s] = 0.5 * (c.E_quad - c.E_J);
}

// ------------------------------------------------------------------ host orchestration
qeq_status cuda_fail(qeq_plan_s* P, cudaError_t e, const char* where) {
  P->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // the error is reported here; do not leave it to the caller's next CUDA call
  return QEQ_ERR_CUDA;
}

#define TRY(expr)                                        \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(P, e_, #expr); \
  } while (0)

#define TRY_ST(expr)                 \
  do {                               \
    qeq_status st_ = (expr);         \
    if (st_ != QEQ_OK) return st_;   \
  } while (0)

int* red_counter(qeq_plan_s* P) { return P->d_counter + 2 * P->n_struct; }
double* red_part(qeq_plan_s* P) {
  return P->d_part + (size_t)P->n_chunks * QEQ_MAX_SPECIES +
         std::max<size_t>((size_t)P->total_bins, (size_t)P->n_chunks * QEQ_GATHER_SPLIT_MAX) + 8;
}

const double* dir_alt(qeq_plan_s* P) { return P->precond == QEQ_PRECOND_FOURIER ? P->d_x : nullptr; }

// z = preconditioned, projected residual; beta and rz (restart: beta = 0)
cudaError_t precondition(qeq_plan_s* P, int restart, int use_active) {
  cudaStream_t s = P->stream;
  int nc = P->n_chunks;
  if (P->precond == QEQ_PRECOND_FOURIER) {
    QEQ_CUDA_TRY(launch_precond(P, P->d_r, P->d_u, 0, use_active));
    count_launch(P);
    k_proj_rz<<<nc, 256, 0, s>>>(P->d_chunks, P->d_r, P->d_u, P->d_w1, P->d_dinv, P->d_z, P->d_x, P->d_sc, restart,
                                 red_part(P), red_counter(P));
  } else {
    count_launch(P);
    k_precond<<<nc, 256, 0, s>>>(P->d_chunks, P->d_r, P->d_dinv, P->d_z, P->d_sc, restart, red_part(P),
                                 red_counter(P));
  }
  return cudaGetLastError();
}

cudaError_t one_iteration(qeq_plan_s* P, int prec) {
  cudaStream_t s = P->stream;
  int nc = P->n_chunks;
  int max_iter = P->desc.max_iter;
  QEQ_CUDA_TRY(launch_matvec(P, prec, P->d_p, P->d_Ap, 1, 1, 1, nullptr));
  count_launch(P);
  k_update<<<nc, 256, 0, s>>>(P->d_chunks, P->d_p, P->d_Ap, P->d_dinv, P->d_q, P->d_r, P->d_sc, red_part(P),
                              red_counter(P), max_iter);
  QEQ_CUDA_TRY(precondition(P, 0, 1));
  count_launch(P);
  k_direction<<<nc, 256, 0, s>>>(P->d_chunks, P->d_z, dir_alt(P), P->d_p, P->d_sc);
  return cudaGetLastError();
}

const int kItersPerCheck = 4;
const int kMaxRestarts = 4;  // residual replacements after a failed final check
// mixed precision: the iterations stop at this fraction of the final check's thresholds
const double kMixedInnerTol = 0.5;
// mixed precision: residual reduction of one round of FP32 iterations (see residual_test)
const double kMixedRoundDrop = 1e-5;
// bound on the relative error of the FP32 operator, against max|A x| + max D max|x|
// (measured errors are below 1e-5 of that scale; 1e-4 leaves a margin of ten)
const double kMixedOpErr = 1e-4;

// host-paced iterations (QEQ_FLAG_NO_GRAPH or the legacy stream): a block of iterations,
// then the host reads whether any structure is still active
cudaError_t run_iterations(qeq_plan_s* P, int prec) {
  cudaStream_t s = P->stream;
  for (int k = 0; k < kItersPerCheck; ++k) QEQ_CUDA_TRY(one_iteration(P, prec));
  count_launch(P);
  k_done<<<1, 256, 0, s>>>(P->d_sc, P->n_struct, P->d_err, P->d_done);
  QEQ_CUDA_TRY(cudaMemcpyAsync(P->h_done, P->d_done, sizeof(int), cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

// the final check of a round (full FP64 residual, or in mixed precision the change-based one)
cudaError_t final_check(qeq_plan_s* P, int prec, bool use_delta) {
  cudaStream_t s = P->stream;
  const int nc = P->n_chunks, max_iter = P->desc.max_iter;
  const int nbv = (int)((P->n_atoms + 255) / 256);
  if (use_delta) {
    count_launch(P, 2);
    k_delta<<<nc, 256, 0, s>>>(P->d_chunks, P->d_q, P->d_q1, P->d_dinv, P->d_x, P->d_sc, red_part(P),
                               red_counter(P));
    QEQ_CUDA_TRY(launch_matvec(P, QEQ_MIXED, P->d_x, P->d_Ap, 1, 0, 0, nullptr));
    k_resid_delta<<<nc, 256, 0, s>>>(P->d_chunks, P->d_chi, P->d_r1, P->d_Ap, P->d_dinv, P->d_r, P->d_sc,
                                     red_part(P), red_counter(P), max_iter, kMixedOpErr);
  } else {
    QEQ_CUDA_TRY(launch_matvec(P, QEQ_FP64, P->d_q, P->d_Ap, 1, 0, 0, nullptr));
    count_launch(P);
    k_resid<<<nc, 256, 0, s>>>(P->d_chunks, P->d_chi, P->d_Ap, P->d_dinv, P->d_r, P->d_sc, 0, red_part(P),
                               red_counter(P), max_iter);
    if (prec == QEQ_MIXED) {
      count_launch(P);
      k_copy2<<<nbv, 256, 0, s>>>(P->d_q, P->d_r, P->n_atoms, P->d_q1, P->d_r1);
    }
  }
  return cudaGetLastError();
}

// Capture the kernels `launch` enqueues into graph g after the nodes deps; deps becomes
// the captured segment's last nodes.  Returns the segment's kernel count in *nk.
template <class F>
cudaError_t capture_segment(qeq_plan_s* P, cudaGraph_t g, std::vector<cudaGraphNode_t>& deps, int64_t* nk,
                            F&& launch) {
  cudaStream_t s = P->stream;
  QEQ_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                             cudaStreamCaptureModeThreadLocal));
  P->capturing = true;
  P->graph_kernels = 0;
  cudaError_t e = launch();
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* d = nullptr;
  size_t n = 0;
  cudaError_t e2 = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &d, nullptr, &n);
  std::vector<cudaGraphNode_t> last(d, d + n);
  cudaGraph_t out = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(s, &out);
  P->capturing = false;
  if (nk) *nk += P->graph_kernels;
  QEQ_CUDA_TRY(e);
  QEQ_CUDA_TRY(e2);
  QEQ_CUDA_TRY(e3);
  deps = last;
  return cudaSuccess;
}

// a conditional node after deps; its body graphs in bodies[0 .. size)
cudaError_t add_conditional(cudaGraph_t g, std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, unsigned size, cudaGraph_t* bodies) {
  // the parameter block is a union (no default constructor): zeroed raw storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& prm = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = size;
  cudaGraphNode_t node;
  QEQ_CUDA_TRY(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &prm));
  for (unsigned i = 0; i < size; ++i) bodies[i] = prm.conditional.phGraph_out[i];
  deps.assign(1, node);
  return cudaSuccess;
}

// The whole PCG of a solve as one graph, paced on the device:
//   WHILE round:                       (h_outer, set by k_round_end)
//     k_round_begin
//     WHILE block:                     (h_inner, set by k_round_begin / k_inner_cond)
//       4 PCG iterations, k_inner_cond
//     mixed: IF change-based check ELSE FP64 check   (h_check, set by k_choose_check)
//     FP64:  FP64 check
//     k_round_end, preconditioned restart direction
// The host launches it once and reads the per-structure results once.
cudaError_t build_solve_graph(qeq_plan_s* P, int prec) {
  if (P->graph_solve) {
    cudaGraphExecDestroy(P->graph_solve);
    P->graph_solve = nullptr;
  }
  cudaStream_t s = P->stream;
  const int ns = P->n_struct, nc = P->n_chunks, max_iter = P->desc.max_iter;
  const int max_restarts = kMaxRestarts;
  const int cap = max_iter / kItersPerCheck + 2;
  cudaGraph_t root = nullptr;
  QEQ_CUDA_TRY(cudaGraphCreate(&root, 0));
  cudaError_t e = cudaSuccess;
  P->gk_inner = 0;
  P->gk_round = 0;
  do {
    cudaGraphConditionalHandle h_outer, h_inner, h_check;
    if ((e = cudaGraphConditionalHandleCreate(&h_outer, root, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    std::vector<cudaGraphNode_t> deps;
    if ((e = capture_segment(P, root, deps, nullptr, [&]() {
           return cudaMemsetAsync(P->d_ctl, 0, sizeof(LoopCtl), s);
         })) != cudaSuccess)
      break;
    cudaGraph_t body_round;
    if ((e = add_conditional(root, deps, h_outer, cudaGraphCondTypeWhile, 1, &body_round)) != cudaSuccess) break;
    if ((e = cudaGraphConditionalHandleCreate(&h_inner, body_round, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
      break;
    std::vector<cudaGraphNode_t> rd;
    if ((e = capture_segment(P, body_round, rd, &P->gk_round, [&]() {
           count_launch(P);
           k_round_begin<<<1, 256, 0, s>>>(P->d_ctl, P->d_sc, ns, P->d_err, h_inner);
           return cudaGetLastError();
         })) != cudaSuccess)
      break;
    cudaGraph_t body_block;
    if ((e = add_conditional(body_round, rd, h_inner, cudaGraphCondTypeWhile, 1, &body_block)) != cudaSuccess) break;
    {
      std::vector<cudaGraphNode_t> bd;
      if ((e = capture_segment(P, body_block, bd, &P->gk_inner, [&]() {
             for (int k = 0; k < kItersPerCheck; ++k) QEQ_CUDA_TRY(one_iteration(P, prec));
             count_launch(P);
             k_inner_cond<<<1, 256, 0, s>>>(P->d_sc, ns, P->d_err, P->d_ctl, cap, h_inner);
             return cudaGetLastError();
           })) != cudaSuccess)
        break;
    }
    if (prec == QEQ_MIXED) {
      // (a handle no conditional node uses makes the instantiation fail: created only here)
      if ((e = cudaGraphConditionalHandleCreate(&h_check, body_round, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        break;
      if ((e = capture_segment(P, body_round, rd, &P->gk_round, [&]() {
             count_launch(P);
             k_choose_check<<<1, 32, 0, s>>>(P->d_ctl, max_restarts, h_check);
             return cudaGetLastError();
           })) != cudaSuccess)
        break;
      cudaGraph_t branch[2];
      if ((e = add_conditional(body_round, rd, h_check, cudaGraphCondTypeIf, 2, branch)) != cudaSuccess) break;
      std::vector<cudaGraphNode_t> b0, b1;
      int64_t k0 = 0, k1 = 0;
      if ((e = capture_segment(P, branch[0], b0, &k0, [&]() { return final_check(P, prec, true); })) != cudaSuccess)
        break;
      if ((e = capture_segment(P, branch[1], b1, &k1, [&]() { return final_check(P, prec, false); })) != cudaSuccess)
        break;
      P->gk_round += std::max(k0, k1);
    } else {
      if ((e = capture_segment(P, body_round, rd, &P->gk_round, [&]() { return final_check(P, prec, false); })) !=
          cudaSuccess)
        break;
    }
    if ((e = capture_segment(P, body_round, rd, &P->gk_round, [&]() {
           count_launch(P);
           k_round_end<<<1, 256, 0, s>>>(P->d_sc, ns, max_restarts, max_iter, P->d_err, P->d_ctl, h_outer);
           QEQ_CUDA_TRY(precondition(P, 1, 1));
           count_launch(P);
           k_direction<<<nc, 256, 0, s>>>(P->d_chunks, P->d_z, dir_alt(P), P->d_p, P->d_sc);
           return cudaGetLastError();
         })) != cudaSuccess)
      break;
    e = cudaGraphInstantiate(&P->graph_solve, root, 0);
  } while (false);
  cudaGraphDestroy(root);
  if (e != cudaSuccess) {
    P->graph_solve = nullptr;
    return e;
  }
  P->graph_solve_prec = prec;
  return cudaSuccess;
}

qeq_status check_inputs(qeq_plan_s* P) {
  int err = 0;
  TRY(cudaMemcpyAsync(P->h_done + 4, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  TRY(cudaStreamSynchronize(P->stream));
  err = P->h_done[4];
  if (err) {
    TRY(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->stream));
    if (err & ERRBIT_J) {
      P->last_error = "hardness J must be > 0";
      return QEQ_ERR_NOT_PD;
    }
    if (err & ERRBIT_PAIRCAP) {
      P->last_error = "real-space pair list exceeds capacity";
      return QEQ_ERR_CAPACITY;
    }
    P->last_error = (err & ERRBIT_SPECIES) ? "species index out of range" : "non-finite input";
    return QEQ_ERR_INVALID;
  }
  return QEQ_OK;
}

// after a call's device work: a bounded device wait that ran out (ERRBIT_TIMEOUT)
qeq_status check_timeout(qeq_plan_s* P) {
  TRY(cudaMemcpyAsync(P->h_done + 5, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  TRY(cudaStreamSynchronize(P->stream));
  if (P->h_done[5] & ERRBIT_TIMEOUT) {
    TRY(cudaMemsetAsync(P->d_err, 0, sizeof(int), P->stream));
    TRY(cudaStreamSynchronize(P->stream));
    P->last_error = "a bounded device wait (bulk copy into shared memory) ran out";
    return QEQ_ERR_TIMEOUT;
  }
  return QEQ_OK;
}

qeq_status prepare(qeq_plan_s* P, const double* d_pos, const int32_t* d_species, const double* d_chi,
                   const double* d_J) {
  if (!d_pos || !d_species || !d_chi || !d_J) {
    P->last_error = "null input pointer";
    return QEQ_ERR_INVALID;
  }
  TRY(cudaSetDevice(P->device));
  TRY(launch_prepare_atoms(P, d_pos, d_species, d_chi, d_J, P->pair_cap > 0));
  return check_inputs(P);
}

qeq_status init_scalars(qeq_plan_s* P, const double* h_qtot) {
  std::vector<PcgScalars> h(P->n_struct);
  for (int s = 0; s < P->n_struct; ++s) {
    PcgScalars& c = h[s];
    memset(&c, 0, sizeof(c));
    c.n = (int)(P->hs[s].atom_end - P->hs[s].atom_begin);
    c.q_tot = h_qtot ? h_qtot[s] : 0.0;
    c.active = 1;
    c.status = QEQ_OK;
  }
  TRY(cudaMemcpyAsync(P->d_sc, h.data(), sizeof(PcgScalars) * h.size(), cudaMemcpyHostToDevice, P->stream));
  TRY(cudaStreamSynchronize(P->stream));  // h goes out of scope
  return QEQ_OK;
}

__global__ void k_set_tol(PcgScalars* sc, int ns, double charge_tol, double rel_tol, double inner,
                          int unconstrained, double scale) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  PcgScalars& c = sc[s];
  c.tol_inf = scale * 0.5 * charge_tol * c.j_min;
  c.tol_l2 = rel_tol > 0 ? scale * rel_tol * sqrt(c.chi_p2) : 0.0;
  c.inner = inner;
  c.unconstrained = unconstrained;
  // mixed precision (inner < 1): a round of FP32 iterations reduces its residual at most
  // kMixedRoundDrop-fold before the next check (the floors are set by each check)
  c.drop = inner < 1.0 ? kMixedRoundDrop : 0.0;
  c.floor_inf = c.floor_l2 = 0.0;
}

// two-RHS solver: per structure sum s (sorted, in q) and sum t (t in input order, in t_in)
__global__ void k_two_rhs_sums(const Chunk* __restrict__ chunks, const int* __restrict__ perm,
                               const double* __restrict__ q, const double* __restrict__ t_in,
                               PcgScalars* __restrict__ sc, double* part, int* counter) {
  const Chunk ch = chunks[blockIdx.x];
  double v[2] = {0.0, 0.0};
  const int op[2] = {RED_SUM, RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    v[0] += q[a];
    v[1] += t_in[perm[a]];
  }
  double tot[2];
  if (chunk_reduce<2>(v, op, ch, part, counter, tot)) {
    sc[ch.s].qsum = tot[0];
    sc[ch.s].tsum = tot[1];
  }
}

// q = s + mu' t with mu' = (q_tot - sum s) / sum t, so that sum q = q_tot; the combined
// charges go to out (input order), from which the final check reads them
__global__ void k_two_rhs_combine(const Chunk* __restrict__ chunks, const int* __restrict__ perm,
                                  const double* __restrict__ q, double* __restrict__ t_out,
                                  const PcgScalars* __restrict__ sc) {
  const Chunk ch = chunks[blockIdx.x];
  const PcgScalars& c = sc[ch.s];
  const double m = (c.q_tot - c.qsum) / c.tsum;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const int i = perm[a];
    t_out[i] = q[a] + m * t_out[i];
  }
}

// ---------------------------------------------------------------- SQNM solver
// Stabilised quasi-Newton minimiser of E(q) = chi.q + 1/2 q.(E + diag J) q on the constraint
// plane (the alternative to CG in the paper's solver comparison, SI solver figure), in the
// Jacobi-scaled coordinates x = D^{1/2} q where the projected gradient is
// g = D^{-1/2} (A q + chi - c 1), c = sum D^-1 (A q + chi) / sum D^-1 (the steepest-descent
// direction -D^{-1/2} g is the PCG's Jacobi direction).  From the last steps dx_i and
// gradient changes dg_i: the significant subspace of the normalised steps (eigenvalues of
// their overlap above 1e-4 of the largest), the symmetrised Hessian in it, Newton steps
// along its eigenvectors with curvatures enlarged by their residues, and a steepest-descent
// step alpha in the complement; alpha grows by 1.1 while the energy falls and halves, with
// the history cleared and the step undone, when it rises (the rise judged from the
// gradients at both ends of the step, exact for the quadratic energy).  A q comes from y = y1 + A (q - q1): y1 = A q1 by the
// last FP64 matvec (q1 = 0 in FP64 plans), the change in the plan's precision.

// y + chi statistics: [0] sum D^-1 (y + chi), [1] sum (y + chi - ref), [2] sum (..)^2, [3] max,
// [4] min of y + chi, [5] the energy chi.q + 1/2 q.y; the convergence test on the projected
// residual -(y + chi) (residual_test's form, negated)
__global__ void k_sqnm_stats(const Chunk* __restrict__ chunks, const double* __restrict__ y1,
                             const double* __restrict__ Ad, const double* __restrict__ chi,
                             const double* __restrict__ dinv, const double* __restrict__ q,
                             PcgScalars* __restrict__ sc, SqnmState* __restrict__ qs, double* part, int* counter,
                             int max_iter, int final_check) {
  const Chunk ch = chunks[blockIdx.x];
  if (!final_check && !sc[ch.s].active) return;
  const double ref = qs[ch.s].c;
  double v[6] = {0, 0, 0, -1e300, 1e300, 0};
  const int op[6] = {RED_SUM, RED_SUM, RED_SUM, RED_MAX, RED_MIN, RED_SUM};
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const double ya = (y1 ? y1[a] : 0.0) + Ad[a];
    const double e = ya + chi[a];
    v[0] += dinv[a] * e;
    v[1] += e - ref;
    v[2] += (e - ref) * (e - ref);
    v[3] = fmax(v[3], e);
    v[4] = fmin(v[4], e);
    v[5] += q[a] * (chi[a] + 0.5 * ya);
  }
  double tot[6];
  if (chunk_reduce<6>(v, op, ch, part, counter, tot)) {
    PcgScalars& c = sc[ch.s];
    SqnmState& S = qs[ch.s];
    const double n = (double)c.n;
    S.c = tot[0] / c.s0;
    S.E = tot[5];
    // residual r = -(y + chi): sum, max, min; ||P r|| about ref
    c.r_sum = -(ref * n + tot[1]);
    c.r_max = -tot[4];
    c.r_min = -tot[3];
    const double dmean = tot[1] / n, mean = -(ref + dmean);
    const double pinf = fmax(c.r_max - mean, mean - c.r_min);
    c.r_l2 = sqrt(fmax(tot[2] - tot[1] * dmean, 0.0));
    // as residual_test: in mixed precision a round also ends once its residual fell `drop`-fold
    const double ti = final_check ? c.tol_inf : fmax(c.inner * c.tol_inf, c.floor_inf);
    const double tl = final_check ? c.tol_l2 : fmax(c.inner * c.tol_l2, c.floor_l2);
    const bool ok = isfinite(pinf) && pinf <= ti && (c.tol_l2 <= 0.0 || c.r_l2 <= tl);
    if (final_check) {
      c.converged = ok ? 1 : 0;
      c.floor_inf = c.drop * pinf;
      c.floor_l2 = c.drop * c.r_l2;
    } else if (ok) {
      c.converged = 1;
      c.active = 0;
    } else if (c.iters >= max_iter) {
      c.active = 0;
    }
  }
}

// g = D^{-1/2} (y + chi - c) (stored), the new gradient change dg_h = g - g_prev into slot h
// (when a step was taken), and the dot products of the new history row and of g with the
// history: [0..H) g.dx_i, [H] g.g, then per slot j: dx_h.dx_j, dx_h.dg_j, dx_j.dg_h, dg_h.dg_j.
// The structure's last chunk adds the chunk partials in chunk order into its state.
__global__ void __launch_bounds__(256) k_sqnm_dots(const Chunk* __restrict__ chunks, const double* __restrict__ y1,
                                                   const double* __restrict__ Ad, const double* __restrict__ chi,
                                                   const double* __restrict__ dinv, const PcgScalars* __restrict__ sc,
                                                   SqnmState* __restrict__ qs, int64_t N, double* __restrict__ g,
                                                   double* __restrict__ dx, double* __restrict__ dg,
                                                   double* __restrict__ part, int* __restrict__ counter) {
  constexpr int H = QEQ_SQNM_HISTORY, ND = QEQ_SQNM_NDOT, PS = QEQ_SQNM_NDOT + 7;
  __shared__ double red[8];
  __shared__ bool last;
  const Chunk ch = chunks[blockIdx.x];
  if (!sc[ch.s].active) return;
  SqnmState& S = qs[ch.s];
  const int cnt = S.count, h = S.head, hp = S.has_prev;
  const double cc = S.c;
  double v[ND];
#pragma unroll
  for (int k = 0; k < ND; ++k) v[k] = 0.0;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    const double ga = sqrt(dinv[a]) * ((y1 ? y1[a] : 0.0) + Ad[a] + chi[a] - cc);
    double dgh = 0.0;
    if (hp && cnt > 0) {
      dgh = ga - g[a];
      dg[(int64_t)h * N + a] = dgh;
    }
    g[a] = ga;
    v[H] += ga * ga;
    const double dxh = (cnt > 0) ? dx[(int64_t)h * N + a] : 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      if (j >= cnt) break;
      const double dxj = dx[(int64_t)j * N + a];
      const double dgj = (j == h) ? dgh : dg[(int64_t)j * N + a];
      v[j] += ga * dxj;
      if (hp) {
        v[H + 1 + 4 * j] += dxh * dxj;
        v[H + 2 + 4 * j] += dxh * dgj;
        v[H + 3 + 4 * j] += dxj * dgh;
        v[H + 4 + 4 * j] += dgh * dgj;
      }
    }
  }
  // fixed-order block sums (shuffle tree, warps in order) of every value
  const int nw = blockDim.x >> 5;
#pragma unroll 1
  for (int k = 0; k < ND; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < nw; ++i) t += red[i];
      part[(size_t)blockIdx.x * PS + k] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter + ch.s, 1) == ch.count - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x != 0) return;
  double t[ND];
  for (int k = 0; k < ND; ++k) t[k] = 0.0;
  for (int c = 0; c < ch.count; ++c)
    for (int k = 0; k < ND; ++k) t[k] += ((volatile double*)part)[(size_t)(ch.first + c) * PS + k];
  counter[ch.s] = 0;
  for (int j = 0; j < cnt; ++j) S.gX[j] = t[j];
  S.gg = t[H];
  if (hp) {
    for (int j = 0; j < cnt; ++j) {
      S.XX[h][j] = S.XX[j][h] = t[H + 1 + 4 * j];
      S.XG[h][j] = t[H + 2 + 4 * j];
      S.XG[j][h] = t[H + 3 + 4 * j];
      S.GG[h][j] = S.GG[j][h] = t[H + 4 + 4 * j];
    }
  }
}

// symmetric eigen-decomposition of an n x n matrix (n <= QEQ_SQNM_HISTORY) by cyclic Jacobi
// rotations: a is overwritten (its diagonal becomes the eigenvalues), v gets the eigenvectors
// as columns
__device__ void sqnm_jacobi_eig(double (*a)[QEQ_SQNM_HISTORY], double (*v)[QEQ_SQNM_HISTORY], int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a[i][i] * a[i][i];
      for (int j = i + 1; j < n; ++j) off += a[i][j] * a[i][j];
    }
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (a[p][q] == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = cs * akp - sn * akq;
          a[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = cs * apk - sn * aqk;
          a[q][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = cs * vkp - sn * vkq;
          v[k][q] = sn * vkp + cs * vkq;
        }
      }
  }
}

// one thread per structure: alpha from the energy change, the subspace quantities and the
// step coefficients; then the slot the coming step is stored in
__global__ void k_sqnm_plan(const PcgScalars* __restrict__ sc, SqnmState* __restrict__ qs, int ns) {
  constexpr int H = QEQ_SQNM_HISTORY;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns || !sc[s].active) return;
  SqnmState& S = qs[s];
  S.revert = 0;
  if (S.has_prev && S.count > 0) {
    // energy change of the last step dx_h, exact for the quadratic E:
    // dE = 1/2 dx_h . (g_prev + g) = g . dx_h - 1/2 dx_h . dg_h (noise scales with the step,
    // unlike a difference of two energies in mixed precision)
    const int h = S.head;
    const double dE = S.gX[h] - 0.5 * S.XG[h][h];
    if (dE > 1e-14 * fabs(S.E)) {
      // the last step raised the energy: undo it (the step kernel subtracts slot head),
      // halve alpha, forget the history; the next matvec re-evaluates the old point
      S.revert = 1;
      S.alpha *= 0.5;
      S.count = 0;
      S.has_prev = 0;
      S.E = S.E_prev;
      return;
    }
    S.alpha = fmin(S.alpha * 1.1, 4.0);
  }
  const int n = S.count;
  for (int i = 0; i < H; ++i) S.coef[i] = 0.0;
  S.subspace = 0;
  if (n > 0) {
    double nrm[H], A[H][H], U[H][H];
    for (int i = 0; i < n; ++i) nrm[i] = sqrt(fmax(S.XX[i][i], 1e-300));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i][j] = S.XX[i][j] / (nrm[i] * nrm[j]);
    sqnm_jacobi_eig(A, U, n);
    double lmax = 0.0;
    for (int l = 0; l < n; ++l) lmax = fmax(lmax, A[l][l]);
    // V: coefficients of the orthonormal subspace vectors on the raw dx_i
    double V[H][H];
    int m = 0;
    for (int l = 0; l < n; ++l) {
      if (!(A[l][l] > 1e-4 * lmax)) continue;
      const double sl = 1.0 / sqrt(A[l][l]);
      for (int i = 0; i < n; ++i) V[i][m] = U[i][l] * sl / nrm[i];
      ++m;
    }
    // subspace Hessian: 1/2 (V^T XG V + (V^T XG V)^T)
    double Hs[H][H], Q[H][H];
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        double t = 0.0;
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) t += V[i][a] * V[j][b] * (S.XG[i][j] + S.XG[j][i]);
        Hs[a][b] = 0.5 * t;
      }
    sqnm_jacobi_eig(Hs, Q, m);
    for (int jdir = 0; jdir < m; ++jdir) {
      double B[H];  // coefficients of direction jdir on the raw dx_i
      for (int i = 0; i < n; ++i) {
        double t = 0.0;
        for (int a = 0; a < m; ++a) t += V[i][a] * Q[a][jdir];
        B[i] = t;
      }
      const double kap = Hs[jdir][jdir];
      double yy = 0.0, wy = 0.0, ww = 0.0, gw = 0.0;
      for (int i = 0; i < n; ++i) {
        gw += B[i] * S.gX[i];
        for (int k = 0; k < n; ++k) {
          yy += B[i] * B[k] * S.GG[i][k];
          wy += B[i] * B[k] * S.XG[i][k];
          ww += B[i] * B[k] * S.XX[i][k];
        }
      }
      const double res2 = fmax(yy - 2.0 * kap * wy + kap * kap * ww, 0.0);
      const double kt = sqrt(kap * kap + res2);
      if (!(kt > 0.0) || !isfinite(kt)) continue;
      const double f = (S.alpha - 1.0 / kt) * gw;
      for (int i = 0; i < n; ++i) S.coef[i] += f * B[i];
    }
    S.subspace = m;
  }
  // slot of the coming step: the next slot, overwriting the oldest entry once full
  const int nh = (n == 0) ? 0 : (S.head + 1) % H;
  S.head = nh;
  S.count = n < H ? n + 1 : H;
  S.has_prev = 1;
  S.E_prev = S.E;
}

__global__ void k_sqnm_count(PcgScalars* __restrict__ sc, int ns) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns && sc[s].active) sc[s].iters += 1;
}

// dx = -alpha g + sum_i coef_i dx_i (scaled coordinates), q += D^{-1/2} dx, dx into the new slot
__global__ void k_sqnm_step(const Chunk* __restrict__ chunks, const PcgScalars* __restrict__ sc,
                            const SqnmState* __restrict__ qs, int64_t N, const double* __restrict__ g,
                            double* __restrict__ dx, const double* __restrict__ dinv, double* __restrict__ q) {
  constexpr int H = QEQ_SQNM_HISTORY;
  const Chunk ch = chunks[blockIdx.x];
  if (!sc[ch.s].active) return;
  const SqnmState& S = qs[ch.s];
  const int cnt = S.count, h = S.head;
  if (S.revert) {  // back to the point before the last step (slot h holds that step)
    for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) q[a] -= sqrt(dinv[a]) * dx[(int64_t)h * N + a];
    return;
  }
  // coefficients of the previous entries (the new slot h held the oldest entry when full)
  double cf[H];
#pragma unroll
  for (int i = 0; i < H; ++i) cf[i] = S.coef[i];
  const double al = S.alpha;
  for (int64_t a = ch.begin + threadIdx.x; a < ch.end; a += blockDim.x) {
    double d = -al * g[a];
#pragma unroll
    for (int i = 0; i < H; ++i)
      if (i < cnt && cf[i] != 0.0) d += cf[i] * dx[(int64_t)i * N + a];
    dx[(int64_t)h * N + a] = d;
    q[a] += sqrt(dinv[a]) * d;
  }
}

__global__ void k_sqnm_init(const PcgScalars* __restrict__ sc, SqnmState* __restrict__ qs, int ns) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  SqnmState& S = qs[s];
  S.count = 0;
  S.head = 0;
  S.has_prev = 0;
  S.alpha = 1.0;
  S.c = 0.0;
  S.E = S.E_prev = 0.0;
  S.subspace = 0;
  S.revert = 0;
  (void)sc;
}

__global__ void k_sub2(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] - b[i];
}

// SQNM rounds from the current q (the start of qeq_solve has run: q on the constraint plane,
// scalars and tolerances set): blocks of SQNM steps paced from the host, an FP64 check per
// round, restarts (with a fresh history) for the structures whose check fails.
qeq_status sqnm_rounds(qeq_plan_s* P, int prec) {
  cudaStream_t s = P->stream;
  const int nc = P->n_chunks, ns = P->n_struct, max_iter = P->desc.max_iter;
  const int nb = (int)((P->n_atoms + 255) / 256);
  const int64_t N = P->n_atoms;
  const bool mixed = prec == QEQ_MIXED;
  int* sq_counter = P->d_counter + 3 * ns;
  for (int outer = 0; outer <= kMaxRestarts + 1; ++outer) {
    count_launch(P);
    k_sqnm_init<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, P->d_sqnm, ns);
    if (mixed) {  // y1 = A q1 in FP64 at the round's start, q1 = q
      TRY(launch_matvec(P, QEQ_FP64, P->d_q, P->d_r1, 1, 0, 0, nullptr));
      count_launch(P);
      k_copy2<<<nb, 256, 0, s>>>(P->d_q, P->d_q, N, P->d_q1, P->d_x);
    }
    TRY(cudaGetLastError());
    const int max_launches = max_iter / kItersPerCheck + 2;
    for (int l = 0; l < max_launches; ++l) {
      for (int k = 0; k < kItersPerCheck; ++k) {
        const double* x = P->d_q;
        if (mixed) {
          count_launch(P);
          k_sub2<<<nb, 256, 0, s>>>(N, P->d_q, P->d_q1, P->d_x);
          x = P->d_x;
        }
        TRY(launch_matvec(P, prec, x, P->d_Ap, 1, 1, 0, nullptr));
        count_launch(P, 5);
        k_sqnm_stats<<<nc, 256, 0, s>>>(P->d_chunks, mixed ? P->d_r1 : nullptr, P->d_Ap, P->d_chi, P->d_dinv, P->d_q,
                                        P->d_sc, P->d_sqnm, red_part(P), red_counter(P), max_iter, 0);
        k_sqnm_dots<<<nc, 256, 0, s>>>(P->d_chunks, mixed ? P->d_r1 : nullptr, P->d_Ap, P->d_chi, P->d_dinv, P->d_sc,
                                       P->d_sqnm, N, P->d_sqnm_g, P->d_sqnm_dx, P->d_sqnm_dg, P->d_sqnm_part,
                                       sq_counter);
        k_sqnm_plan<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, P->d_sqnm, ns);
        k_sqnm_step<<<nc, 256, 0, s>>>(P->d_chunks, P->d_sc, P->d_sqnm, N, P->d_sqnm_g, P->d_sqnm_dx, P->d_dinv,
                                       P->d_q);
        k_sqnm_count<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, ns);
        TRY(cudaGetLastError());
      }
      count_launch(P);
      k_done<<<1, 256, 0, s>>>(P->d_sc, ns, P->d_err, P->d_done);
      TRY(cudaMemcpyAsync(P->h_done, P->d_done, sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaStreamSynchronize(s));
      if (P->h_done[0]) break;
    }
    // FP64 check of every structure: y = A q, the projected residual, the energy terms
    TRY(launch_matvec(P, QEQ_FP64, P->d_q, P->d_Ap, 1, 0, 0, nullptr));
    count_launch(P, 2);
    k_sqnm_stats<<<nc, 256, 0, s>>>(P->d_chunks, nullptr, P->d_Ap, P->d_chi, P->d_dinv, P->d_q, P->d_sc, P->d_sqnm,
                                    red_part(P), red_counter(P), max_iter, 1);
    k_after_check<<<1, 256, 0, s>>>(P->d_sc, ns, kMaxRestarts, max_iter, P->d_err, P->d_done);
    TRY(cudaGetLastError());
    TRY(cudaMemcpyAsync(P->h_done, P->d_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (P->h_done[0]) break;
  }
  return QEQ_OK;
}

// Every PCG round from the current q and r: the first direction, then the device-paced
// graph (or the host loop) until every structure has stopped.
qeq_status pcg_rounds(qeq_plan_s* P, int prec) {
  cudaStream_t s = P->stream;
  const int nc = P->n_chunks, ns = P->n_struct, max_iter = P->desc.max_iter;
  TRY(precondition(P, 1, 1));
  count_launch(P);
  k_direction<<<nc, 256, 0, s>>>(P->d_chunks, P->d_z, dir_alt(P), P->d_p, P->d_sc);
  TRY(cudaGetLastError());
  const int max_restarts = kMaxRestarts;
  if (P->graph_ok) {
    // device-paced: every round of the PCG in one graph launch
    if (!P->graph_solve || P->graph_solve_prec != prec) TRY(build_solve_graph(P, prec));
    TRY(cudaGraphLaunch(P->graph_solve, s));
  } else {
    for (int outer = 0; outer <= max_restarts + 1; ++outer) {
      // inner iterations (structures drop out as they converge); the device stops every
      // structure at max_iter, the host bound is a second guard
      const int max_launches = max_iter / kItersPerCheck + 2;
      for (int l = 0; l < max_launches; ++l) {
        TRY(run_iterations(P, prec));
        if (P->h_done[0]) break;
      }
      TRY(final_check(P, prec, prec == QEQ_MIXED && outer > 0 && outer < max_restarts));
      count_launch(P);
      k_after_check<<<1, 256, 0, s>>>(P->d_sc, ns, max_restarts, max_iter, P->d_err, P->d_done);
      TRY(precondition(P, 1, 1));
      count_launch(P);
      k_direction<<<nc, 256, 0, s>>>(P->d_chunks, P->d_z, dir_alt(P), P->d_p, P->d_sc);
      TRY(cudaGetLastError());
      TRY(cudaMemcpyAsync(P->h_done, P->d_done, sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaStreamSynchronize(s));
      if (P->h_done[0]) break;
    }
  }
  return QEQ_OK;
}

// kernels the device-paced graph ran so far in this solve (read from its loop counters)
qeq_status account_graph(qeq_plan_s* P) {
  if (!P->graph_ok) return QEQ_OK;
  LoopCtl ctl;
  TRY(cudaMemcpyAsync(&ctl, P->d_ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, P->stream));
  TRY(cudaStreamSynchronize(P->stream));
  P->launches += P->gk_inner * ctl.replays_total + P->gk_round * ctl.outer;
  return QEQ_OK;
}

// Two-RHS solver (the iterative-QEq formulation used for comparison with n2p2): plain
// PCG on A t = 1 and A s = -chi, A = E + diag J (no charge constraint), then
// q = s + mu' t with mu' = (q_tot - sum s)/sum t.  Each sub-solve stops at a quarter of
// the constrained threshold; the combined charges then get the usual projected FP64
// check.  t waits in the caller's output buffer while s is solved.  Returns the sub-solves'
// iterations and worst status.
qeq_status two_rhs_phase(qeq_plan_s* P, const double* d_chi_user, const double* h_qtot, double* d_q_user,
                         int* iters, int* restarts, int* status) {
  cudaStream_t s = P->stream;
  const int nc = P->n_chunks, ns = P->n_struct, prec = P->precision, max_iter = P->desc.max_iter;
  const int nb = (int)((P->n_atoms + 255) / 256);
  std::vector<PcgScalars> h(ns);
  for (int i = 0; i < ns; ++i) iters[i] = restarts[i] = status[i] = 0;
  for (int rhs = 0; rhs < 2; ++rhs) {
    if (rhs == 0) {  // chi := -1: r = 1 - A t
      count_launch(P);
      k_fill<<<nb, 256, 0, s>>>(P->d_chi, P->n_atoms, -1.0);
    } else {  // the caller's chi again (prepare sorted it into d_chi)
      count_launch(P);
      k_sort_in<<<nb, 256, 0, s>>>(P->d_perm, P->n_atoms, d_chi_user, P->d_chi);
      TRY_ST(init_scalars(P, h_qtot));
    }
    count_launch(P, 2);
    k_init<<<nc, 256, 0, s>>>(P->d_chunks, P->d_perm, nullptr, QEQ_WARM_COLD, nullptr, P->d_dinv, P->d_chi, P->d_J,
                              P->d_q, P->d_sc, red_part(P), red_counter(P));
    k_set_tol<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, ns, P->desc.charge_tol, P->desc.residual_tol,
                                               prec == QEQ_MIXED ? kMixedInnerTol : 1.0, 1, 0.25);
    TRY(cudaGetLastError());
    if (P->precond == QEQ_PRECOND_FOURIER) {  // w1 is read (times 0) by the direction kernel
      count_launch(P);
      k_fill<<<nb, 256, 0, s>>>(P->d_x, P->n_atoms, 1.0);
      TRY(launch_precond(P, P->d_x, P->d_w1, 1, 0));
    }
    TRY(launch_matvec(P, prec, P->d_q, P->d_Ap, 1, 0, 0, nullptr));
    count_launch(P);
    k_resid<<<nc, 256, 0, s>>>(P->d_chunks, P->d_chi, P->d_Ap, P->d_dinv, P->d_r, P->d_sc, 0, red_part(P),
                               red_counter(P), max_iter);
    TRY(cudaGetLastError());
    TRY_ST(pcg_rounds(P, prec));
    TRY_ST(account_graph(P));
    TRY(cudaMemcpyAsync(h.data(), P->d_sc, sizeof(PcgScalars) * ns, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < ns; ++i) {
      iters[i] += h[i].iters;
      restarts[i] += h[i].restarts;
      if (h[i].status != QEQ_OK && status[i] == QEQ_OK) status[i] = h[i].status;
    }
    if (rhs == 0) {  // t -> the caller's buffer (input order)
      count_launch(P);
      k_unsort<<<nb, 256, 0, s>>>(P->d_perm, P->n_atoms, P->d_q, d_q_user);
      TRY(cudaGetLastError());
    }
  }
  count_launch(P, 2);
  k_two_rhs_sums<<<nc, 256, 0, s>>>(P->d_chunks, P->d_perm, P->d_q, d_q_user, P->d_sc, red_part(P), red_counter(P));
  k_two_rhs_combine<<<nc, 256, 0, s>>>(P->d_chunks, P->d_perm, P->d_q, d_q_user, P->d_sc);
  TRY(cudaGetLastError());
  // the combined charges as the start of a constrained "solve" with no iterations: its
  // statistics, tolerance and the FP64 check of the result
  TRY_ST(init_scalars(P, h_qtot));
  count_launch(P, 2);
  k_init<<<nc, 256, 0, s>>>(P->d_chunks, P->d_perm, d_q_user, QEQ_WARM_USER, nullptr, P->d_dinv, P->d_chi, P->d_J,
                            P->d_q, P->d_sc, red_part(P), red_counter(P));
  k_set_tol<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, ns, P->desc.charge_tol, P->desc.residual_tol, 1.0, 0, 1.0);
  TRY(cudaGetLastError());
  TRY(final_check(P, QEQ_FP64, false));
  return QEQ_OK;
}

}  // namespace

extern "C" qeq_status qeq_solve(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_chi,
                                const double* d_J, const double* h_qtot, int32_t warm, double* d_q, double* d_mu,
                                qeq_info* h_info) {
  if (!P) return QEQ_ERR_INVALID;
  if (!d_q) {
    P->last_error = "d_q is required";
    return QEQ_ERR_INVALID;
  }
  if (!h_qtot) {
    P->last_error = "h_qtot is required";
    return QEQ_ERR_INVALID;
  }
  for (int s = 0; s < P->n_struct; ++s)
    if (!std::isfinite(h_qtot[s])) {
      P->last_error = "non-finite q_tot";
      return QEQ_ERR_INVALID;
    }
  qeq_status st = prepare(P, d_pos, d_species, d_chi, d_J);
  if (st != QEQ_OK) return st;
  st = init_scalars(P, h_qtot);
  if (st != QEQ_OK) return st;
  cudaStream_t s = P->stream;
  const int nc = P->n_chunks, ns = P->n_struct;
  const int prec = P->precision;
  const int max_iter = P->desc.max_iter;
  const bool two_rhs = (P->desc.flags & QEQ_FLAG_TWO_RHS) != 0;
  std::vector<int> warm_kept(ns, 0);
  std::vector<int> tr_iters(ns, 0), tr_rest(ns, 0), tr_status(ns, 0);
  if (two_rhs) {
    if (warm != QEQ_WARM_COLD) {
      P->last_error = "the two-RHS solver starts cold";
      return QEQ_ERR_INVALID;
    }
    if (P->precond == QEQ_PRECOND_FOURIER) TRY(launch_precond_setup(P));
    TRY_ST(two_rhs_phase(P, d_chi, h_qtot, d_q, tr_iters.data(), tr_rest.data(), tr_status.data()));
  } else {
  int wm = (warm == QEQ_WARM_USER) ? QEQ_WARM_USER : QEQ_WARM_COLD;
  if (warm == QEQ_WARM_MLP) {
    if (!P->mlp) {
      P->last_error = "QEQ_WARM_MLP needs a network attached with qeq_plan_set_warm_start";
      return QEQ_ERR_INVALID;
    }
    TRY(launch_mlp_warm_start(P, P->d_q));
    wm = QEQ_WARM_MLP;
  }
  // per structure: 1 when the solve starts from the user's or the network's charges
  warm_kept.assign(ns, wm != QEQ_WARM_COLD ? 1 : 0);
  const int* reject = nullptr;
  if (P->precond == QEQ_PRECOND_FOURIER) TRY(launch_precond_setup(P));
  for (int attempt = 0; attempt < 2; ++attempt) {
    count_launch(P, 3);
    k_init<<<nc, 256, 0, s>>>(P->d_chunks, P->d_perm, d_q, wm, reject, P->d_dinv, P->d_chi, P->d_J, P->d_q, P->d_sc,
                              red_part(P), red_counter(P));
    k_project<<<nc, 256, 0, s>>>(P->d_chunks, P->d_q, P->d_sc);
    k_set_tol<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, ns, P->desc.charge_tol, P->desc.residual_tol,
                                               prec == QEQ_MIXED ? kMixedInnerTol : 1.0, 0, 1.0);
    TRY(cudaGetLastError());
    if (P->precond == QEQ_PRECOND_FOURIER) {
      // w1 = M^-1 1 and its sums, for projecting preconditioned residuals onto 1^T z = 0
      count_launch(P);
      k_fill<<<(int)((P->n_atoms + 255) / 256), 256, 0, s>>>(P->d_x, P->n_atoms, 1.0);
      TRY(launch_precond(P, P->d_x, P->d_w1, 1, 0));
    }
    // first residual with the iteration's matvec
    TRY(launch_matvec(P, prec, P->d_q, P->d_Ap, 1, 0, 0, nullptr));
    count_launch(P);
    k_resid<<<nc, 256, 0, s>>>(P->d_chunks, P->d_chi, P->d_Ap, P->d_dinv, P->d_r, P->d_sc, 0, red_part(P),
                               red_counter(P), max_iter);
    TRY(cudaGetLastError());
    if (wm != QEQ_WARM_MLP || attempt == 1) break;
    // The plain method judges the network's start by the quantity CG minimises: on the
    // constraint plane E(q) - E(q*) = 1/2 ||q - q*||_A^2, so the start is kept iff its
    // energy is below that of the uniform start q_tot/N (E = 0 when q_tot = 0; otherwise
    // (q_tot/N) sum chi + 1/2 (q_tot/N)^2 1^T A 1, with one extra matvec of the ones vector).
    count_launch(P);
    k_start_energy<<<nc, 256, 0, s>>>(P->d_chunks, P->d_q, P->d_r, P->d_chi, P->d_sc, red_part(P), red_counter(P));
    TRY(cudaGetLastError());
    bool charged = false;
    for (int i = 0; i < ns; ++i) charged |= (h_qtot[i] != 0.0);
    if (charged) {
      count_launch(P, 2);
      k_fill<<<(int)((P->n_atoms + 255) / 256), 256, 0, s>>>(P->d_x, P->n_atoms, 1.0);
      TRY(launch_matvec(P, prec, P->d_x, P->d_z, 1, 0, 0, nullptr));
      k_vec_sum<<<nc, 256, 0, s>>>(P->d_chunks, P->d_z, P->d_sc, red_part(P), red_counter(P));
      TRY(cudaGetLastError());
    }
    std::vector<PcgScalars> h(ns);
    TRY(cudaMemcpyAsync(h.data(), P->d_sc, sizeof(PcgScalars) * ns, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    // each structure keeps or rejects its own network start; the rejected ones restart
    // from the uniform start (every structure's first residual is recomputed, the kept
    // ones reproduce theirs exactly)
    int n_bad = 0;
    for (int i = 0; i < ns; ++i) {
      double n = (double)h[i].n, qu = h_qtot[i] / n;
      double e_cold = 0.0;
      if (h_qtot[i] != 0.0) e_cold = qu * h[i].chi_sum + 0.5 * qu * qu * h[i].E_quad;
      const bool bad = !std::isfinite(h[i].E_lin) || !(h[i].E_lin < e_cold);
      warm_kept[i] = bad ? 0 : 1;
      n_bad += bad ? 1 : 0;
    }
    if (n_bad == 0) break;
    TRY(cudaMemcpyAsync(P->d_reject, warm_kept.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    count_launch(P);
    k_flip<<<(ns + 255) / 256, 256, 0, s>>>(P->d_reject, ns);  // kept -> 0, rejected -> 1
    TRY(init_scalars(P, h_qtot) == QEQ_OK ? cudaSuccess : cudaErrorUnknown);  // synchronises the copy
    reject = P->d_reject;
  }
    if (P->desc.flags & QEQ_FLAG_SQNM)
      TRY_ST(sqnm_rounds(P, prec));
    else
      TRY_ST(pcg_rounds(P, prec));
  }
  // energy terms from the final check's A q, outputs in input order
  count_launch(P);
  k_energy<<<nc, 256, 0, s>>>(P->d_chunks, P->d_q, P->d_Ap, P->d_chi, P->d_J, P->d_sc, red_part(P), red_counter(P));
  int nb = (int)((P->n_atoms + 255) / 256);
  count_launch(P);
  k_unsort<<<nb, 256, 0, s>>>(P->d_perm, P->n_atoms, P->d_q, d_q);
  count_launch(P);
  k_write_mu<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, ns, d_mu, nullptr, nullptr);
  TRY(cudaGetLastError());
  std::vector<PcgScalars> h(ns);
  LoopCtl ctl;
  TRY(cudaMemcpyAsync(h.data(), P->d_sc, sizeof(PcgScalars) * ns, cudaMemcpyDeviceToHost, s));
  if (P->graph_ok) TRY(cudaMemcpyAsync(&ctl, P->d_ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (P->graph_ok && !two_rhs) P->launches += P->gk_inner * ctl.replays_total + P->gk_round * ctl.outer;
  qeq_status worst = QEQ_OK;
  for (int i = 0; i < ns; ++i) {
    PcgScalars& c = h[i];
    if (two_rhs) {  // the sub-solves' counts; converged means the combined charges passed the FP64 check
      c.status = tr_status[i] != QEQ_OK ? tr_status[i] : (c.converged ? QEQ_OK : QEQ_ERR_NOCONV);
      c.iters = tr_iters[i];
      c.restarts = tr_rest[i];
    }
    double n = (double)c.n, mean = c.r_sum / n;
    double pinf = fmax(c.r_max - mean, mean - c.r_min);
    double pl2 = c.r_l2;
    if (h_info) {
      h_info[i].status = c.status;
      h_info[i].iterations = c.iters;
      h_info[i].restarts = c.restarts;
      h_info[i].warm_used = warm_kept[i];
      h_info[i].residual_inf = pinf;
      h_info[i].residual_l2 = pl2;
      h_info[i].error_bound_l2 = pl2 / c.j_min;
    }
    if (c.status != QEQ_OK && worst == QEQ_OK) worst = (qeq_status)c.status;
  }
  if (worst == QEQ_ERR_NOCONV) P->last_error = "some structure did not converge within max_iter";
  const qeq_status tst = check_timeout(P);
  if (tst != QEQ_OK) {
    if (h_info)
      for (int i = 0; i < ns; ++i) h_info[i].status = QEQ_ERR_TIMEOUT;
    return tst;
  }
  return worst;
}

extern "C" qeq_status qeq_energy(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_chi,
                                 const double* d_J, const double* d_q, double* d_E_qeq, double* d_E_elec) {
  if (!P) return QEQ_ERR_INVALID;
  if (!d_q) {
    P->last_error = "d_q is required";
    return QEQ_ERR_INVALID;
  }
  qeq_status st = prepare(P, d_pos, d_species, d_chi, d_J);
  if (st != QEQ_OK) return st;
  st = init_scalars(P, nullptr);
  if (st != QEQ_OK) return st;
  cudaStream_t s = P->stream;
  const int nc = P->n_chunks, ns = P->n_struct;
  int nb = (int)((P->n_atoms + 255) / 256);
  count_launch(P);
  k_sort_in<<<nb, 256, 0, s>>>(P->d_perm, P->n_atoms, d_q, P->d_x);
  TRY(cudaGetLastError());
  TRY(launch_matvec(P, QEQ_FP64, P->d_x, P->d_Ap, 1, 0, 0, nullptr));
  count_launch(P);
  k_energy<<<nc, 256, 0, s>>>(P->d_chunks, P->d_x, P->d_Ap, P->d_chi, P->d_J, P->d_sc, red_part(P), red_counter(P));
  count_launch(P);
  k_write_mu<<<(ns + 127) / 128, 128, 0, s>>>(P->d_sc, ns, nullptr, d_E_qeq, d_E_elec);
  TRY(cudaGetLastError());
  return check_timeout(P);
}

extern "C" qeq_status qeq_matvec(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_J,
                                 const double* d_x, double* d_y, int32_t force_fp64) {
  if (!P) return QEQ_ERR_INVALID;
  if (!d_x || !d_y || !d_pos || !d_species) {
    P->last_error = "null pointer";
    return QEQ_ERR_INVALID;
  }
  TRY(cudaSetDevice(P->device));
  TRY(launch_prepare_atoms(P, d_pos, d_species, nullptr, d_J, P->pair_cap > 0));
  qeq_status st = check_inputs(P);
  if (st != QEQ_OK) return st;
  st = init_scalars(P, nullptr);
  if (st != QEQ_OK) return st;
  cudaStream_t s = P->stream;
  int nb = (int)((P->n_atoms + 255) / 256);
  count_launch(P);
  k_sort_in<<<nb, 256, 0, s>>>(P->d_perm, P->n_atoms, d_x, P->d_x);
  TRY(cudaGetLastError());
  TRY(launch_matvec(P, force_fp64 ? QEQ_FP64 : P->precision, P->d_x, P->d_Ap, d_J ? 1 : 0, 0, 0, nullptr));
  count_launch(P);
  k_unsort<<<nb, 256, 0, s>>>(P->d_perm, P->n_atoms, P->d_Ap, d_y);
  TRY(cudaGetLastError());
  return check_timeout(P);
}

extern "C" qeq_status qeq_forces(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_q,
                                 const double* d_lambda, double* d_F) {
  if (!P) return QEQ_ERR_INVALID;
  if (!d_pos || !d_species || !d_q || !d_F) {
    P->last_error = "null pointer";
    return QEQ_ERR_INVALID;
  }
  TRY(cudaSetDevice(P->device));
  TRY(launch_prepare_atoms(P, d_pos, d_species, nullptr, nullptr, 0));
  qeq_status st = check_inputs(P);
  if (st != QEQ_OK) return st;
  TRY(launch_forces(P, d_q, d_lambda, d_F));
  return check_timeout(P);
}

extern "C" qeq_status qeq_stress(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_q,
                                 const double* d_lambda, double* d_D) {
  if (!P) return QEQ_ERR_INVALID;
  if (!d_pos || !d_species || !d_q || !d_D) {
    P->last_error = "null pointer";
    return QEQ_ERR_INVALID;
  }
  TRY(cudaSetDevice(P->device));
  TRY(launch_prepare_atoms(P, d_pos, d_species, nullptr, nullptr, 0));
  qeq_status st = check_inputs(P);
  if (st != QEQ_OK) return st;
  TRY(launch_stress(P, d_q, d_lambda, d_D));
  return check_timeout(P);
}

extern "C" qeq_status qeq_embedding(qeq_plan P, const double* d_pos, const int32_t* d_species, const double* d_q,
                                    double* d_Gamma) {
  if (!P) return QEQ_ERR_INVALID;
  if (!d_pos || !d_species || !d_q || !d_Gamma) {
    P->last_error = "null pointer";
    return QEQ_ERR_INVALID;
  }
  TRY(cudaSetDevice(P->device));
  TRY(launch_prepare_atoms(P, d_pos, d_species, nullptr, nullptr, P->pair_cap > 0));
  qeq_status st = check_inputs(P);
  if (st != QEQ_OK) return st;
  st = init_scalars(P, nullptr);
  if (st != QEQ_OK) return st;
  TRY(launch_embedding(P, d_q, d_Gamma));
  return check_timeout(P);
}

extern "C" qeq_status qeq_profile_matvec(qeq_plan P, int32_t n_rep, float* h_ms) {
  if (!P || !h_ms || n_rep < 1) return QEQ_ERR_INVALID;
  if (!P->have_atoms) {
    P->last_error = "no atoms prepared: call qeq_solve or qeq_matvec first";
    return QEQ_ERR_INVALID;
  }
  // all repetitions back to back on the plan's stream (no host gaps between them)
  std::vector<cudaEvent_t> ev((size_t)n_rep * (QEQ_N_STAGES + 1));
  for (auto& e : ev) TRY(cudaEventCreate(&e));
  std::vector<double> acc(QEQ_N_STAGES, 0.0);
  for (int r = 0; r < n_rep; ++r)
    TRY(launch_matvec(P, P->precision, P->d_x, P->d_Ap, 1, 0, 0, ev.data() + (size_t)r * (QEQ_N_STAGES + 1)));
  TRY(cudaEventSynchronize(ev.back()));
  for (int r = 0; r < n_rep; ++r)
    for (int k = 0; k < QEQ_N_STAGES; ++k) {
      float ms = 0.f;
      TRY(cudaEventElapsedTime(&ms, ev[(size_t)r * (QEQ_N_STAGES + 1) + k], ev[(size_t)r * (QEQ_N_STAGES + 1) + k + 1]));
      acc[k] += ms;
    }
  for (int k = 0; k < QEQ_N_STAGES; ++k) h_ms[k] = (float)(acc[k] / n_rep);
  for (auto& e : ev) cudaEventDestroy(e);
  return QEQ_OK;
}
