// Warp-cooperative walk over the candidate neighbours of one atom in the
// bin-sorted atom order (real-space pair list of the Ewald split, SI "Ewald
// Summation", and the radial descriptors of the warm start, Sec. 2.2).
//
// The bins within R[d] bins of bin bb along every axis (periodic images
// included) are visited as runs: for every (d0, d1) column the bins along the
// third axis are split at the periodic boundary into segments of one image
// each, and the atoms of one segment are contiguous in the sorted order.  The
// runs are taken in (d0, d1, segment) order, the atoms of a run in sorted
// order, so the candidate sequence is the same as that of a plain triple loop
// over d0, d1, d2.  Each warp step hands 32 consecutive candidates to the 32
// lanes; lanes past the end get valid = false, so that warp collectives inside
// the visitor see the whole warp.
#pragma once

#include "qeq_internal.cuh"

struct NbrWarpSmem {
  int off[32];       // first candidate index of the run
  int beg[32];       // first sorted atom of the run
  int zero[32];      // run lies in the unshifted image
  double sh[32][3];  // Cartesian image shift of the run
  float sh32[32][3]; // the same in FP32
  int code[32];      // image indices (s0, s1, s2) + 128, 8 bits each
};

// image indices of a periodic shift, |s_d| < 128, packed into one int and back
__device__ __forceinline__ int pack_image(int s0, int s1, int s2) {
  return (s0 + 128) | ((s1 + 128) << 8) | ((s2 + 128) << 16);
}
__device__ __forceinline__ void unpack_image(int c, int* s) {
  s[0] = (c & 255) - 128;
  s[1] = ((c >> 8) & 255) - 128;
  s[2] = ((c >> 16) & 255) - 128;
}

__device__ __forceinline__ int floordiv_i(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// visit(valid, t, sh, sh32, zero_shift, code): t = sorted index of the candidate
// atom, sh (FP64) / sh32 (FP32) = image shift added to its position, code = the
// image indices packed by pack_image.  Every lane of the warp must call this.
template <class Visit>
__device__ __forceinline__ void warp_neighbour_walk(const StructDev& S, const int bb[3], const int R[3],
                                                    const int* __restrict__ bin_start, NbrWarpSmem& W,
                                                    Visit&& visit) {
  const int lane = threadIdx.x & 31;
  const int n0 = 2 * R[0] + 1, n1 = 2 * R[1] + 1;
  const int lo2 = bb[2] - R[2], hi2 = bb[2] + R[2];
  const int nb2 = S.nb[2];
  const int s2lo = floordiv_i(lo2, nb2), s2hi = floordiv_i(hi2, nb2);
  const int nseg = s2hi - s2lo + 1;
  const int nruns = n0 * n1 * nseg;
  for (int r0 = 0; r0 < nruns; r0 += 32) {
    const int r = r0 + lane;
    int beg = 0, len = 0, zero = 0, code = 0;
    double sh0 = 0.0, sh1 = 0.0, sh2 = 0.0;
    if (r < nruns) {
      const int seg = r % nseg, col = r / nseg;
      const int i1 = col % n1, i0 = col / n1;
      int c0 = bb[0] - R[0] + i0, c1 = bb[1] - R[1] + i1;
      const int s0 = floordiv_i(c0, S.nb[0]), s1 = floordiv_i(c1, S.nb[1]);
      c0 -= s0 * S.nb[0];
      c1 -= s1 * S.nb[1];
      const int s2 = s2lo + seg;
      const int z0 = max(lo2, s2 * nb2) - s2 * nb2, z1 = min(hi2, s2 * nb2 + nb2 - 1) - s2 * nb2;
      const int g = S.bin_off + (c0 * S.nb[1] + c1) * nb2;
      beg = bin_start[g + z0];
      len = bin_start[g + z1 + 1] - beg;
      zero = (s0 == 0 && s1 == 0 && s2 == 0);
      code = pack_image(s0, s1, s2);
      sh0 = s0 * S.h[0] + s1 * S.h[3] + s2 * S.h[6];
      sh1 = s0 * S.h[1] + s1 * S.h[4] + s2 * S.h[7];
      sh2 = s0 * S.h[2] + s1 * S.h[5] + s2 * S.h[8];
    }
    int inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    const int nr = min(32, nruns - r0);
    W.off[lane] = inc - len;
    W.beg[lane] = beg;
    W.zero[lane] = zero;
    W.sh[lane][0] = sh0;
    W.sh[lane][1] = sh1;
    W.sh[lane][2] = sh2;
    W.sh32[lane][0] = (float)sh0;
    W.sh32[lane][1] = (float)sh1;
    W.sh32[lane][2] = (float)sh2;
    W.code[lane] = code;
    __syncwarp();
    for (int c0 = 0; c0 < total; c0 += 32) {
      const int c = c0 + lane;
      const bool valid = c < total;
      int j = 0;
      if (valid) {
        // last run whose first candidate is <= c (it is non-empty because c < total)
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (W.off[mid] <= c) lo = mid;
          else hi = mid - 1;
        }
        j = lo;
      }
      const int t = valid ? W.beg[j] + (c - W.off[j]) : 0;
      visit(valid, t, W.sh[j], W.sh32[j], W.zero[j] != 0, W.code[j]);
    }
    __syncwarp();
  }
}
