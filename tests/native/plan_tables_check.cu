// Host check of the plan tables the matvec kernels index with (csrc/qeq_internal.cuh:
// fft_radices, fft_plan_fill, make_fastdiv, brick_candidates, fft_work_lists).  For every
// mesh length the plan can choose (2^a 3^b 5^c up to 1024) and both radix limits (FP32 and
// FP64 passes):
//   * the stage radices are register radices no larger than the limit, their product is
//     K, there are at most QEQ_MAX_STAGES of them, and no ordered factorisation with
//     fewer stages exists (brute force over the same radix set);
//   * the stage constants satisfy Q_s L_s = K, S_s R_s = L_s, Q_{s+1} = Q_s R_s;
//   * the frequency table (block-order position -> frequency) and the position table
//     (frequency -> position) are inverse permutations of 0 .. K-1, and every block
//     offset lies inside the line;
//   * the division (mulhi(n, m) + n) >> s with make_fastdiv's (m, s) equals n / d for
//     every divisor the plans carry, exhaustively for n < 2^22 (the kernels divide
//     indices of one shared-memory tile, far below that) and on seeded samples up to
//     2^31 - 1.
// For every such length and B-spline order 4, 6, 8, each spread brick's candidate bins
// hold, without repeats, every bin whose atoms (stencil base f, points f - p + 1 .. f mod K,
// bin f / 8) reach the brick (brute force over f).  For the FFT work lists of a set of
// mesh shapes and line counts: every z, y and inverse-y line is covered exactly once, and
// every x line (y, z) exactly once as itself or as its mirror (-y, -z) of an x item.
// For the preconditioner's coarse-spread tiles (pre_tile_range) over pairs of fine and
// coarse lengths and group sizes: the tile start lies on the coarse line, its extent is at
// most the line, and the cubic stencils (points f - 3 .. f) of every coarse base f that an
// atom of the group's fine bins can have, widened by one point each way for the rounding
// of its coordinate, lie in the tile.
// Prints a summary and exits non-zero on the first violated property.
#include <cstdio>
#include <cstdint>
#include <random>
#include <set>
#include <vector>

#include "../../paper_2607_17978_b300/csrc/qeq_internal.cuh"

static bool smooth(int n) {
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

// fewest stages of any ordered factorisation of k into the radices {2..24} allowed by maxR
static int min_stages(int k, int maxR) {
  static const int kR[] = {24, 20, 18, 16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  std::vector<int> best(k + 1, 1 << 20);
  best[1] = 0;
  for (int v = 2; v <= k; ++v)
    for (int r : kR)
      if (r <= maxR && v % r == 0 && best[v / r] + 1 < best[v]) best[v] = best[v / r] + 1;
  return best[k];
}

static uint32_t div_magic(uint32_t n, const FastDiv& f) {
  const uint32_t hi = (uint32_t)(((uint64_t)n * f.m) >> 32);
  return (hi + n) >> f.s;
}

// every base position whose stencil reaches a brick has its bin among the candidates
static bool check_bricks(int K, int p) {
  StructDev T{};
  T.K[0] = T.K[1] = T.K[2] = K;
  const int nbins = (K + QEQ_BIN - 1) / QEQ_BIN;
  for (int d = 0; d < 3; ++d) {
    const int e = (d == 2) ? QEQ_BRICK_Z : QEQ_BRICK_XY;
    for (int b = 0; b * e < K; ++b) {
      int bc[3] = {0, 0, 0};
      bc[d] = b;
      int out[QEQ_BRICK_CAND];
      brick_candidates(T, p, bc, out);
      const int nc = out[d];
      const int* cand = out + 4 + 8 * d;
      if (nc < 1 || nc > 8) return false;
      for (int i = 0; i < nc; ++i) {
        if (cand[i] < 0 || cand[i] >= nbins) return false;
        for (int j = 0; j < i; ++j)
          if (cand[j] == cand[i]) return false;  // a repeated bin would spread its atoms twice
      }
      const int x0 = b * e, x1 = std::min(x0 + e, K);
      for (int f = 0; f < K; ++f) {
        bool reaches = false;
        for (int j = 0; j < p; ++j) {
          const int x = ((f - j) % K + K) % K;
          reaches |= (x >= x0 && x < x1);
        }
        if (!reaches) continue;
        bool found = false;
        for (int i = 0; i < nc; ++i) found |= (cand[i] == f / QEQ_BIN);
        if (!found) {
          printf("FAIL bricks K=%d p=%d d=%d brick %d: bin %d of base %d missing\n", K, p, d, b, f / QEQ_BIN, f);
          return false;
        }
      }
    }
  }
  return true;
}

static bool check_work_lists(int K0, int K1, int K2, int ncm, int tl, int tlx) {
  StructDev T{};
  T.K[0] = K0;
  T.K[1] = K1;
  T.K[2] = K2;
  T.ncm = ncm;
  std::vector<int> z((size_t)ncm * K0 * K1), y((size_t)ncm * K2 * K0), yi((size_t)ncm * K0 * K2), x((size_t)K1 * K2);
  bool ok = true;
  fft_work_lists(
      T, 0, tl, tlx,
      [&](int4 it) {  // {s, c, x, y0}: lines y0 .. y0 + tl - 1 of column x
        for (int l = 0; l < tl && it.w + l < K1; ++l) z[((size_t)it.y * K0 + it.z) * K1 + it.w + l]++;
      },
      [&](int4 it) {  // {s, c, z, x0}
        for (int l = 0; l < tl && it.w + l < K0; ++l) y[((size_t)it.y * K2 + it.z) * K0 + it.w + l]++;
      },
      [&](int4 it) {  // {s, c, x, z0}
        for (int l = 0; l < tl && it.w + l < K2; ++l) yi[((size_t)it.y * K0 + it.z) * K2 + it.w + l]++;
      },
      [&](int4 it) {  // {s, z, y0, lines}: lines (y, z) and their mirrors (-y, -z)
        if (it.w < 1 || it.w > tlx || it.z + it.w > K1 || 2 * it.y > K2) ok = false;
        for (int l = 0; l < it.w; ++l) {
          const int yy = it.z + l, my = (K1 - yy) % K1, mz = (K2 - it.y) % K2;
          x[(size_t)yy * K2 + it.y]++;
          if (my != yy || mz != it.y) x[(size_t)my * K2 + mz]++;
        }
      });
  for (int v : z) ok &= (v == 1);
  for (int v : y) ok &= (v == 1);
  for (int v : yi) ok &= (v == 1);
  for (int v : x) ok &= (v == 1);
  if (!ok) printf("FAIL work lists K=(%d,%d,%d) ncm=%d tl=%d tlx=%d\n", K0, K1, K2, ncm, tl, tlx);
  return ok;
}

static bool check_pre_tiles(int Kf, int Kc, int g) {
  const int nb = (Kf + QEQ_BIN - 1) / QEQ_BIN;
  for (int b0 = 0; b0 < nb; b0 += g) {
    int o, ext;
    pre_tile_range(b0, g, nb, Kc, Kf, o, ext);
    if (o < 0 || o >= Kc || ext < 1 || ext > Kc) return false;
    const int b1 = std::min(b0 + g, nb);
    // coordinates u in [8 b0 / Kf, min(8 b1, Kf) / Kf): coarse bases floor(u Kc), +-1
    const int lo = (int)(((long long)QEQ_BIN * b0 * Kc) / Kf) - 1;
    const int hi = (int)(((long long)std::min(QEQ_BIN * b1, Kf) * Kc + Kf - 1) / Kf);  // largest base + 1
    for (int f = lo; f <= hi; ++f)
      for (int j = 0; j < 4; ++j) {
        const int x = (((f - j) % Kc) + Kc) % Kc;
        const int t = ((x - o) % Kc + Kc) % Kc;
        if (t >= ext) {
          printf("FAIL pre tiles Kf=%d Kc=%d g=%d b0=%d: point %d outside [%d, %d + %d)\n", Kf, Kc, g, b0, x, o, o,
                 ext);
          return false;
        }
      }
  }
  return true;
}

int main() {
  const int allowed[] = {2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24};
  std::set<uint32_t> divisors;
  int lengths = 0;
  for (int maxR : {24, QEQ_MAXR64}) {
    for (int K = 2; K <= 1024; ++K) {
      if (!smooth(K)) continue;
      ++lengths;
      const int K4 = (K + 3) & ~3;
      FftPlanDev f{};
      std::vector<double2> tw64(K);
      std::vector<float2> tw32(K);
      std::vector<int> tab(3 * K4, -1);
      if (!fft_plan_fill(K, f, tw64.data(), tw32.data(), tab.data(), maxR)) {
        printf("FAIL K=%d maxR=%d: no plan\n", K, maxR);
        return 1;
      }
      if (f.nst < 1 || f.nst > QEQ_MAX_STAGES || f.nst != min_stages(K, maxR)) {
        printf("FAIL K=%d maxR=%d: %d stages, fewest possible %d\n", K, maxR, f.nst, min_stages(K, maxR));
        return 1;
      }
      long long prod = 1;
      for (int s = 0; s < f.nst; ++s) {
        bool ok = false;
        for (int r : allowed) ok |= (f.radix[s] == r);
        if (!ok || f.radix[s] > maxR) {
          printf("FAIL K=%d maxR=%d: radix %d at stage %d\n", K, maxR, f.radix[s], s);
          return 1;
        }
        prod *= f.radix[s];
        if ((long long)f.Q[s] * f.L[s] != K || f.S[s] * f.radix[s] != f.L[s] ||
            (s + 1 < f.nst && f.Q[s + 1] != f.Q[s] * f.radix[s])) {
          printf("FAIL K=%d maxR=%d: stage constants at stage %d\n", K, maxR, s);
          return 1;
        }
        divisors.insert((uint32_t)(K / f.radix[s]));
        divisors.insert((uint32_t)f.S[s]);
        if (f.fnb[s].d != (uint32_t)(K / f.radix[s]) || f.fS[s].d != (uint32_t)f.S[s]) {
          printf("FAIL K=%d maxR=%d: divisor tables at stage %d\n", K, maxR, s);
          return 1;
        }
      }
      divisors.insert((uint32_t)K);
      if (prod != K || f.fK.d != (uint32_t)K) {
        printf("FAIL K=%d maxR=%d: radices multiply to %lld\n", K, maxR, prod);
        return 1;
      }
      const int* freq = tab.data() + K4;
      const int* pos = tab.data() + 2 * K4;
      std::vector<int> seen(K, 0);
      for (int p = 0; p < K; ++p) {
        const int fq = freq[p];
        if (fq < 0 || fq >= K || seen[fq]++ || pos[fq] != p) {
          printf("FAIL K=%d maxR=%d: frequency/position tables at %d\n", K, maxR, p);
          return 1;
        }
      }
      const int nblk = K / f.radix[f.nst - 1];
      for (int u = 0; u < nblk; ++u)
        if (tab[u] < 0 || tab[u] >= K) {
          printf("FAIL K=%d maxR=%d: block offset %d of base %d\n", K, maxR, tab[u], u);
          return 1;
        }
    }
  }
  std::mt19937_64 gen(20260);
  std::uniform_int_distribution<uint32_t> big(0, 0x7FFFFFFFu);
  for (uint32_t d : divisors) {
    const FastDiv f = make_fastdiv(d);
    for (uint32_t n = 0; n < (1u << 22); ++n)
      if (div_magic(n, f) != n / d) {
        printf("FAIL division: %u / %u gives %u\n", n, d, div_magic(n, f));
        return 1;
      }
    for (int t = 0; t < 200000; ++t) {
      const uint32_t n = (t == 0) ? 0x7FFFFFFFu : big(gen);
      if (div_magic(n, f) != n / d) {
        printf("FAIL division: %u / %u gives %u\n", n, d, div_magic(n, f));
        return 1;
      }
    }
  }
  int bricks = 0;
  for (int K = 12; K <= 1024; ++K) {
    if (!smooth(K)) continue;
    for (int p : {4, 6, 8}) {
      if (K < 2 * p) continue;
      if (!check_bricks(K, p)) {
        printf("FAIL bricks K=%d p=%d\n", K, p);
        return 1;
      }
      ++bricks;
    }
  }
  const int shapes[][3] = {{12, 12, 12}, {15, 16, 18}, {16, 20, 25}, {27, 30, 32}, {45, 40, 36}, {64, 64, 64},
                           {81, 75, 72}, {96, 100, 90}, {135, 128, 120}, {288, 288, 288}, {480, 480, 480},
                           {1000, 27, 1000}};
  int lists = 0;
  for (const auto& k : shapes)
    for (int ncm : {1, 2})
      for (int tl : {1, 8, 64})
        for (int tlx : {1, 4, 32}) {
          if (!check_work_lists(k[0], k[1], k[2], ncm, tl, tlx)) return 1;
          ++lists;
        }
  int tiles = 0;
  for (int Kf = 12; Kf <= 1000; ++Kf) {
    if (!smooth(Kf)) continue;
    for (int Kc = 4; Kc <= Kf; ++Kc) {
      if (!smooth(Kc)) continue;
      const int nb = (Kf + QEQ_BIN - 1) / QEQ_BIN;
      for (int g : {1, QEQ_PRE_TILE_G, 3, 5, nb}) {
        if (!check_pre_tiles(Kf, Kc, g)) return 1;
        ++tiles;
      }
    }
  }
  printf("plan tables: %d (length, radix limit) FFT plans, %zu divisors exact, %d (length, order) brick tables, "
         "%d work-list cases, %d coarse-tile cases: ok\n", lengths, divisors.size(), bricks, lists, tiles);
  return 0;
}
