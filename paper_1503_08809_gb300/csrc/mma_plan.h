// mma_plan.h -- schedules of the slice products of the tensor-core form as
// runs of tcgen05 MMAs (host code of tc.cu; plain C++ without CUDA, so the
// CPU tests compile it and check its invariants).
//
// One 16-deep K step of a tile multiplies every A slice sa with the B slices
// sb = 0 .. MAXLEV - sa.  B slices lie w rows apart in shared memory, so a run
// of n consecutive sb is one MMA with N = n w (at most 256) whose result
// columns fall on n consecutive accumulators spaced w TMEM columns apart.
// Accumulator 0 takes level 0 (sa + sb = 0) and 1 takes level 1 -- both exact
// integer sums in FP32 -- and 2, 3, ... take levels >= 2, which the drain adds
// up; the drain reads accumulators 0 .. used - 1 (used is 4 or 5), so a
// schedule must write every one of them.  In a chunk the first MMA on an
// accumulator overwrites it, so a run touches only fresh or only used
// accumulators.  Of the schedules that fit in 512 TMEM columns the search
// keeps the one of least issue cost, an MMA (M = 128, K = 16) costed at
// max(80, N / 2) clocks -- the rate measured for back-to-back MMAs from one
// thread, flat up to N = 160.
//
// Run word: sa (bits 0-3), first sb (4-7), n (8-11), first accumulator
// (12-15), fresh flag (16).  Header word: runs (bits 0-7), accumulators
// used (bits 8-15).
#pragma once
#include <cstdint>
#include <cstring>

namespace modal {
namespace plan {

constexpr int SLICES = 5;     // BF16 slices per operand
constexpr int MAXLEV = 4;     // products with sa + sb <= MAXLEV
constexpr int RUNS_MAX = 16;  // runs per schedule
constexpr int MIN_ACC = 4;    // accumulators the drain always reads

struct Search {
  int w, nacc, R;
  double best = 1e30;
  uint32_t best_plan[RUNS_MAX];
  int best_n = 0, best_used = 0;
  uint32_t cur[RUNS_MAX];
  void rec(int sa, int sb, unsigned fresh, double cost, int n, int used) {
    if (cost >= best || n > RUNS_MAX) return;
    if (sa == SLICES) {
      // every accumulator the drain reads must have been written
      const unsigned touched = ~fresh & ((1u << nacc) - 1u);
      if (used < MIN_ACC || touched != (1u << used) - 1u) return;
      best = cost;
      best_n = n;
      best_used = used;
      memcpy(best_plan, cur, sizeof cur);
      return;
    }
    const int nb = MAXLEV - sa + 1;
    if (sb >= nb) return rec(sa + 1, 0, fresh, cost, n, used);
    if (n == RUNS_MAX) return;
    for (int len = (R < nb - sb ? R : nb - sb); len >= 1; --len) {
      const int L = sa + sb;
      const int lo = L < 2 ? L : 2, hi = L < 2 ? L : nacc - len;
      for (int a0 = lo; a0 <= hi; ++a0) {
        if (a0 + len > nacc) continue;
        bool ok = true, allf = true, nonef = true;
        for (int t = 0; t < len; ++t) {
          const int a = a0 + t, lv = L + t;
          if (!((a >= 2 && lv >= 2) || a == lv)) ok = false;
          const bool f = (fresh >> a) & 1u;
          allf = allf && f;
          nonef = nonef && !f;
        }
        if (!ok || !(allf || nonef)) continue;
        const unsigned mask = ((1u << len) - 1u) << a0;
        const double c = (len * w / 2.0 > 80.0) ? len * w / 2.0 : 80.0;
        cur[n] = (uint32_t)sa | (uint32_t)sb << 4 | (uint32_t)len << 8 | (uint32_t)a0 << 12 |
                 (allf ? 1u << 16 : 0u);
        rec(sa, sb + len, fresh & ~mask, cost + c, n + 1, used > a0 + len ? used : a0 + len);
      }
    }
  }
};

// One MMA per product: levels 0, 1, 2 on accumulators 0, 1, 2 and levels 3
// and 4 on accumulator 3 -- always valid (4 x w <= 512 for w <= 128).
inline void singles_plan(uint32_t (&out)[1 + RUNS_MAX]) {
  memset(out, 0, sizeof out);
  int n = 0;
  for (int sa = 0; sa < SLICES; ++sa)
    for (int sb = 0; sa + sb <= MAXLEV; ++sb) {
      const int L = sa + sb, acc = L < 3 ? L : 3;
      // the first product on each accumulator (in this order: sa = 0) overwrites it
      const bool fresh = sa == 0 && sb <= 3;
      out[1 + n++] = (uint32_t)sa | (uint32_t)sb << 4 | 1u << 8 | (uint32_t)acc << 12 | (fresh ? 1u << 16 : 0u);
    }
  out[0] = (uint32_t)n | (uint32_t)MIN_ACC << 8;
}

// Schedule of the 2-SM (CTA pair) form.  The pair's MMA takes the columns
// 0 .. N/2-1 of B from the even CTA's shared memory and N/2 .. N-1 from the
// odd CTA's, at the same offsets.  The odd CTA holds the B slices shifted by
// one (its slot j holds slice j + 1; slot 4 holds zeros), so an MMA with
// N = 2w at slot j multiplies the A slice by B slices j and j + 1 at once:
// a run of exactly two, whose columns fall on accumulators acc and acc + 1.
// Nine such runs cover the 15 products with sa + sb <= 4; three of them pair
// a wanted product with the zero slot or with a level-5 product (which only
// adds a smaller term to an accumulator of levels >= 2).  Accumulators: 0 =
// level 0, 1 = level 1 (exact), 2 and 3 = levels >= 2.  The two fresh runs
// come first (the first touch of an accumulator in a chunk overwrites it).
constexpr int PAIR_RUNS = 9;
inline void pair_plan(uint32_t (&out)[1 + RUNS_MAX]) {
  static const int runs[PAIR_RUNS][4] = {  // sa, slot j, first accumulator, fresh
      {0, 2, 2, 1}, {0, 0, 0, 1}, {1, 0, 1, 0}, {0, 4, 2, 0}, {1, 2, 2, 0},
      {2, 0, 2, 0}, {2, 2, 2, 0}, {3, 0, 2, 0}, {4, 0, 2, 0}};
  memset(out, 0, sizeof out);
  for (int r = 0; r < PAIR_RUNS; ++r)
    out[1 + r] = (uint32_t)runs[r][0] | (uint32_t)runs[r][1] << 4 | 2u << 8 | (uint32_t)runs[r][2] << 12 |
                 (runs[r][3] ? 1u << 16 : 0u);
  out[0] = (uint32_t)PAIR_RUNS | (uint32_t)MIN_ACC << 8;
}

// The schedule of least modelled cost for tile width w (a multiple of 16,
// 16 .. 128); the singles schedule if the search finds none.
inline void mma_plan(int w, uint32_t (&out)[1 + RUNS_MAX]) {
  Search ps;
  ps.w = w;
  ps.nacc = 512 / w < 15 ? 512 / w : 15;
  ps.R = 256 / w < SLICES ? 256 / w : SLICES;
  ps.rec(0, 0, (1u << ps.nacc) - 1u, 0.0, 0, 0);
  if (ps.best_n == 0) return singles_plan(out);
  memset(out, 0, sizeof out);
  out[0] = (uint32_t)ps.best_n | (uint32_t)ps.best_used << 8;
  for (int r = 0; r < ps.best_n; ++r) out[1 + r] = ps.best_plan[r];
}

}  // namespace plan
}  // namespace modal
