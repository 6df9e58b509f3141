// Host check of the index helpers of common.cuh: the pair index {u, v} <->
// uv round trip for bases up to 64 functions, and the triple-product layout
// GLayout in both of its forms (one expansion of the permanent throughout,
// and the split one) -- blocks laid end to end, index() a bijection onto
// [0, size()), checked_index() rejecting every out-of-range argument, the
// entry of (a <= b <= c, uv, t) lying in the row of its Y pair and the
// column of its M row, and the Y pairs listed once each, block by block.
// Prints violations; exit 1 if any.
#include <math.h>
#include <cstdio>
#include <vector>

#include "../paper_1503_08809_gb300/csrc/common.cuh"

using namespace modal;

int main() {
  long bad = 0;
  for (int v = 0; v < 64; ++v)
    for (int u = 0; u <= v; ++u) {
      const int uv = pair_index(u, v);
      int uu, vv;
      pair_decode(uv, uu, vv);
      if (uv != v * (v + 1) / 2 + u || pair_index(v, u) != uv || uu != u || vv != v) {
        if (bad++ < 5) printf("pair %d %d -> %d -> %d %d\n", u, v, uv, uu, vv);
      }
    }
  const int sizes[][2] = {{1, 1}, {1, 5}, {3, 2}, {5, 4}, {7, 3}, {6, 6}, {8, 2}};
  for (int split = 0; split < 2; ++split)
  for (auto &sz : sizes) {
    const GLayout g = split ? make_glayout_split(sz[0], sz[1]) : make_glayout(sz[0], sz[1]);
    // Y pairs: block by block, each pair the block's rows need exactly once
    {
      int j = 0;
      for (int b = 0; b < g.nbl; ++b) {
        if (g.ypair0(b) != j && bad++ < 5) printf("ypair0 %d\n", b);
        for (int i = 0; i < g.ypairs(b); ++i, ++j) {
          int x, y;
          g.y_pair(j, x, y);
          const bool ok = g.first(b) ? (x == i && y == b) : (x == b && y == b + i);
          if (!ok && bad++ < 5) printf("y_pair %d -> %d %d (block %d)\n", j, x, y, b);
        }
        if (g.rows(b) != (int64_t)g.ypairs(b) * g.P2 && bad++ < 5) printf("rows %d\n", b);
      }
      if (g.ypairs_total() != j && bad++ < 5) printf("ypairs_total\n");
      if (!split && j != g.nbl * (g.nbl + 1) / 2 && bad++ < 5) printf("all pairs\n");
    }
    int64_t off = 0;
    for (int b = 0; b < g.nbl; ++b) {
      if (g.offset(b) != off && bad++ < 5) printf("offset %d\n", b);
      off += g.rows(b) * g.cols(b);
    }
    if (g.size() != off && bad++ < 5) printf("size\n");
    std::vector<int> hit((size_t)g.size(), 0);
    for (int a = -1; a <= g.nbl; ++a)
      for (int b = -1; b <= g.nbl; ++b)
        for (int c = -1; c <= g.nbl; ++c)
          for (int uv = -1; uv <= g.P2; ++uv)
            for (int t = -1; t <= g.nbp; ++t) {
              const bool valid = a >= 0 && a <= b && b <= c && c < g.nbl && uv >= 0 && uv < g.P2 && t >= 0 &&
                                 t < g.nbp;
              const int64_t i = g.checked_index(a, b, uv, c, t);
              if (!valid) {
                if (i != -1 && bad++ < 5) printf("accepted %d %d %d %d %d\n", a, b, uv, c, t);
                continue;
              }
              if (i < 0 || i >= g.size()) {
                if (bad++ < 5) printf("out of range %d %d %d %d %d\n", a, b, uv, c, t);
                continue;
              }
              // its row holds the Y pair of the expansion, its column the M row
              const int64_t rel = i - g.offset(b), row = rel / g.cols(b), col = rel % g.cols(b);
              int x, y;
              g.y_pair(g.ypair0(b) + (int)(row / g.P2), x, y);
              const int mrow = (int)((g.colstart(b) + col) / g.nbp), mt = (int)((g.colstart(b) + col) % g.nbp);
              const bool ok = row % g.P2 == uv && mt == t &&
                              (g.first(b) ? (x == a && y == b && mrow == c) : (x == b && y == c && mrow == a));
              if (!ok && bad++ < 5) printf("entry of %d %d %d %d %d misplaced\n", a, b, uv, c, t);
              hit[(size_t)i]++;
            }
    for (size_t i = 0; i < hit.size(); ++i)
      if (hit[i] != 1 && bad++ < 5) printf("entry %zu hit %d times (nbl %d nbp %d)\n", i, hit[i], g.nbl, g.nbp);
  }
  printf("%ld violations\n", bad);
  return bad ? 1 : 0;
}
