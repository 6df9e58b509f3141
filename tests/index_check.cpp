// Host check of the index helpers of common.cuh: the pair index {u, v} <->
// uv round trip for bases up to 64 functions, and the triple-product layout
// GLayout -- blocks laid end to end, index() a bijection onto [0, size()),
// checked_index() rejecting every out-of-range argument.  Prints violations;
// exit 1 if any.
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
  const int sizes[][2] = {{1, 1}, {1, 5}, {3, 2}, {5, 4}, {7, 3}, {6, 6}};
  for (auto &sz : sizes) {
    const GLayout g = make_glayout(sz[0], sz[1]);
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
              hit[(size_t)i]++;
            }
    for (size_t i = 0; i < hit.size(); ++i)
      if (hit[i] != 1 && bad++ < 5) printf("entry %zu hit %d times (nbl %d nbp %d)\n", i, hit[i], g.nbl, g.nbp);
  }
  printf("%ld violations\n", bad);
  return bad ? 1 : 0;
}
