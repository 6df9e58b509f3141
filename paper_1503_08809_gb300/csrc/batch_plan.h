// batch_plan.h -- how a batch of uneven problems is spread over concurrent
// streams (host code of the batched entry point; plain C++, so the CPU
// tests compile it and check it).
//
// Problems in decreasing cost, each to the stream with the least cost so far
// (longest processing time first, Graham's rule: makespan within 4/3 - 1/(3S)
// of the optimum); each stream owns one scratch block, sized for the largest
// plan it runs, at 256-byte aligned offsets.
#pragma once
#include <algorithm>
#include <cstddef>
#include <vector>

namespace modal {
namespace batch {

constexpr int MAX_STREAMS = 8;

struct Layout {
  int ns = 1;
  std::vector<int> stream_of;            // problem -> stream
  size_t off[MAX_STREAMS + 1] = {};      // scratch block k = [off[k], off[k + 1])
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// cost[i]: work estimate of problem i; bytes[i]: its scratch; ns in 1 .. MAX_STREAMS
inline Layout layout(int n, const double *cost, const size_t *bytes, int ns) {
  Layout bl;
  bl.ns = ns;
  bl.stream_of.assign(n, 0);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  double load[MAX_STREAMS] = {};
  size_t need[MAX_STREAMS] = {};
  for (int i : order) {
    int best = 0;
    for (int k = 1; k < ns; ++k)
      if (load[k] < load[best]) best = k;
    bl.stream_of[i] = best;
    load[best] += cost[i];
    need[best] = bytes[i] > need[best] ? bytes[i] : need[best];
  }
  bl.off[0] = 0;
  for (int k = 0; k < ns; ++k) bl.off[k + 1] = bl.off[k] + align256(need[k] ? need[k] : 256);
  return bl;
}

}  // namespace batch
}  // namespace modal
