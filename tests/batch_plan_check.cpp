// Reads "n ns" then n lines "cost bytes" from stdin and prints the batch
// layout of batch_plan.h: the stream of each problem, then the ns + 1
// scratch offsets.
#include <cstdio>
#include <vector>

#include "../paper_1503_08809_gb300/csrc/batch_plan.h"

int main() {
  int n, ns;
  if (scanf("%d %d", &n, &ns) != 2) return 2;
  std::vector<double> cost(n);
  std::vector<size_t> bytes(n);
  for (int i = 0; i < n; ++i) {
    unsigned long long b;
    if (scanf("%lf %llu", &cost[i], &b) != 2) return 2;
    bytes[i] = (size_t)b;
  }
  const modal::batch::Layout bl = modal::batch::layout(n, cost.data(), bytes.data(), ns);
  for (int i = 0; i < n; ++i) printf("%d ", bl.stream_of[i]);
  printf("\n");
  for (int k = 0; k <= ns; ++k) printf("%zu ", bl.off[k]);
  printf("\n");
  return 0;
}
