// Reads lines "kind args..." from stdin and prints what grid_plan.h gives:
//   c rows cols          -> rows_per_cta, ctas
//   w rows cols sms      -> waves
//   k n_x n_mu cols cmax sms -> chunk, then the cost of every chunk in [1, cmax]
#include <cstdio>

#include "../paper_1503_08809_gb300/csrc/grid_plan.h"

using namespace modal::gridp;

int main() {
  char kind;
  while (scanf(" %c", &kind) == 1) {
    if (kind == 'c') {
      long long rows, cols;
      if (scanf("%lld %lld", &rows, &cols) != 2) return 2;
      printf("%d %lld\n", rows_per_cta(cdiv(rows, TILE), cdiv(cols, TILE)), (long long)ctas(rows, cols));
    } else if (kind == 'w') {
      long long rows, cols;
      int sms;
      if (scanf("%lld %lld %d", &rows, &cols, &sms) != 3) return 2;
      printf("%lld\n", (long long)waves(rows, cols, sms));
    } else if (kind == 'k') {
      long long n_x, n_mu, cols, cmax;
      int sms;
      if (scanf("%lld %lld %lld %lld %d", &n_x, &n_mu, &cols, &cmax, &sms) != 5) return 2;
      printf("%d", chunk(n_x, n_mu, cols, cmax, sms));
      for (long long c = 1; c <= cmax; ++c) printf(" %lld", (long long)chunk_cost(n_x, c, n_mu, cols, sms));
      printf("\n");
    } else {
      return 2;
    }
  }
  return 0;
}
