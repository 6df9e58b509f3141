// Reads n, then n lines "bh bl" (hex floats), accumulates them with the
// df_add of fp_bits.h from (0, 0) and prints the final (hi, lo) as hex.
#include <cstdio>

#include "../paper_1503_08809_gb300/csrc/fp_bits.h"

int main() {
  long n;
  if (scanf("%ld", &n) != 1) return 2;
  float hi = 0.f, lo = 0.f;
  for (long i = 0; i < n; ++i) {
    float bh, bl;
    if (scanf("%a %a", &bh, &bl) != 2) return 2;
    modal::fpb::df_add(hi, lo, bh, bl);
  }
  printf("%a %a\n", hi, lo);
  return 0;
}
