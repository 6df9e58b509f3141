// Checks the slicing of oz_split.h on host: for double-FP32 values (H, L)
// with |H + L| <= 2^7 and |L| <= min(ulp(H)/2, 2^-14), every slice is exact
// in BF16 (low 16 bits of the float zero), slice s is a multiple of 2^(-7 s)
// within its bound (64, the fourth 64.5 + |L| 2^21, the first 128), and |H + L - sum of slices| <= 2^-29 + 2^-37.  Random,
// extreme (|H| = 128) and tie cases; prints the violations, exit 1 if any.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../paper_1503_08809_gb300/csrc/oz_split.h"

using modal::ozs::split_hl;

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next() {
  state ^= state << 13;
  state ^= state >> 7;
  state ^= state << 17;
  return state;
}
static double uni() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
static uint32_t bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
}

int main(int argc, char **argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  long bad = 0;
  for (long i = 0; i < n; ++i) {
    float H;
    switch (i % 4) {
      case 0: H = (float)((uni() * 2 - 1) * 128.0); break;                                   // uniform
      case 1: H = (float)((uni() * 2 - 1) * ldexp(1.0, -(int)(next() % 40))); break;          // small
      case 2: H = (next() & 1) ? 128.f : -128.f; break;                                       // extreme
      default: {                                                                               // ties
        const int s = 1 + (int)(next() % 4), k = (int)(next() % 64);
        H = (float)(ldexp((double)k + 0.5, -7 * s) * ((next() & 1) ? 1 : -1));
      }
    }
    // a valid low part: |L| <= ulp(H)/2 and <= 2^-14
    const double ulp = H == 0.f ? 0.0 : ldexp(1.0, (int)std::ilogb(H) - 23);
    const double lmax = std::fmin(ulp / 2, ldexp(1.0, -14));
    const float L = (float)((uni() * 2 - 1) * lmax);
    if (std::fabs((double)H + (double)L) > 128.0) continue;
    float q[5];
    split_hl(H, L, q);
    double sum = 0;
    bool ok = true;
    for (int s = 0; s < 5; ++s) {
      if (bits(q[s]) & 0xffffu) ok = false;                          // exact in BF16
      const double w = ldexp((double)q[s], 7 * s);                   // units of 2^(-7 s)
      if (w != std::rint(w)) ok = false;
      // the fourth slice rounds (residual + L): half a unit more
      const double bound = s == 0 ? 128.0 : (s == 3 ? 64.5 + std::fabs((double)L) * ldexp(1.0, 21) : 64.0);
      if (std::fabs(w) > bound) ok = false;
      sum += (double)q[s];
    }
    if (std::fabs((double)H + (double)L - sum) > ldexp(1.0, -29) + ldexp(1.0, -37)) ok = false;
    if (!ok) {
      if (bad < 5) printf("violation H=%a L=%a q=%a %a %a %a %a\n", H, L, q[0], q[1], q[2], q[3], q[4]);
      ++bad;
    }
  }
  printf("checked %ld violations %ld\n", n, bad);
  return bad ? 1 : 0;
}
