// Checks the integer-bit conversions of fp_bits.h against their FP64
// counterparts, bit for bit, on random and adversarial inputs (ties, carries
// into the exponent, range edges, zeros, subnormals).  Prints the number of
// mismatches of each function; exit status 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <initializer_list>

#include "../paper_1503_08809_gb300/csrc/fp_bits.h"

using namespace modal::fpb;

static uint64_t state = 88172645463325252ull;
static uint64_t next() {  // xorshift64
  state ^= state << 13;
  state ^= state >> 7;
  state ^= state << 17;
  return state;
}

int main(int argc, char **argv) {
  const long n = argc > 1 ? atol(argv[1]) : 2000000;
  long bad_split = 0, bad_scale = 0, checked = 0;
  for (long i = 0; i < n; ++i) {
    uint64_t u = next();
    switch (i % 6) {
      case 1: u = (u & 0x800fffffffffffffull) | ((uint64_t)(950 + next() % 200) << 52); break;  // fast path
      case 2: u = (u & 0x800fffffe0000000ull) | (1ull << 28) | ((uint64_t)(950 + next() % 200) << 52); break;  // tie
      case 3: u = (u & 0x8000000000000000ull) | ((uint64_t)(950 + next() % 200) << 52) | 0xfffffff000000ull |
                  (next() & 0xffffff); break;  // carry into the exponent
      case 4: u = (u & 0x800fffffffffffffull) | ((uint64_t)((next() & 1) ? 946 + next() % 8 : 1145 + next() % 8) << 52);
              break;  // range edges
      case 5: u = (next() & 1) ? (u & 0x8000000000000000ull) : (u & 0x800fffffffffffffull); break;  // zero, subnormal
      default: break;
    }
    const double x = d_from(u);
    if (std::isnan(x)) continue;
    ++checked;
    const f2 a = df_from_d(x), b = df_from_d_fast(x);
    if (f_bits(a.h) != f_bits(b.h) || f_bits(a.l) != f_bits(b.l)) ++bad_split;
    // f32_scaled_f64 on the two halves, with exponents across the double range
    const int e = (int)(next() % 2300) - 1150;
    for (float y : {a.h, a.l}) {
      if (std::isnan(y)) continue;
      const double r1 = ldexp((double)y, e), r2 = f32_scaled_f64(y, e);
      if (d_bits(r1) != d_bits(r2)) ++bad_scale;
    }
  }
  printf("checked %ld split_mismatch %ld scale_mismatch %ld\n", checked, bad_split, bad_scale);
  return (bad_split || bad_scale) ? 1 : 0;
}
