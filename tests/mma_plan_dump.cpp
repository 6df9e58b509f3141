// Prints the MMA schedules of mma_plan.h (the searched one for every tile
// width, then the singles fallback, then the pair schedule) as hex words: "w header run run ...".
#include <cstdio>

#include "../paper_1503_08809_gb300/csrc/mma_plan.h"

static void dump(int w, const uint32_t (&o)[1 + modal::plan::RUNS_MAX]) {
  printf("%d %x", w, o[0]);
  for (unsigned r = 0; r < (o[0] & 0xffu); ++r) printf(" %x", o[1 + r]);
  printf("\n");
}

int main() {
  uint32_t o[1 + modal::plan::RUNS_MAX];
  for (int w = 16; w <= 128; w += 16) {
    modal::plan::mma_plan(w, o);
    dump(w, o);
  }
  modal::plan::singles_plan(o);
  for (int w = 16; w <= 128; w += 16) dump(-w, o);  // negative width: the fallback at width w
  modal::plan::pair_plan(o);
  dump(0, o);                                       // width 0: the 2-SM (pair) schedule, any width
  return 0;
}
