// Host check of the direct form's enumeration on the tensor cores
// (csrc/dtc_enum.h) against a brute-force list of the sorted triples: for
// several grids, both weight modes and several tile and batch sizes, the
// batches cut from the device cursor cover every tile once and the triples
// in order; each triple of a batch is the brute-force one; every GEMM item's
// rows are the class rows of its tile's l1 and land on its triples' blocks;
// the number of batches stays inside the host's bound.  Prints violations;
// exit 1 if any.
#include <cstdio>
#include <vector>

#include "../paper_1503_08809_gb300/csrc/dtc_enum.h"

using namespace modal;

struct Tri {
  int l1, l2, l3;
  bool operator==(const Tri &o) const { return l1 == o.l1 && l2 == o.l2 && l3 == o.l3; }
};

static long bad = 0;
#define CHECK(c, ...)                          \
  do {                                         \
    if (!(c) && bad++ < 8) printf(__VA_ARGS__); \
  } while (0)

static void check(const std::vector<int> &grid, bool parity, int nbp, int64_t nt_max, int64_t np_max) {
  const int ng = (int)grid.size(), cpt = 128 / nbp, P2 = nbp * (nbp + 1) / 2;
  const int nct = (P2 + 127) / 128, wu = ((P2 + nct - 1) / nct + 15) / 16 * 16, urows = nct * wu;
  // class order
  std::vector<int> crow;
  for (int i = 0; i < ng; ++i)
    if (!parity || !(grid[i] & 1)) crow.push_back(i);
  const int n0 = (int)crow.size();
  if (parity)
    for (int i = 0; i < ng; ++i)
      if (grid[i] & 1) crow.push_back(i);
  const int cls[2] = {n0, (int)crow.size() - n0};
  // per-pair counts and scans
  const int64_t npairs = (int64_t)ng * ng;
  std::vector<int64_t> tri_cnt(npairs, 0), tile_cnt(npairs, 0), nz(npairs, 0);
  for (int i2 = 0; i2 < ng; ++i2)
    for (int i3 = i2; i3 < ng; ++i3) {
      const dtc::Run r = dtc::run(i2, i3, grid.data(), crow.data(), cls, parity);
      tri_cnt[i2 * ng + i3] = r.n;
      tile_cnt[i2 * ng + i3] = (r.n + cpt - 1) / cpt;
      nz[i2 * ng + i3] = r.n > 0;
    }
  std::vector<int64_t> tri_off(npairs), tile_off(npairs), slot_of(npairs);
  int64_t a = 0, b = 0, c = 0;
  for (int64_t i = 0; i < npairs; ++i) {
    tri_off[i] = a;
    tile_off[i] = b;
    slot_of[i] = c;
    a += tri_cnt[i];
    b += tile_cnt[i];
    c += nz[i];
  }
  const int64_t tot[3] = {a, b, c};
  std::vector<int> pairs_nz(c > 0 ? c : 1);
  for (int64_t i = 0; i < npairs; ++i)
    if (nz[i]) pairs_nz[slot_of[i]] = (int)i;
  // brute force: pairs (i2 <= i3) in row-major order, then l1 ascending
  std::vector<Tri> brute;
  for (int i2 = 0; i2 < ng; ++i2)
    for (int i3 = i2; i3 < ng; ++i3)
      for (int i1 = 0; i1 <= i2; ++i1) {
        const int l1 = grid[i1], l2 = grid[i2], l3 = grid[i3];
        if (l1 + l2 < l3 || (parity && ((l1 + l2 + l3) & 1))) continue;
        brute.push_back({l1, l2, l3});
      }
  CHECK((int64_t)brute.size() == tot[0], "count %zu vs %lld\n", brute.size(), (long long)tot[0]);
  // batches
  const int64_t pairs_sorted = (int64_t)ng * (ng + 1) / 2;
  const int64_t bound = (pairs_sorted + (int64_t)ng * (ng + 1) * (ng + 2) / 6 / cpt + nt_max - 1) / nt_max +
                        (pairs_sorted + np_max - 1) / np_max;
  int64_t cursor = 0, tiles_seen = 0, tri_seen = 0, nbatch = 0;
  while (true) {
    const dtc::Batch bt = dtc::next_batch(cursor, tot, nct, cpt, npairs, tile_off.data(), tri_off.data(),
                                          slot_of.data(), pairs_nz.data(), nt_max, np_max);
    if (bt.nt == 0) break;
    ++nbatch;
    CHECK(bt.t0 == tiles_seen && bt.trip0 == tri_seen, "batch order\n");
    CHECK(bt.n_tri > 0 && bt.n_tri <= bt.nt * cpt && bt.nt <= nt_max, "batch sizes\n");
    CHECK(bt.nslots > 0 && bt.nslots <= np_max, "batch pairs %lld\n", (long long)bt.nslots);
    // the fill's view of each triple
    for (int64_t tb = 0; tb < bt.n_tri; ++tb) {
      const int64_t t = bt.trip0 + tb;
      const int64_t pr = dtc::find(tri_off.data(), npairs, t);
      const dtc::Run r = dtc::run((int)(pr / ng), (int)(pr % ng), grid.data(), crow.data(), cls, parity);
      const int k = (int)(t - tri_off[pr]);
      CHECK(k >= 0 && k < r.n, "triple %lld outside its run\n", (long long)t);
      const Tri got{grid[crow[r.k0 + k]], grid[pr / ng], grid[pr % ng]};
      CHECK(t < (int64_t)brute.size() && got == brute[t], "triple %lld differs\n", (long long)t);
    }
    // items: rows of each tile are its l1's class rows; triples covered once
    std::vector<int> cover(bt.n_tri, 0);
    for (int64_t j = 0; j < bt.nt; ++j)
      for (int h = 0; h < nct; ++h) {
        const dtc::Item it = dtc::item(bt, j, h, tile_off.data(), tri_off.data(), slot_of.data(), npairs, ng,
                                       grid.data(), crow.data(), cls, parity, cpt, nbp, wu, urows);
        const int n = it.packed & 0xffff, col0 = it.packed >> 16;
        CHECK(n >= 1 && n <= cpt && col0 == h * wu, "item size\n");
        CHECK(it.a_row0 % nbp == 0 && it.a_row0 / nbp + n <= ng, "item rows\n");
        CHECK(it.b_row0 >= 0 && it.b_row0 + wu <= np_max * urows, "item B rows\n");
        CHECK(it.tri0 >= 0 && it.tri0 + n <= bt.n_tri, "item triples\n");
        for (int q = 0; q < n && it.tri0 + q < bt.n_tri; ++q) {
          const Tri &tr = brute[bt.trip0 + it.tri0 + q];
          CHECK(grid[crow[it.a_row0 / nbp + q]] == tr.l1, "item row l1\n");
          if (h == 0) cover[it.tri0 + q]++;
        }
      }
    for (int64_t q = 0; q < bt.n_tri; ++q) CHECK(cover[q] == 1, "triple covered %d times\n", cover[q]);
    tiles_seen += bt.nt;
    tri_seen += bt.n_tri;
  }
  CHECK(tiles_seen == tot[1] && tri_seen == tot[0], "coverage\n");
  CHECK(nbatch <= bound, "batches %lld > bound %lld\n", (long long)nbatch, (long long)bound);
}

int main() {
  std::vector<std::vector<int>> grids;
  {
    std::vector<int> g;  // sparse: every l to 50, step 2 to 200, step 5 to 500, step 10 above
    for (int l = 2; l <= 600; l += (l < 50 ? 1 : l < 200 ? 2 : l < 500 ? 5 : 10)) g.push_back(l);
    grids.push_back(g);
  }
  {
    std::vector<int> g;
    for (int l = 2; l <= 48; ++l) g.push_back(l);
    grids.push_back(g);
  }
  grids.push_back({4});
  grids.push_back({2, 9});
  grids.push_back({3, 5, 9, 100});
  grids.push_back({10, 11, 12, 13, 40, 41, 70});
  for (const auto &g : grids)
    for (int parity = 0; parity < 2; ++parity) {
      check(g, parity, 20, 64, 16);
      check(g, parity, 3, 4096, 1024);
      check(g, parity, 7, 2, 1);
      check(g, parity, 1, 37, 5);
    }
  printf("%ld violations\n", bad);
  return bad ? 1 : 0;
}
