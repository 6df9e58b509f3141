// dtc_enum.h -- index logic of the direct form on the tensor cores (tc.cu):
// the l1 run of a pair (l2, l3), the search over scanned offsets, the cut of
// the next batch of tiles and a tile's GEMM item.  Plain C++ usable from
// device and host code, so the CPU tests check it against a brute-force
// enumeration of the sorted triples (tests/test_dtc_enum.py).
//
// Terms.  Grid points are class-ordered (class 0 = even l with exact 3j
// weights, every point otherwise; then class 1): crow[k] is the grid index
// of class row k, cls = {size of class 0, size of class 1}.  A pair is the
// grid index pair (i2 <= i3), flattened as i2 * ng + i3; its triples are the
// class rows of the l1 with l3 - l2 <= l1 <= l2 (and l1 + l2 + l3 even with
// exact weights), cut into tiles of cpt consecutive l1.  Per-pair counts are
// scanned into tri_off (triples), tile_off (tiles) and slot_of (pairs that
// have tiles), pairs_nz listing those pairs.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define DTC_HD __host__ __device__ __forceinline__
#else
#define DTC_HD inline
#endif

namespace modal {
namespace dtc {

struct Batch {
  int64_t t0, nt;         // tiles [t0, t0 + nt) (nt = 0: past the end)
  int64_t trip0, n_tri;   // triples [trip0, trip0 + n_tri)
  int64_t slot0, nslots;  // pairs with tiles: slots [slot0, slot0 + nslots)
  int n_items;            // GEMM items (nt x column tiles)
  int pad;
};

// first class row k in [lo, hi) with grid[crow[k]] >= v (hi if none)
DTC_HD int lower(const int *grid, const int *crow, int lo, int hi, int v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (grid[crow[mid]] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// the l1 of the pair (i2 <= i3): class rows [k0, k0 + n)
struct Run {
  int k0, n;
};
DTC_HD Run run(int i2, int i3, const int *grid, const int *crow, const int *cls, bool parity) {
  const int l2 = grid[i2], l3 = grid[i3];
  const int c = parity ? ((l2 + l3) & 1) : 0;
  const int base = c ? cls[0] : 0, end = base + cls[c];
  const int k0 = lower(grid, crow, base, end, l3 - l2);
  const int k1 = lower(grid, crow, base, end, l2 + 1);
  return {k0, k1 > k0 ? k1 - k0 : 0};
}

// last index with off[idx] <= t (entries with zero count share the next
// entry's offset, so this is the entry whose range holds t)
DTC_HD int64_t find(const int64_t *off, int64_t n, int64_t t) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

DTC_HD int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// The batch starting at tile *cursor: at most nt_max tiles and np_max pairs;
// advances the cursor.  tot = {triples, tiles, pairs with tiles}.
DTC_HD Batch next_batch(int64_t &cursor, const int64_t *tot, int nct, int cpt, int64_t npairs,
                        const int64_t *tile_off, const int64_t *tri_off, const int64_t *slot_of,
                        const int *pairs_nz, int64_t nt_max, int64_t np_max) {
  const int64_t ntiles = tot[1], nslots = tot[2];
  Batch r{};
  r.t0 = cursor;
  if (r.t0 >= ntiles) {
    r.t0 = ntiles;
    return r;
  }
  const int64_t pa = find(tile_off, npairs, r.t0);
  r.slot0 = slot_of[pa];
  int64_t t1 = min64(r.t0 + nt_max, ntiles);
  if (r.slot0 + np_max < nslots) t1 = min64(t1, tile_off[pairs_nz[r.slot0 + np_max]]);
  r.nt = t1 - r.t0;
  r.trip0 = tri_off[pa] + (r.t0 - tile_off[pa]) * cpt;
  int64_t trip1 = tot[0];
  if (t1 < ntiles) {
    const int64_t pb = find(tile_off, npairs, t1);
    trip1 = tri_off[pb] + (t1 - tile_off[pb]) * cpt;
  }
  r.n_tri = trip1 - r.trip0;
  r.nslots = slot_of[find(tile_off, npairs, t1 - 1)] - r.slot0 + 1;
  r.n_items = (int)(r.nt * nct);
  cursor = t1;
  return r;
}

// The GEMM item of tile j of a batch and column tile h: {A row, B row,
// first triple of the batch, n | col0 << 16}.
struct Item {
  int a_row0, b_row0, tri0, packed;
};
DTC_HD Item item(const Batch &b, int64_t j, int h, const int64_t *tile_off, const int64_t *tri_off,
                 const int64_t *slot_of, int64_t npairs, int ng, const int *grid, const int *crow, const int *cls,
                 bool parity, int cpt, int nbp, int wu, int urows) {
  const int64_t T = b.t0 + j;
  const int64_t pr = find(tile_off, npairs, T);
  const int tl = (int)(T - tile_off[pr]);
  const Run r = run((int)(pr / ng), (int)(pr % ng), grid, crow, cls, parity);
  const int k = r.k0 + tl * cpt, n = r.n - tl * cpt < cpt ? r.n - tl * cpt : cpt;
  const int tri0 = (int)(tri_off[pr] + (int64_t)tl * cpt - b.trip0);
  const int slot = (int)(slot_of[pr] - b.slot0);
  return {k * nbp, slot * urows + h * wu, tri0, n | (h * wu) << 16};
}

}  // namespace dtc
}  // namespace modal
