// grid_plan.h -- grids of the exact-slicing GEMM in its dense-output modes
// (the l contraction, the adjoint's GEMMs) and the radial chunk of the
// tensor-core adjoint (host code; plain C++, so the CPU tests compile it and
// check it).
//
// A dense-output GEMM covers C[rows][cols] with 128 x 128 tiles; when there
// are more than four waves of tiles on a 152-SM part, each CTA runs up to
// four consecutive row tiles one after another, so that its set-up, pipeline
// fill and last drain are shared by several tiles (keeping about four waves
// of CTAs).
// The adjoint streams its radial points in chunks; each chunk runs one such
// GEMM over its slices (rows) and the n_b^2 entries (x, y) of M (columns).
// A part-full last wave of CTAs costs as long as a full one, so the chunk is
// chosen, between half and all of the largest one that memory allows, to
// need the fewest waves over the whole call, plus a tenth of a wave per
// chunk for its other launches (ties go to the larger chunk).
#pragma once
#include <cstdint>

namespace modal {
namespace gridp {

constexpr int64_t TILE = 128;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// row tiles per CTA of the dense-output GEMM (nrt row tiles, nct column tiles)
inline int rows_per_cta(int64_t nrt, int64_t nct) {
  const int64_t r = nrt * nct / (4 * 152);
  return (int)(r < 1 ? 1 : (r > 4 ? 4 : r));
}

// CTAs of that grid
inline int64_t ctas(int64_t rows, int64_t cols) {
  const int64_t nrt = cdiv(rows, TILE), nct = cdiv(cols, TILE);
  return nct * cdiv(nrt, rows_per_cta(nrt, nct));
}

// its duration in waves of one row tile on num_sms SMs
inline int64_t waves(int64_t rows, int64_t cols, int num_sms) {
  const int64_t nrt = cdiv(rows, TILE), nct = cdiv(cols, TILE);
  return rows_per_cta(nrt, nct) * cdiv(ctas(rows, cols), num_sms);
}

// cost of streaming n_x radial points in chunks of c (tenths of a wave)
inline int64_t chunk_cost(int64_t n_x, int64_t c, int64_t n_mu, int64_t cols, int num_sms) {
  const int64_t full = n_x / c, rest = n_x % c;
  int64_t cost = full * (10 * waves(c * n_mu, cols, num_sms) + 1);
  if (rest) cost += 10 * waves(rest * n_mu, cols, num_sms) + 1;
  return cost;
}

// the chunk in [ceil(cmax / 2), cmax] of least cost; cmax itself when
// num_sms <= 0 or n_x <= 0
inline int chunk(int64_t n_x, int64_t n_mu, int64_t cols, int64_t cmax, int num_sms) {
  if (cmax < 1) cmax = 1;
  if (num_sms <= 0 || n_x <= 0) return (int)cmax;
  int64_t best = cmax, best_cost = -1;
  for (int64_t c = cmax; c >= 1 && 2 * c >= cmax; --c) {
    const int64_t cost = chunk_cost(n_x, c, n_mu, cols, num_sms);
    if (best_cost < 0 || cost < best_cost) best = c, best_cost = cost;
  }
  return (int)best;
}

}  // namespace gridp
}  // namespace modal
