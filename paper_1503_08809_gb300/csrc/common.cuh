// common.cuh -- shared device/host helpers for libmodal (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/modal.h"

#define MODAL_PI 3.14159265358979323846

namespace modal {

static inline __host__ __device__ int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline __host__ __device__ int cdiv(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Double-double arithmetic from the error-free transformations of Dekker
// (1971) and Knuth (TAOCP vol. 2): a value is hi + lo with |lo| <= ulp(hi)/2,
// giving ~106 significant bits.  Used where the paper asks for more than FP64
// (Gauss-Legendre nodes, Section 2.2) and for the 3j product table.
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dd dd_fast_two_sum(double a, double b) {  // |a| >= |b|
  double s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dd dd_two_prod(double a, double b) {
  double p = a * b;
  return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = dd_two_sum(x.hi, y.hi);
  dd t = dd_two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = dd_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return dd_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  dd p = dd_two_prod(x.hi, y.hi);
  p.lo = fma(x.hi, y.lo, p.lo);
  p.lo = fma(x.lo, y.hi, p.lo);
  return dd_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd x, double d) {
  dd p = dd_two_prod(x.hi, d);
  p.lo = fma(x.lo, d, p.lo);
  return dd_fast_two_sum(p.hi, p.lo);
}
// x / d for a double d: long division with one correction term.
__device__ __forceinline__ dd dd_div_d(dd x, double d) {
  double q1 = x.hi / d;
  dd p = dd_two_prod(q1, d);
  dd r = dd_two_sum(x.hi, -p.hi);
  r.lo -= p.lo;
  r.lo += x.lo;
  double q2 = (r.hi + r.lo) / d;
  return dd_fast_two_sum(q1, q2);
}
// x / y: two long-division steps.
__device__ __forceinline__ dd dd_div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = dd_sub(x, dd_mul_d(y, q1));
  double q2 = r.hi / y.hi;
  r = dd_sub(r, dd_mul_d(y, q2));
  double q3 = r.hi / y.hi;
  dd q = dd_fast_two_sum(q1, q2);
  return dd_add(q, {q3, 0.0});
}

// ---------------------------------------------------------------------------
// Index helpers for the unordered pair {u, v} (u <= v) of basis indices:
// uv = v (v + 1) / 2 + u.  n_pairs(n) = n (n + 1) / 2.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int pair_index(int u, int v) {
  if (u > v) { int t = u; u = v; v = t; }
  return v * (v + 1) / 2 + u;
}
__host__ __device__ __forceinline__ void pair_decode(int uv, int &u, int &v) {
  int vv = (int)((sqrtf(8.0f * (float)uv + 1.0f) - 1.0f) * 0.5f);
  while (vv * (vv + 1) / 2 > uv) --vv;
  while ((vv + 1) * (vv + 2) / 2 <= uv) ++vv;
  v = vv;
  u = uv - vv * (vv + 1) / 2;
}

// ---------------------------------------------------------------------------
// Layout of the unsymmetrised triple-product table G used by the separable
// path.  With Y_xy{u,v}(s) = w_s (M_xu M_yv + M_xv M_yu) for x <= y and
// u <= v, the 3x3 permanent of Eq. 2D for a sorted late triple a <= b <= c
// can be expanded along the row of c or along the row of a:
//   perm = Y_ab{p,r} M_ct + Y_ab{p,t} M_cr + Y_ab{r,t} M_cp     (row of c)
//        = Y_bc{p,r} M_at + Y_bc{p,t} M_ar + Y_bc{r,t} M_ap     (row of a).
// G is stored in blocks by the middle index b.  Block b < h takes the first
// form, G[(a, uv), (c, t)] = sum_s Y_ab{u,v}(s) M_ct(s): rows (a in [0, b],
// uv), columns (c in [b, nb_late), t); block b >= h the second, G[(c, uv),
// (a, t)] = sum_s Y_bc{u,v}(s) M_at(s): rows (c in [b, nb_late), uv), columns
// (a in [0, b], t).  Either way a block has (b+1)(nb_late-b) P2 nb_prim
// entries, row-major, blocks end to end.  h = nb_late gives the first form
// throughout; h = (nb_late + 1) / 2 (make_glayout_split) keeps every block at
// least (nb_late + 1) / 2 column groups wide and needs the Y rows of only the
// pairs (a, b) with b < h and (b, c) with b >= h -- about half of them.  The
// Y operand lists the pairs a block uses block by block (y_pair), so block
// b's rows are the Y rows [ypair0(b) P2, ...) and its columns the M rows
// [colstart(b), colstart(b) + cols(b)).
// ---------------------------------------------------------------------------
struct GLayout {
  int nbl, nbp, P2, h;
  __host__ __device__ bool first(int b) const { return b < h; }
  __host__ __device__ int64_t rows(int b) const { return (int64_t)(first(b) ? b + 1 : nbl - b) * P2; }
  __host__ __device__ int64_t cols(int b) const { return (int64_t)(first(b) ? nbl - b : b + 1) * nbp; }
  __host__ __device__ int64_t colstart(int b) const { return first(b) ? (int64_t)b * nbp : 0; }
  __host__ __device__ int64_t offset(int b) const {
    // sum_{i=1..b} i (nbl - i + 1) * P2 * nbp
    int64_t B = b;
    int64_t s = (int64_t)(nbl + 1) * B * (B + 1) / 2 - B * (B + 1) * (2 * B + 1) / 6;
    return s * P2 * nbp;
  }
  __host__ __device__ int64_t size() const { return offset(nbl); }
  // pairs of Y rows used by block b, the first of them in Y order, and all of them
  __host__ __device__ int ypairs(int b) const { return first(b) ? b + 1 : nbl - b; }
  __host__ __device__ int ypair0(int b) const {
    const int f = b < h ? b : h;  // blocks of the first form before b: 1 + 2 + ... + f pairs
    const int n2 = b - f;         // blocks h .. b-1 of the second form: nbl-h + ... + nbl-b+1 pairs
    return f * (f + 1) / 2 + n2 * (2 * nbl - 2 * h - n2 + 1) / 2;
  }
  __host__ __device__ int ypairs_total() const { return ypair0(nbl); }
  // the pair x <= y of Y pair j (0 <= j < ypairs_total())
  __host__ __device__ void y_pair(int j, int &x, int &y) const {
    int b = 0;
    while (b + 1 < nbl && ypair0(b + 1) <= j) ++b;
    const int i = j - ypair0(b);
    if (first(b)) {
      x = i;
      y = b;
    } else {
      x = b;
      y = b + i;
    }
  }
  __host__ __device__ int64_t index(int a, int b, int uv, int c, int t) const {
#ifdef MODAL_DEBUG
    return checked_index(a, b, uv, c, t);
#else
    return first(b) ? offset(b) + ((int64_t)a * P2 + uv) * cols(b) + (int64_t)(c - b) * nbp + t
                    : offset(b) + ((int64_t)(c - b) * P2 + uv) * cols(b) + (int64_t)a * nbp + t;
#endif
  }
  // index() with every argument checked: 0 <= a <= b <= c < nbl,
  // 0 <= uv < P2, 0 <= t < nbp; -1 otherwise.  index() itself checks only in
  // builds with MODAL_DEBUG defined (callers then skip a negative index).
  __host__ __device__ int64_t checked_index(int a, int b, int uv, int c, int t) const {
    if (a < 0 || a > b || b > c || c >= nbl || uv < 0 || uv >= P2 || t < 0 || t >= nbp) return -1;
    return first(b) ? offset(b) + ((int64_t)a * P2 + uv) * cols(b) + (int64_t)(c - b) * nbp + t
                    : offset(b) + ((int64_t)(c - b) * P2 + uv) * cols(b) + (int64_t)a * nbp + t;
  }
};

static inline GLayout make_glayout(int nbl, int nbp) { return GLayout{nbl, nbp, nbp * (nbp + 1) / 2, nbl}; }
static inline GLayout make_glayout_split(int nbl, int nbp) {
  return GLayout{nbl, nbp, nbp * (nbp + 1) / 2, (nbl + 1) / 2};
}

}  // namespace modal
