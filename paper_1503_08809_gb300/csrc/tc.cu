// tc.cu -- tensor-core (tcgen05) form of the separable path with exponent-
// aligned BF16 splitting (Ozaki, Ogita, Oishi & Rump 2012).
//
// Both dense contractions of the separable path -- the l contraction of
// Eq. legendre and the slice reduction of the triple product of Eq. 2D --
// run as C = A B^T over K on 5th-generation tensor cores:
//
//  * every row of A and B is scaled by a power of two 2^e (per K chunk) so
//    that |x / 2^e| <= 1, then written as five BF16 slices of 7 bits each
//    (oz_split.h): x / 2^e * 2^7 = q0 + q1 2^-7 + q2 2^-14 + q3 2^-21 +
//    q4 2^-28 (35 bits), |q0| <= 128, |qs| <= 64 except the fourth, which
//    takes the low part of the double-FP32 value (<= 192);
//  * the 15 slice products with s + t <= 4 are issued as runs of
//    tcgen05.mma (mma_plan.h: consecutive B slices of one A slice in one MMA)
//    into four or five TMEM accumulators: level 0 (q0 q0'), level 1
//    (q0 q1' + q1 q0') and levels 2-4 on the others.  With at most 1024 K
//    terms per chunk the level-0 and level-1 partial sums are integers (in
//    units of 1 and 2^-7) of magnitude at most 2^24, hence exact in the FP32
//    accumulator whatever the summation order;
//  * at the end of each chunk the epilogue warps read the accumulators
//    (tcgen05.ld), apply the row and column scales and add the chunk into a
//    double-FP32 (hi, lo) running sum (hi in registers, lo in shared
//    memory; fp_bits.h), offset by a global exponent bias so that the FP32
//    range cannot overflow.  The result is written (or added) in FP64, its
//    conversion assembled from the bits (fp_bits.h).
//
// Operands are staged by TMA (cp.async.bulk.tensor, 64-byte swizzle) in a
// two-stage mbarrier pipeline; one thread issues the MMAs.  Every wait is
// bounded: on give-up the CTA raises an error word, drains its copies in
// flight, frees TMEM and returns.
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <queue>
#include <vector>

#include "common.cuh"
#include "direct.cuh"
#include "grid_plan.h"
#include "kernels.cuh"
#include "ptx.cuh"
#include "tc.cuh"
#include "mma_plan.h"
#include "fp_bits.h"
#include "oz_split.h"
#include "dtc_enum.h"

namespace modal {

// double-FP32 values and FP64 <-> double-FP32 conversions by integer work
using fpb::df_from_d;
using fpb::df_from_d_fast;
using fpb::f2;
using fpb::f32_scaled_f64;
using fpb::df_add;

static thread_local char g_tc_err[256] = "";
const char *tc_last_error() { return g_tc_err; }

constexpr int OZ_BETA = 7;        // bits per slice
constexpr int OZ_SLICES = 5;      // slices per operand
constexpr int OZ_MAXLEV = 4;      // products with s + t <= 4 (15 of the 25)
constexpr int OZ_KC = 1024;       // K terms per exact chunk
constexpr int OZ_BM = 128;        // rows per tile (TMEM lanes)
constexpr int OZ_BN = 128;        // columns per tile
constexpr int OZ_BK = 32;         // K per stage: 64-byte rows, 64-byte swizzle
constexpr int OZ_STAGES = 2;
constexpr int OZ_PREFETCH = 4;    // stages of A prefetched into L2 ahead of their loads
constexpr int OZ_ROWB = OZ_BK * 2;                       // bytes per smem row
constexpr int OZ_A_BYTES = OZ_SLICES * OZ_BM * OZ_ROWB;  // 40 KB
constexpr int OZ_B_BYTES = OZ_SLICES * OZ_BN * OZ_ROWB;  // 40 KB
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;       // TMA warp, MMA warp, epilogue
constexpr int OZ_LO_BYTES = OZ_BM * OZ_BN * 4;            // low halves of the running sums
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES + 1024 /*align*/ + 256 /*barriers*/;
static_assert(OZ_SMEM <= 232448, "shared memory per CTA");
constexpr long long OZ_WAIT_CYCLES = 4000000000LL;       // ~2 s at 2 GHz
static_assert(OZ_KC % OZ_BK == 0, "chunk must hold whole stages");

// error word bits
constexpr int ERR_TIMEOUT = 1;
constexpr int ERR_RANGE = 2;  // a value outside the FP32 exponent range of the split operands

// ---------------------------------------------------------------------------
// Splitting helpers (FP64 input)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int exp_bound(double m) {  // smallest e with m <= 2^e
  if (!(m > 0.0)) return -100000;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// Exact 2^k as a float for k in [-126, 127] (built from the exponent bits).
__device__ __forceinline__ float pow2f(int k) {
  k = max(-126, min(127, k));
  return __int_as_float((k + 127) << 23);
}

// 2^k for k <= 127, and 0 below the normal range (a scale that small only
// multiplies contributions far below the FP32 resolution of the result).
__device__ __forceinline__ float pow2f_or0(int k) {
  return k < -126 ? 0.f : __int_as_float((min(k, 127) + 127) << 23);
}

// Scale factors 2^(BETA - e) as two exact float factors (the exponent range of
// the values may exceed one float exponent).  e < -99999 marks an all-zero row.
struct SplitScale {
  float s1, s2;
  bool zero;
};
__device__ __forceinline__ SplitScale split_scale(int e) {
  SplitScale r;
  r.zero = e < -99999;
  const int k = r.zero ? 0 : OZ_BETA - e;
  r.s1 = pow2f(k / 2);
  r.s2 = pow2f(k - k / 2);
  return r;
}

// The slicing of one double-FP32 value: oz_split.h (host and device code).
static_assert(OZ_BETA == ozs::BETA && OZ_SLICES == ozs::SLICES, "one slicing for splits and kernels");
constexpr int OZ_FOLD = ozs::FOLD;  // slice before which L joins the residual
using ozs::split_hl;
__host__ __device__ constexpr float oz_pow2c(int k) { return ozs::pow2c(k); }

__device__ __forceinline__ void split_scaled(float h, float l, const SplitScale &sc,
                                              __nv_bfloat16 (&out)[OZ_SLICES]) {
  float q[OZ_SLICES];
  const float H = sc.zero ? 0.f : (h * sc.s1) * sc.s2;
  const float L = sc.zero ? 0.f : (l * sc.s1) * sc.s2;
  split_hl(H, L, q);
#pragma unroll
  for (int s = 0; s < OZ_SLICES; ++s) out[s] = __float2bfloat16_rn(q[s]);
}

__device__ __forceinline__ void split_f2(float h, float l, int e, __nv_bfloat16 (&out)[OZ_SLICES]) {
  split_scaled(h, l, split_scale(e), out);
}

// exponent e with |x| <= 2^e for every |x| <= m (1 + 2^-20): room for the
// low part of a double-FP32 value and for rounding of the maximum itself
__device__ __forceinline__ int exp_bound_f(float m) {
  if (!(m > 0.f)) return -100000;
  int e;
  frexpf(m * (1.0f + 1.0f / 1048576.0f), &e);
  return e;
}

// Rows of the l-contraction operands.  Row r of A is A[j][l] q_a(l) with
// r = (j, a); row r of B is q~_p(l, x0 + xl) with r = (xl, p).  One warp per
// (row, K chunk): pass 1 finds max |x|, pass 2 writes the slices; only the
// one product A q uses the FP64 unit (the split into double-FP32 is integer
// work, df_from_d_fast).
template <bool IS_A>
__global__ void k_split_lrows(int64_t rows, int L, int Kpad, const double *__restrict__ Atab,
                              const double *__restrict__ q, const double *__restrict__ qt, int nbl, int nbp,
                              int x0, __nv_bfloat16 *__restrict__ out, int *__restrict__ ex,
                              int *__restrict__ emax, int *__restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nch = cdiv(L, OZ_KC);
  if (w >= rows * nch) return;
  const int64_t r = w / nch;
  const int ch = (int)(w % nch);
  auto val = [&](int l) -> double {
    if (IS_A) {
      int j = (int)(r / nbl), a = (int)(r % nbl);
      return Atab[(int64_t)j * L + l] * q[(int64_t)a * L + l];
    } else {
      int xl = (int)(r / nbp), p = (int)(r % nbp);
      return qt[((int64_t)(x0 + xl) * nbp + p) * L + l];
    }
  };
  const int l0 = ch * OZ_KC, l1 = min(L, l0 + OZ_KC);
  float m = 0.f;
  for (int l = l0 + lane; l < l1; l += 32) m = fmaxf(m, fabsf(__double2float_rn(val(l))));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (!(m < 1e37f)) {  // also catches inf/NaN
    if (lane == 0) atomicOr(err, ERR_RANGE);
    m = 0.f;
  }
  const int e = exp_bound_f(m);
  const int64_t sstride = rows * (int64_t)Kpad;
  const int lend = min(Kpad, l0 + OZ_KC);
  for (int l = l0 + lane; l < lend; l += 32) {
    const double v = l < L ? val(l) : 0.0;
    const f2 vd = df_from_d_fast(v);
    __nv_bfloat16 o[OZ_SLICES];
    split_f2(vd.h, vd.l, e, o);
#pragma unroll
    for (int s = 0; s < OZ_SLICES; ++s) out[s * sstride + r * Kpad + l] = o[s];
  }
  if (lane == 0) {
    ex[(int64_t)ch * rows + r] = e;
    if (e > -99999) atomicMax(emax, e);
  }
}

// words[0] = error bits and words[1] = exponent maximum of the A operand of
// the l contraction (both set once per call); words[2..7] = per-chunk maxima.
// mode 0: per chunk (words 2..7); 1: per call (all); 2: per problem of a
// batch (word 1 and 2..7, keeping the error bits of earlier problems)
__global__ void k_init_words(int *w, int mode) {
  const int t = threadIdx.x;
  if (t == 0) {
    if (mode == 1) w[0] = 0;
  } else if (t == 1) {
    if (mode != 0) w[1] = -100000;
  } else if (t < 8) {
    w[t] = -100000;
  }
}

// ---------------------------------------------------------------------------
// The GEMM kernel.
// OUT_MODE 0: l contraction, store M[(xl*n_mu + j)*nbl + a)*nbp + p] from row
//             (j, a) and column (xl, p).
// OUT_MODE 1: triple product, add into the G block of b (rows (a,{u,v}),
//             columns (c,t), c >= b) -- tiles decoded from blockIdx.x.
// ---------------------------------------------------------------------------
// MMA schedule of one 16-deep K step for a tile of width w (see mma_plans):
// plan[0] = number of runs | accumulators used << 8; plan[1 + r] = run r as
// sa | first sb << 4 | count << 8 | accumulator << 12 | first-touch << 16.
constexpr int OZ_PLAN_MAX = 16;  // >= 15: the all-singles schedule always fits
struct OzParams {
  uint32_t plan[OZ_BN / 16][1 + OZ_PLAN_MAX];  // by w / 16 - 1
  int64_t rowsA, rowsB;   // operand rows (TMA extents)
  int Kpad;               // K extent (multiple of OZ_BK)
  int nchunks;            // K chunks of OZ_KC
  const int *eA;          // [nchunks][rowsA]
  const int *eB;          // [nchunks][rowsB]
  const int *emaxA, *emaxB;
  double *out;
  int *err;
  // OUT_MODE 0
  int n_mu, nbl, nbp;
  int rows_per_cta;       // row tiles each CTA runs one after another (OUT_MODE 0)
  // OUT_MODE 1
  GLayout g;
  long long wait_cycles;
  // OUT_MODE 2: dense C[r][c] at out[r * ld_r + c * ld_c], stored or added;
  // with kdev, no work at all when *kdev <= koff (a batch past the end)
  int64_t ld_r, ld_c;
  int out_accumulate;
  const int64_t *kdev;
  int64_t koff;
  // OUT_MODE 3 (direct form): work items {A row, B row, first triple, n | col0 << 16},
  // item blockIdx.x + t gridDim.x for t = 0, 1, ... below *item_count; tile row
  // c nbp + p is function p of the item's triple c < n, stored at
  // out[((tri0 + c) nbp + p) P2 + col0 + col] for col0 + col < P2
  const int4 *items;
  const int *item_count;
  int P2, wtile;
  // OUT_MODE 1: each tile's K chunks split over ksplit consecutive CTAs of
  // chunks_per_split chunks each; the first adds its partial sums into out,
  // part k >= 1 stores them at out_part + (k - 1) part_stride (added in
  // order afterwards, so the result does not depend on which part ends first)
  int ksplit, chunks_per_split;
  double *out_part;
  int64_t part_stride;
  int tile0;  // OUT_MODE 1: first tile of the launch (tiles in block order)
};


// Width of the column tiles of a G block with `cols` columns: the block is cut
// into ceil(cols / 128) tiles of equal width, rounded up to a multiple of 16
// (the MMA N granularity), so narrow blocks do not pay for 128 columns.
__host__ __device__ inline int g_tile_width(int64_t cols) {
  const int64_t nct = cdiv64(cols, OZ_BN);
  return (int)(cdiv64(cdiv64(cols, nct), 16) * 16);
}
// the same with column tiles of at most `cap` (a multiple of 16, <= OZ_BN)
__host__ __device__ inline int g_tile_width_cap(int64_t cols, int cap) {
  const int64_t nct = cdiv64(cols, cap);
  return (int)(cdiv64(cdiv64(cols, nct), 16) * 16);
}

// Tensor maps of the B operand with boxes of 16, 32, ..., 128 rows: a tile of
// MMA width N loads only its N rows of B (slices then lie N * 64 bytes apart).
struct BMaps {
  CUtensorMap m[OZ_BN / 16];
};

template <int OUT_MODE>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ BMaps bmaps, OzParams P) {
  if (OUT_MODE == 2 && P.kdev && *P.kdev <= P.koff) return;  // the whole CTA: nothing to add
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  float *lo_s = (float *)(sm + OZ_STAGES * OZ_STAGE_BYTES);  // [col][row]
  uint64_t *full = (uint64_t *)(sm + OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES);
  uint64_t *empty = full + OZ_STAGES;
  uint64_t *acc_full = empty + OZ_STAGES;
  uint64_t *acc_empty = acc_full + 1;
  uint64_t *mma_done = acc_empty + 1;
  uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // ---- tile ----
  int64_t a_row0, b_row0, R, C;  // operand row origins, valid rows/cols of this tile
  int64_t out_base = 0;
  int bblk = 0;
  int ntile = OZ_BN;  // MMA N of this tile (a multiple of 16)
  int ntt = 1;  // tiles of this CTA (OUT_MODE 0: row tiles of one column tile)
  bool lead = true;  // the first column tile of its row tile: it prefetches A
  int kc0 = 0, nchk = P.nchunks;  // this CTA's exact K chunks [kc0, kc0 + nchk) of every tile
  if (OUT_MODE == 3) {
    const int nit = *P.item_count;
    if ((int)blockIdx.x >= nit) return;  // the whole CTA: no item
    ntt = (nit - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    lead = false;
    ntile = P.wtile;
    a_row0 = b_row0 = 0;  // per item
    R = C = 0;
  } else if (OUT_MODE != 1) {
    // column tiles vary fastest, so the CTAs that share a row tile of A run
    // together and A is read from HBM about once; each CTA then moves on to
    // the next row tile, so its set-up, pipeline fill and last drain are
    // shared by several tiles and overlap the neighbouring tile's work
    const int64_t rt0 = (int64_t)blockIdx.y * P.rows_per_cta;
    lead = blockIdx.x == 0;
    ntt = (int)min((int64_t)P.rows_per_cta, cdiv64(P.rowsA, OZ_BM) - rt0);
    a_row0 = rt0 * OZ_BM;
    b_row0 = (int64_t)blockIdx.x * OZ_BN;
    R = min((int64_t)OZ_BM, P.rowsA - a_row0);
    C = min((int64_t)OZ_BN, P.rowsB - b_row0);
  } else {
    const int ks = P.ksplit > 1 ? P.ksplit : 1;
    int t = (int)blockIdx.x / ks + P.tile0, rt = 0, ct = 0;
    if (ks > 1) {
      kc0 = ((int)blockIdx.x % ks) * P.chunks_per_split;
      nchk = min(P.chunks_per_split, P.nchunks - kc0);
    }
    if (nchk <= 0) return;  // the whole CTA: an empty K range
    int64_t rowoff = 0;
    for (bblk = 0; bblk < P.g.nbl; ++bblk) {
      int nrt = (int)cdiv64(P.g.rows(bblk), OZ_BM), nct = (int)cdiv64(P.g.cols(bblk), OZ_BN);
      if (t < nrt * nct) {
        rt = t / nct;
        ct = t % nct;
        break;
      }
      t -= nrt * nct;
      rowoff += P.g.rows(bblk);
    }
    if (bblk >= P.g.nbl) return;
    lead = ct == 0;
    // the block's columns go to its column tiles in equal widths (multiples of 16)
    ntile = g_tile_width(P.g.cols(bblk));
    a_row0 = rowoff + (int64_t)rt * OZ_BM;
    b_row0 = P.g.colstart(bblk) + (int64_t)ct * ntile;
    R = min((int64_t)OZ_BM, P.g.rows(bblk) - (int64_t)rt * OZ_BM);
    C = min((int64_t)ntile, P.g.cols(bblk) - (int64_t)ct * ntile);
    out_base = P.g.offset(bblk) + (int64_t)rt * OZ_BM * P.g.cols(bblk) + (int64_t)ct * ntile;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, 32 * OZ_EPI_WARPS);
    ptx::mbar_init(mma_done, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int steps_per_chunk = OZ_KC / OZ_BK;
  const int kbase = kc0 * steps_per_chunk;  // first K step of the CTA's range
  const int ksteps = min(P.Kpad / OZ_BK, (kc0 + nchk) * steps_per_chunk) - kbase;
  const CUtensorMap *tmB = &bmaps.m[ntile / 16 - 1];
  const uint32_t stage_bytes = (uint32_t)(OZ_A_BYTES + OZ_SLICES * ntile * OZ_ROWB);

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      ptx::prefetch_tmap(tmB);
      int issued = 0;
      bool stop = false;
      for (int tt = 0; tt < ntt && !stop; ++tt) {
        int ar = (int)(a_row0 + (int64_t)tt * OZ_BM), br = (int)b_row0;
        if (OUT_MODE == 3) {
          const int4 it = P.items[blockIdx.x + (int64_t)tt * gridDim.x];
          ar = it.x;
          br = it.y;
        }
        // A tiles are pulled into L2 OZ_PREFETCH stages ahead of their loads,
        // so that the two-stage ring waits on L2 rather than on HBM latency;
        // only the first column tile of a row tile does it (the others load
        // the same rows at about the same time, and their prefetches would
        // only add L2 lookups: 2.6 % of the triple GEMM's time)
        if (lead)
          for (int i = 0; i < OZ_PREFETCH && i < ksteps; ++i)
            ptx::tma_prefetch_3d(&tmA, (kbase + i) * OZ_BK, ar, 0);
        for (int i = 0; i < ksteps; ++i) {
          const int g = tt * ksteps + i;  // step count of the CTA: stage and phase
          const int s = g % OZ_STAGES;
          const uint32_t ph = (uint32_t)((g / OZ_STAGES) & 1);
          if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) {
            stop = true;
            break;
          }
          unsigned char *st = sm + s * OZ_STAGE_BYTES;
          ptx::mbar_arrive_expect_tx(&full[s], stage_bytes);
          ptx::tma_load_3d(st, &tmA, &full[s], (kbase + i) * OZ_BK, ar, 0);
          ptx::tma_load_3d(st + OZ_A_BYTES, tmB, &full[s], (kbase + i) * OZ_BK, br, 0);
          if (lead && i + OZ_PREFETCH < ksteps)
            ptx::tma_prefetch_3d(&tmA, (kbase + i + OZ_PREFETCH) * OZ_BK, ar, 0);
          ++issued;
        }
      }
      // on abort: wait (bounded) for the copies in flight before anyone frees smem
      if (*abort_flag) {
        for (int i = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); i < issued; ++i) {
          volatile int dummy = 0;
          ptx::mbar_wait(&full[i % OZ_STAGES], (uint32_t)((i / OZ_STAGES) & 1), &dummy, OZ_WAIT_CYCLES);
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0) {
      const uint32_t idesc0 = ptx::idesc_bf16_f32(OZ_BM, 0);  // N goes in per run
      const uint32_t *plan = P.plan[ntile / 16 - 1];
      const int nruns = (int)(plan[0] & 0xffu);
      uint32_t run[OZ_PLAN_MAX];
#pragma unroll
      for (int r = 0; r < OZ_PLAN_MAX; ++r) run[r] = plan[1 + r];
      const uint32_t sbase = ptx::smem_u32(sm);
      int chunk = 0;  // chunks of the CTA, over all its tiles
      const int nsteps = ntt * ksteps;
      for (int g = 0; g < nsteps; ++g) {
        const int i = g % ksteps;  // step inside the tile
        const int s = g % OZ_STAGES;
        const uint32_t ph = (uint32_t)((g / OZ_STAGES) & 1);
        const bool chunk_start = (i % steps_per_chunk) == 0;
        if (chunk_start && chunk > 0) {
          // accumulators must have been drained by the epilogue
          if (!ptx::mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), abort_flag, P.wait_cycles)) break;
        }
        if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) break;
        ptx::tc_fence_after();
        const uint32_t a0 = sbase + s * OZ_STAGE_BYTES;
        // descriptors of slice 0 at k = 0; the other operands differ only in the
        // start-address field, by compile-time offsets (>> 4)
        const uint64_t ad0 = ptx::smem_desc(a0, 16, 8 * OZ_ROWB, ptx::SW_64B);
        const uint64_t bd0 = ptx::smem_desc(a0 + OZ_A_BYTES, 16, 8 * OZ_ROWB, ptx::SW_64B);
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
          for (int r = 0; r < OZ_PLAN_MAX; ++r) {
            if (r >= nruns) break;
            const uint32_t e = run[r];
            const uint32_t sa = e & 15u, sb = (e >> 4) & 15u, n = (e >> 8) & 15u, acc = (e >> 12) & 15u;
            // the first touch of an accumulator in a chunk overwrites it
            const bool first = chunk_start && kk == 0 && ((e >> 16) & 1u);
            const uint32_t N = n * (uint32_t)ntile;
            const uint64_t ad = ad0 + (uint64_t)((sa * OZ_BM * OZ_ROWB + kk * 32) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((sb * (uint32_t)ntile * OZ_ROWB + kk * 32) >> 4);
            ptx::mma_bf16(tmem + acc * (uint32_t)ntile, ad, bd, idesc0 | ((N >> 3) << 17), first ? 0u : 1u);
          }
        }
        ptx::mma_commit(&empty[s]);  // stage s may be refilled once these MMAs retire
        const bool chunk_end = ((i + 1) % steps_per_chunk) == 0 || i + 1 == ksteps;  // per tile
        if (chunk_end) {
          ptx::mma_commit(acc_full);
          ++chunk;
        }
      }
      // every MMA this thread issued has retired before TMEM can be freed
      ptx::mma_commit(mma_done);
      volatile int dummy = 0;
      ptx::mbar_wait(mma_done, 0, &dummy, OZ_WAIT_CYCLES);
    }
  } else {
    // ================= epilogue: drain each chunk into double-FP32 =================
    const int ew = warp - 2;                 // 0..7
    const int quarter = warp & 3;            // TMEM lane quarter this warp may access
    const int chalf = ew >> 2;               // column half
    const int row = quarter * 32 + lane;     // tile row of this thread
    const int col0 = chalf * 64;
    const int emA = *P.emaxA, emB = *P.emaxB;
    const int ebias = emA + emB + 40;
    const int nacc = (int)((P.plan[ntile / 16 - 1][0] >> 8) & 0xffu);
    float hi[64];  // high halves in registers, low halves in lo_s
    bool ok = true;
    for (int tt = 0; tt < ntt && ok; ++tt) {
    int64_t ar0 = a_row0 + (int64_t)tt * OZ_BM;  // this tile's first row of A
    int64_t br0 = b_row0;                         // and of B
    int64_t Rt = OUT_MODE != 1 ? min((int64_t)OZ_BM, P.rowsA - ar0) : R;
    int64_t Ct = C;
    int4 it = make_int4(0, 0, 0, 0);
    if (OUT_MODE == 3) {
      it = P.items[blockIdx.x + (int64_t)tt * gridDim.x];
      ar0 = it.x;
      br0 = it.y;
      Rt = (int64_t)(it.w & 0xffff) * P.nbp;
      Ct = min((int64_t)ntile, (int64_t)(P.P2 - (it.w >> 16)));
    }
#pragma unroll
    for (int c = 0; c < 64; ++c) {
      hi[c] = 0.f;
      lo_s[(col0 + c) * OZ_BM + row] = 0.f;
    }
    for (int cl = 0; cl < nchk; ++cl) {
      const int ch = kc0 + cl;          // exact K chunk
      const int cg = tt * nchk + cl;    // chunk count of the CTA (barrier phase)
      // the whole warp goes on or gives up together (shuffles below)
      const bool got = ptx::mbar_wait(acc_full, (uint32_t)(cg & 1), abort_flag, P.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      ptx::tc_fence_after();
      // the chunk's scale 2^(ea + eb - 2 BETA - ebias) = row factor x column factor;
      // lane i holds the column factors of columns col0 + i and col0 + 32 + i
      const int ea = (ar0 + row < P.rowsA) ? P.eA[(int64_t)ch * P.rowsA + ar0 + row] : -100000;
      const float fa = pow2f_or0(ea - emA);
      float fbl[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t bcol = br0 + col0 + h * 32 + lane;
        const int eb = (bcol < P.rowsB) ? __ldg(P.eB + (int64_t)ch * P.rowsB + bcol) : -100000;
        fbl[h] = pow2f_or0(eb - emB - 2 * OZ_BETA - 40);
      }
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < 16; ++cb) {
        if (col0 + cb * 4 >= ntile) break;  // columns beyond the MMA width (warp-uniform)
        // accumulators ntile columns apart: level 0, level 1, then levels >= 2
        float v0[4], v1[4], v2[4], v3[4], v4[4];
        const uint32_t cc = (uint32_t)(col0 + cb * 4);
        const uint32_t w = (uint32_t)ntile;
        ptx::tmem_ld4(tl + cc, v0);
        ptx::tmem_ld4(tl + w + cc, v1);
        ptx::tmem_ld4(tl + 2 * w + cc, v2);
        ptx::tmem_ld4(tl + 3 * w + cc, v3);
        if (nacc > 4) ptx::tmem_ld4(tl + 4 * w + cc, v4);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 4; ++k) v2[k] += nacc > 4 ? v3[k] + v4[k] : v3[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = cb * 4 + k;
          const float f = fa * __shfl_sync(0xffffffffu, fbl[c >> 5], c & 31);
          // exact level-0 and level-1 sums, then the rest
          float s = v0[k] + v1[k];
          float bb = s - v0[k];
          float e = (v0[k] - (s - bb)) + (v1[k] - bb);
          e += v2[k];
          float lo = lo_s[(col0 + c) * OZ_BM + row];
          df_add(hi[c], lo, s * f, e * f);
          lo_s[(col0 + c) * OZ_BM + row] = lo;
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(acc_empty);
    }
    if (ok && !*abort_flag && row < Rt) {
      // OUT_MODE 0 writes M[x][j][a][p] for A row (j, a) and B row (x, p):
      // the row's offset once per tile, the column's (x, p) stepped along
      int64_t mrow = 0, mx = 0;
      int xl = 0, p = 0;
      if (OUT_MODE == 0) {
        const int64_t rA = ar0 + row, rB = b_row0 + col0;
        mrow = rA * P.nbp;  // (j nbl + a) nbp, as rA = j nbl + a
        mx = (int64_t)P.n_mu * P.nbl * P.nbp;
        xl = (int)(rB / P.nbp);
        p = (int)(rB % P.nbp);
      }
      double *zrow = nullptr;  // OUT_MODE 3: this row's Z entries (triple c, function p)
      if (OUT_MODE == 3)
        zrow = P.out + ((int64_t)(it.z + row / P.nbp) * P.nbp + row % P.nbp) * P.P2 + (it.w >> 16);
#pragma unroll  // full unroll keeps hi[]/lo[] in registers
      for (int c = 0; c < 64; ++c) {
        const int col = col0 + c;
        if (col < Ct) {
          const double v = f32_scaled_f64(hi[c], ebias) + f32_scaled_f64(lo_s[(col0 + c) * OZ_BM + row], ebias);
          if (OUT_MODE == 0) {
            P.out[xl * mx + mrow + p] = v;
          } else if (OUT_MODE == 3) {
            zrow[col] = v;
          } else if (OUT_MODE == 2) {
            double *d = P.out + (ar0 + row) * P.ld_r + (b_row0 + col) * P.ld_c;
            *d = P.out_accumulate ? *d + v : v;
          } else {
            const int64_t o = out_base + (int64_t)row * P.g.cols(bblk) + col;
            if (kc0 == 0) P.out[o] += v;
            else P.out_part[(int64_t)(kc0 / P.chunks_per_split - 1) * P.part_stride + o] = v;
          }
        }
        if (OUT_MODE == 0 && ++p == P.nbp) {
          p = 0;
          ++xl;
        }
      }
    }
    }  // tiles of the CTA
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.err, ERR_TIMEOUT);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// The triple GEMM on CTA pairs (2-SM tcgen05.mma, M = 256).
//
// A cluster of two CTAs takes two 128-row tiles of one G block (rows
// 2 rp * 128 + rank * 128 ..) and one column tile of width w.  Each CTA's
// shared memory holds its own 128 rows of the five A slices; the even CTA
// holds the five B slices of the column tile, the odd CTA the same slices
// shifted by one (slot j = slice j + 1, slot 4 = zeros from the tensor map's
// out-of-range fill).  The pair MMA reads B columns 0 .. N/2-1 from the even
// CTA and N/2 .. N-1 from the odd CTA, so one MMA of N = 2w at slot j
// multiplies the A slice by B slices j and j + 1 (mma_plan.h, pair_plan):
// each SM's tensor core reads half of the B columns it would read alone.
// The even CTA issues everything: the four TMA loads of a stage (into both
// CTAs' shared memory, all signalled on its own mbarrier), the MMAs and the
// commits; both CTAs drain their own accumulators (their 128 rows of D).
// Roles of the odd CTA: TMEM allocation and the drain only.
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_gemm_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ BMaps bmaps, OzParams P) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  float *lo_s = (float *)(sm + OZ_STAGES * OZ_STAGE_BYTES);  // [col][row]
  uint64_t *full = (uint64_t *)(sm + OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES);
  uint64_t *empty = full + OZ_STAGES;
  uint64_t *acc_full = empty + OZ_STAGES;
  uint64_t *acc_empty = acc_full + 1;
  uint64_t *mma_done = acc_empty + 1;
  uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_ctarank();  // 0: issues the pair's work, 1: its partner
  const bool leader = rank == 0;

  // ---- tile of the pair: row tiles 2 rp, 2 rp + 1 of block bblk, column tile ct ----
  int t = (int)(blockIdx.x >> 1), rp = 0, ct = 0, bblk;
  int64_t rowoff = 0;
  for (bblk = 0; bblk < P.g.nbl; ++bblk) {
    const int nrp = (int)cdiv64(cdiv64(P.g.rows(bblk), OZ_BM), 2), nct = (int)cdiv64(P.g.cols(bblk), OZ_BN);
    if (t < nrp * nct) {
      rp = t / nct;
      ct = t % nct;
      break;
    }
    t -= nrp * nct;
    rowoff += P.g.rows(bblk);
  }
  if (bblk >= P.g.nbl) return;  // both CTAs of a cluster decode the same tile
  const bool lead = ct == 0;    // the first column tile prefetches the rows of A
  const int ntile = g_tile_width(P.g.cols(bblk));
  const int64_t pair_row0 = rowoff + (int64_t)rp * 2 * OZ_BM;       // first A row of the pair
  const int64_t rt_loc = (int64_t)rp * 2 + rank;                      // this CTA's row tile in the block
  const int64_t R = min((int64_t)OZ_BM, P.g.rows(bblk) - rt_loc * OZ_BM);  // may be <= 0 (odd tail)
  const int64_t C = min((int64_t)ntile, P.g.cols(bblk) - (int64_t)ct * ntile);
  const int64_t a_row0 = pair_row0 + (int64_t)rank * OZ_BM;
  const int64_t b_row0 = P.g.colstart(bblk) + (int64_t)ct * ntile;
  const int64_t out_base = P.g.offset(bblk) + rt_loc * OZ_BM * P.g.cols(bblk) + (int64_t)ct * ntile;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, 2 * OZ_EPI_WARPS);  // one arrival per drain warp of both CTAs
    ptx::mbar_init(mma_done, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(tmem_slot, 512);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  ptx::cluster_sync();  // both CTAs' barriers and TMEM exist before either is used
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksteps = P.Kpad / OZ_BK;
  const int steps_per_chunk = OZ_KC / OZ_BK;
  const CUtensorMap *tmB = &bmaps.m[ntile / 16 - 1];
  const uint32_t stage_bytes = (uint32_t)(OZ_A_BYTES + OZ_SLICES * ntile * OZ_ROWB);

  if (warp == 0) {
    // ================= TMA producer (even CTA) =================
    if (leader && lane == 0) {
      ptx::prefetch_tmap(&tmA);
      ptx::prefetch_tmap(tmB);
      const uint32_t own = ptx::smem_u32(sm), peer = ptx::mapa_shared(own, 1);
      const int ar = (int)pair_row0;
      if (lead)
        for (int i = 0; i < OZ_PREFETCH && i < ksteps; ++i) {
          ptx::tma_prefetch_3d(&tmA, i * OZ_BK, ar, 0);
          ptx::tma_prefetch_3d(&tmA, i * OZ_BK, ar + OZ_BM, 0);
        }
      int issued = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % OZ_STAGES;
        const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
        if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) break;
        const uint32_t fb = ptx::smem_u32(&full[s]), so = (uint32_t)(s * OZ_STAGE_BYTES);
        ptx::mbar_arrive_expect_tx(&full[s], 2 * stage_bytes);
        ptx::tma_load_3d_pair(own + so, &tmA, fb, i * OZ_BK, ar, 0);
        ptx::tma_load_3d_pair(own + so + OZ_A_BYTES, tmB, fb, i * OZ_BK, (int)b_row0, 0);
        ptx::tma_load_3d_pair(peer + so, &tmA, fb, i * OZ_BK, ar + OZ_BM, 0);
        ptx::tma_load_3d_pair(peer + so + OZ_A_BYTES, tmB, fb, i * OZ_BK, (int)b_row0, 1);  // slices 1..5
        if (lead && i + OZ_PREFETCH < ksteps) {
          ptx::tma_prefetch_3d(&tmA, (i + OZ_PREFETCH) * OZ_BK, ar, 0);
          ptx::tma_prefetch_3d(&tmA, (i + OZ_PREFETCH) * OZ_BK, ar + OZ_BM, 0);
        }
        ++issued;
      }
      // on abort: wait (bounded) for the copies in flight, which land in both
      // CTAs and all complete on this CTA's barriers
      if (*abort_flag) {
        for (int i = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); i < issued; ++i) {
          volatile int dummy = 0;
          ptx::mbar_wait(&full[i % OZ_STAGES], (uint32_t)((i / OZ_STAGES) & 1), &dummy, OZ_WAIT_CYCLES);
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer (even CTA) =================
    if (leader && lane == 0) {
      const uint32_t idesc = ptx::idesc_bf16_f32(2 * OZ_BM, 2 * ntile);
      const uint32_t *plan = P.plan[0];
      const int nruns = (int)(plan[0] & 0xffu);
      uint32_t run[OZ_PLAN_MAX];
#pragma unroll
      for (int r = 0; r < OZ_PLAN_MAX; ++r) run[r] = plan[1 + r];
      const uint32_t sbase = ptx::smem_u32(sm);
      int chunk = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % OZ_STAGES;
        const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
        const bool chunk_start = (i % steps_per_chunk) == 0;
        if (chunk_start && chunk > 0) {
          // both CTAs have drained the accumulators of the previous chunk
          if (!ptx::mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), abort_flag, P.wait_cycles)) break;
        }
        if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) break;
        ptx::tc_fence_after();
        const uint32_t a0 = sbase + s * OZ_STAGE_BYTES;
        const uint64_t ad0 = ptx::smem_desc(a0, 16, 8 * OZ_ROWB, ptx::SW_64B);
        const uint64_t bd0 = ptx::smem_desc(a0 + OZ_A_BYTES, 16, 8 * OZ_ROWB, ptx::SW_64B);
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
          for (int r = 0; r < OZ_PLAN_MAX; ++r) {
            if (r >= nruns) break;
            const uint32_t e = run[r];
            const uint32_t sa = e & 15u, j = (e >> 4) & 15u, acc = (e >> 12) & 15u;
            const bool first = chunk_start && kk == 0 && ((e >> 16) & 1u);
            const uint64_t ad = ad0 + (uint64_t)((sa * OZ_BM * OZ_ROWB + kk * 32) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((j * (uint32_t)ntile * OZ_ROWB + kk * 32) >> 4);
            ptx::mma_bf16_pair(tmem + acc * (uint32_t)ntile, ad, bd, idesc, first ? 0u : 1u);
          }
        }
        ptx::mma_commit_pair(&empty[s]);
        const bool chunk_end = ((i + 1) % steps_per_chunk) == 0 || i + 1 == ksteps;
        if (chunk_end) {
          ptx::mma_commit_pair_mc(acc_full, (uint16_t)3);  // both CTAs' drains
          ++chunk;
        }
      }
      ptx::mma_commit_pair(mma_done);
      volatile int dummy = 0;
      ptx::mbar_wait(mma_done, 0, &dummy, OZ_WAIT_CYCLES);
    }
  } else {
    // ================= epilogue (both CTAs): drain own 128 rows =================
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int chalf = ew >> 2;
    const int row = quarter * 32 + lane;
    const int col0 = chalf * 64;
    const int emA = *P.emaxA, emB = *P.emaxB;
    const int ebias = emA + emB + 40;
    const uint32_t empty_addr = leader ? 0u : ptx::mapa_shared(ptx::smem_u32(acc_empty), 0);
    float hi[64];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 64; ++c) {
      hi[c] = 0.f;
      lo_s[(col0 + c) * OZ_BM + row] = 0.f;
    }
    for (int ch = 0; ch < P.nchunks; ++ch) {
      const bool got = ptx::mbar_wait(acc_full, (uint32_t)(ch & 1), abort_flag, P.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      ptx::tc_fence_after();
      const int ea = (a_row0 + row < P.rowsA) ? P.eA[(int64_t)ch * P.rowsA + a_row0 + row] : -100000;
      const float fa = pow2f_or0(ea - emA);
      float fbl[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t bcol = b_row0 + col0 + h * 32 + lane;
        const int eb = (bcol < P.rowsB) ? __ldg(P.eB + (int64_t)ch * P.rowsB + bcol) : -100000;
        fbl[h] = pow2f_or0(eb - emB - 2 * OZ_BETA - 40);
      }
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < 16; ++cb) {
        if (col0 + cb * 4 >= ntile) break;
        float v0[4], v1[4], v2[4], v3[4];
        const uint32_t cc = (uint32_t)(col0 + cb * 4);
        const uint32_t w = (uint32_t)ntile;
        ptx::tmem_ld4(tl + cc, v0);
        ptx::tmem_ld4(tl + w + cc, v1);
        ptx::tmem_ld4(tl + 2 * w + cc, v2);
        ptx::tmem_ld4(tl + 3 * w + cc, v3);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = cb * 4 + k;
          const float f = fa * __shfl_sync(0xffffffffu, fbl[c >> 5], c & 31);
          float s = v0[k] + v1[k];
          float bb = s - v0[k];
          float e = (v0[k] - (s - bb)) + (v1[k] - bb);
          e += v2[k] + v3[k];
          float lo = lo_s[(col0 + c) * OZ_BM + row];
          df_add(hi[c], lo, s * f, e * f);
          lo_s[(col0 + c) * OZ_BM + row] = lo;
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (leader) ptx::mbar_arrive(acc_empty);
        else ptx::mbar_arrive_cluster(empty_addr);
      }
    }
    if (ok && !*abort_flag && row < R) {
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        const int col = col0 + c;
        if (col < C) {
          const double v = f32_scaled_f64(hi[c], ebias) + f32_scaled_f64(lo_s[(col0 + c) * OZ_BM + row], ebias);
          double *d = P.out + out_base + (int64_t)row * P.g.cols(bblk) + col;
          *d += v;
        }
      }
    }
  }
  // neither CTA frees TMEM or exits while its partner may still use its
  // shared memory (TMA writes, MMA operand reads, remote arrivals)
  ptx::tc_fence_before();
  ptx::cluster_sync();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.err, ERR_TIMEOUT);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// The triple GEMM as a persistent kernel draining a device work queue.
//
// Work items are (G tile, K range) pairs: a tile of a G block (128 rows x
// w columns, as in k_ozaki_gemm<1>) over a whole number of exact K chunks.
// The host lists them in order of decreasing modelled cost (longest first);
// each CTA's producer thread takes the next item with an atomic fetch-add on
// a counter in device memory and hands its number to the MMA thread and the
// eight drain warps through a four-slot ring in shared memory (mbarriers
// "item full" / "item empty", bounded waits), then streams the item's
// operands.  The TMEM accumulators and the TMA ring carry on from item to
// item, so one item's drain and write-out overlap the next item's MMAs.  A
// tile split into several K ranges is summed into G with FP64 atomic adds.
// No CTA ever waits for another CTA: the grid need not be resident at once.
// ---------------------------------------------------------------------------
constexpr int Q_ITEMS_MAX = 4096;  // items of the in-parameter queue table
constexpr int Q_RING = 4;          // item slots between the producer and the consumers
struct QueueParams {
  OzParams o;
  int wmax;          // column tiles of at most wmax (a multiple of 16, <= OZ_BN)
  int n_items;       // items in the queue
  int nkr;           // K ranges per tile (1: tiles are not split)
  int chunks_per_kr; // exact K chunks per range (the last range may be shorter)
  int *head;         // device counter of taken items (zero before the launch)
  uint32_t item[Q_ITEMS_MAX];  // tile << 8 | K range, in the order of taking
};

// tile t of the triple product's block structure (tiles of 128 rows x w columns, w <= wmax)
__device__ __forceinline__ void q_tile(const GLayout &g, int wmax, int t, int &bblk, int &rt, int &ct,
                                       int64_t &rowoff) {
  rowoff = 0;
  for (bblk = 0; bblk < g.nbl; ++bblk) {
    const int nrt = (int)cdiv64(g.rows(bblk), OZ_BM), nct = (int)cdiv64(g.cols(bblk), wmax);
    if (t < nrt * nct) {
      rt = t / nct;
      ct = t % nct;
      return;
    }
    t -= nrt * nct;
    rowoff += g.rows(bblk);
  }
}

struct QItem {
  int64_t a_row0, b_row0, R, C, out_base, ldo;
  int ntile, c0, c1;  // MMA width; K chunks [c0, c1)
  bool lead, split;
};

__device__ __forceinline__ QItem q_decode(const QueueParams &Q, uint32_t code) {
  QItem it;
  const int t = (int)(code >> 8), kr = (int)(code & 0xffu);
  int bblk, rt, ct;
  int64_t rowoff;
  q_tile(Q.o.g, Q.wmax, t, bblk, rt, ct, rowoff);
  it.ntile = g_tile_width_cap(Q.o.g.cols(bblk), Q.wmax);
  it.a_row0 = rowoff + (int64_t)rt * OZ_BM;
  it.b_row0 = Q.o.g.colstart(bblk) + (int64_t)ct * it.ntile;
  it.R = min((int64_t)OZ_BM, Q.o.g.rows(bblk) - (int64_t)rt * OZ_BM);
  it.C = min((int64_t)it.ntile, Q.o.g.cols(bblk) - (int64_t)ct * it.ntile);
  it.ldo = Q.o.g.cols(bblk);
  it.out_base = Q.o.g.offset(bblk) + (int64_t)rt * OZ_BM * it.ldo + (int64_t)ct * it.ntile;
  it.c0 = kr * Q.chunks_per_kr;
  it.c1 = min(Q.o.nchunks, it.c0 + Q.chunks_per_kr);
  it.lead = ct == 0 && kr == 0;
  it.split = Q.nkr > 1;
  return it;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_gemm_q(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ BMaps bmaps,
                   const __grid_constant__ QueueParams Q) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  float *lo_s = (float *)(sm + OZ_STAGES * OZ_STAGE_BYTES);  // [col][row]
  uint64_t *full = (uint64_t *)(sm + OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES);
  uint64_t *empty = full + OZ_STAGES;
  uint64_t *acc_full = empty + OZ_STAGES;
  uint64_t *acc_empty = acc_full + 1;
  uint64_t *mma_done = acc_empty + 1;
  uint64_t *item_full = mma_done + 1;
  uint64_t *item_empty = item_full + Q_RING;
  uint32_t *tmem_slot = (uint32_t *)(item_empty + Q_RING);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  volatile int *item_ring = (volatile int *)(tmem_slot + 2);  // [Q_RING]
  const OzParams &P = Q.o;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, OZ_EPI_WARPS);  // one arrival per drain warp
    ptx::mbar_init(mma_done, 1);
    for (int r = 0; r < Q_RING; ++r) {
      ptx::mbar_init(&item_full[r], 1);
      ptx::mbar_init(&item_empty[r], 1 + OZ_EPI_WARPS);  // the MMA thread and every drain warp
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int steps_per_chunk = OZ_KC / OZ_BK;
  const int ksteps = P.Kpad / OZ_BK;

  if (warp == 0) {
    // ================= queue + TMA producer =================
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      int issued = 0;  // stages issued by this CTA over all its items
      for (int j = 0;; ++j) {
        const int slot = j % Q_RING;
        if (!ptx::mbar_wait(&item_empty[slot], (uint32_t)(((j / Q_RING) & 1) ^ 1), abort_flag, P.wait_cycles)) break;
        const int it_no = atomicAdd(Q.head, 1);
        const int code = it_no < Q.n_items ? (int)Q.item[it_no] : -1;
        item_ring[slot] = code;
        ptx::mbar_arrive(&item_full[slot]);  // release: the slot is written
        if (code < 0) break;
        const QItem it = q_decode(Q, (uint32_t)code);
        const CUtensorMap *tmB = &bmaps.m[it.ntile / 16 - 1];
        const uint32_t stage_bytes = (uint32_t)(OZ_A_BYTES + OZ_SLICES * it.ntile * OZ_ROWB);
        const int i0 = it.c0 * steps_per_chunk, i1 = min(ksteps, it.c1 * steps_per_chunk);
        const int ar = (int)it.a_row0;
        if (it.lead)
          for (int i = i0; i < i0 + OZ_PREFETCH && i < i1; ++i) ptx::tma_prefetch_3d(&tmA, i * OZ_BK, ar, 0);
        bool stop = false;
        for (int i = i0; i < i1; ++i) {
          const int s = issued % OZ_STAGES;
          const uint32_t ph = (uint32_t)((issued / OZ_STAGES) & 1);
          if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) {
            stop = true;
            break;
          }
          unsigned char *st = sm + s * OZ_STAGE_BYTES;
          ptx::mbar_arrive_expect_tx(&full[s], stage_bytes);
          ptx::tma_load_3d(st, &tmA, &full[s], i * OZ_BK, ar, 0);
          ptx::tma_load_3d(st + OZ_A_BYTES, tmB, &full[s], i * OZ_BK, (int)it.b_row0, 0);
          if (it.lead && i + OZ_PREFETCH < i1) ptx::tma_prefetch_3d(&tmA, (i + OZ_PREFETCH) * OZ_BK, ar, 0);
          ++issued;
        }
        if (stop) break;
      }
      if (*abort_flag) {  // the copies in flight land before shared memory is released
        for (int i = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); i < issued; ++i) {
          volatile int dummy = 0;
          ptx::mbar_wait(&full[i % OZ_STAGES], (uint32_t)((i / OZ_STAGES) & 1), &dummy, OZ_WAIT_CYCLES);
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0) {
      const uint32_t idesc0 = ptx::idesc_bf16_f32(OZ_BM, 0);
      const uint32_t sbase = ptx::smem_u32(sm);
      int g = 0;      // stages consumed over all items
      int chunk = 0;  // chunks over all items (accumulator phases)
      for (int j = 0;; ++j) {
        const int slot = j % Q_RING;
        if (!ptx::mbar_wait(&item_full[slot], (uint32_t)((j / Q_RING) & 1), abort_flag, P.wait_cycles)) break;
        const int code = item_ring[slot];
        ptx::mbar_arrive(&item_empty[slot]);
        if (code < 0) break;
        const QItem it = q_decode(Q, (uint32_t)code);
        // the width's schedule in registers (the issue loop is this thread's critical path)
        const uint32_t *plan = P.plan[it.ntile / 16 - 1];
        const int nruns = (int)(plan[0] & 0xffu);
        uint32_t run[OZ_PLAN_MAX];
#pragma unroll
        for (int r = 0; r < OZ_PLAN_MAX; ++r) run[r] = plan[1 + r];
        const int i0 = it.c0 * steps_per_chunk, i1 = min(ksteps, it.c1 * steps_per_chunk);
        bool stop = false;
        for (int i = i0; i < i1; ++i, ++g) {
          const int s = g % OZ_STAGES;
          const uint32_t ph = (uint32_t)((g / OZ_STAGES) & 1);
          const bool chunk_start = ((i - i0) % steps_per_chunk) == 0;
          if (chunk_start && chunk > 0 &&
              !ptx::mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), abort_flag, P.wait_cycles)) {
            stop = true;
            break;
          }
          if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) {
            stop = true;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t a0 = sbase + s * OZ_STAGE_BYTES;
          const uint64_t ad0 = ptx::smem_desc(a0, 16, 8 * OZ_ROWB, ptx::SW_64B);
          const uint64_t bd0 = ptx::smem_desc(a0 + OZ_A_BYTES, 16, 8 * OZ_ROWB, ptx::SW_64B);
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
            for (int r = 0; r < OZ_PLAN_MAX; ++r) {
              if (r >= nruns) break;
              const uint32_t e = run[r];
              const uint32_t sa = e & 15u, sb = (e >> 4) & 15u, n = (e >> 8) & 15u, acc = (e >> 12) & 15u;
              const bool first = chunk_start && kk == 0 && ((e >> 16) & 1u);
              const uint32_t N = n * (uint32_t)it.ntile;
              const uint64_t ad = ad0 + (uint64_t)((sa * OZ_BM * OZ_ROWB + kk * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((sb * (uint32_t)it.ntile * OZ_ROWB + kk * 32) >> 4);
              ptx::mma_bf16(tmem + acc * (uint32_t)it.ntile, ad, bd, idesc0 | ((N >> 3) << 17), first ? 0u : 1u);
            }
          }
          ptx::mma_commit(&empty[s]);
          if (((i - i0 + 1) % steps_per_chunk) == 0 || i + 1 == i1) {
            ptx::mma_commit(acc_full);
            ++chunk;
          }
        }
        if (stop) break;
      }
      ptx::mma_commit(mma_done);
      volatile int dummy = 0;
      ptx::mbar_wait(mma_done, 0, &dummy, OZ_WAIT_CYCLES);
    }
  } else {
    // ================= drain each chunk into double-FP32; write the item out =================
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int chalf = ew >> 2;
    const int row = quarter * 32 + lane;
    const int col0 = chalf * 64;
    const int emA = *P.emaxA, emB = *P.emaxB;
    const int ebias = emA + emB + 40;
    float hi[64];
    int chunk = 0;
    bool ok = true;
    for (int j = 0; ok; ++j) {
      const int slot = j % Q_RING;
      const bool got_item = ptx::mbar_wait(&item_full[slot], (uint32_t)((j / Q_RING) & 1), abort_flag, P.wait_cycles);
      if (!__all_sync(0xffffffffu, got_item)) break;
      const int code = item_ring[slot];
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&item_empty[slot]);
      if (code < 0) break;
      const QItem it = q_decode(Q, (uint32_t)code);
      const int nacc = (int)((P.plan[it.ntile / 16 - 1][0] >> 8) & 0xffu);
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        hi[c] = 0.f;
        lo_s[(col0 + c) * OZ_BM + row] = 0.f;
      }
      for (int ch = it.c0; ch < it.c1; ++ch, ++chunk) {
        const bool got = ptx::mbar_wait(acc_full, (uint32_t)(chunk & 1), abort_flag, P.wait_cycles);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        ptx::tc_fence_after();
        const int ea = (it.a_row0 + row < P.rowsA) ? P.eA[(int64_t)ch * P.rowsA + it.a_row0 + row] : -100000;
        const float fa = pow2f_or0(ea - emA);
        float fbl[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t bcol = it.b_row0 + col0 + h * 32 + lane;
          const int eb = (bcol < P.rowsB) ? __ldg(P.eB + (int64_t)ch * P.rowsB + bcol) : -100000;
          fbl[h] = pow2f_or0(eb - emB - 2 * OZ_BETA - 40);
        }
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
        for (int cb = 0; cb < 16; ++cb) {
          if (col0 + cb * 4 >= it.ntile) break;  // columns beyond the MMA width (warp-uniform)
          float v0[4], v1[4], v2[4], v3[4], v4[4];
          const uint32_t cc = (uint32_t)(col0 + cb * 4);
          const uint32_t w = (uint32_t)it.ntile;
          ptx::tmem_ld4(tl + cc, v0);
          ptx::tmem_ld4(tl + w + cc, v1);
          ptx::tmem_ld4(tl + 2 * w + cc, v2);
          ptx::tmem_ld4(tl + 3 * w + cc, v3);
          if (nacc > 4) ptx::tmem_ld4(tl + 4 * w + cc, v4);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int k = 0; k < 4; ++k) v2[k] += nacc > 4 ? v3[k] + v4[k] : v3[k];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int c = cb * 4 + k;
            const float f = fa * __shfl_sync(0xffffffffu, fbl[c >> 5], c & 31);
            float s = v0[k] + v1[k];
            float bb = s - v0[k];
            float e = (v0[k] - (s - bb)) + (v1[k] - bb);
            e += v2[k];
            float lo = lo_s[(col0 + c) * OZ_BM + row];
            df_add(hi[c], lo, s * f, e * f);
            lo_s[(col0 + c) * OZ_BM + row] = lo;
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(acc_empty);
      }
      if (ok && !*abort_flag && row < it.R) {
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int col = col0 + c;
          if (col < it.C) {
            const double v = f32_scaled_f64(hi[c], ebias) + f32_scaled_f64(lo_s[(col0 + c) * OZ_BM + row], ebias);
            double *d = P.out + it.out_base + (int64_t)row * it.ldo + col;
            if (it.split) atomicAdd(d, v);  // other K ranges of the tile add concurrently
            else *d += v;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.err, ERR_TIMEOUT);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static const EncodeTiledFn fn = [] {  // resolved once (thread-safe static initialisation)
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

// 3-D map over [slices][rows][Kpad] BF16, box (OZ_BK, box_rows, slices): rows of
// 64 bytes with the 64-byte swizzle the tcgen05 descriptors expect.
static int make_slices_map(CUtensorMap *m, const void *base, int64_t rows, int Kpad, int box_rows) {
  const int bk = OZ_BK;
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    snprintf(g_tc_err, sizeof g_tc_err, "cuTensorMapEncodeTiled unavailable");
    return MODAL_EUNSUPPORTED;
  }
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)OZ_SLICES};
  cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)rows * Kpad * 2};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, (cuuint32_t)OZ_SLICES};
  cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(g_tc_err, sizeof g_tc_err, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MODAL_EINVAL;
  }
  return MODAL_OK;
}

// Schedules of the slice products as MMA runs: mma_plan.h (host code).
static_assert(OZ_SLICES == plan::SLICES && OZ_MAXLEV == plan::MAXLEV && OZ_PLAN_MAX == plan::RUNS_MAX,
              "the schedules and the kernels agree on the slicing");
static void fill_mma_plans(uint32_t (&dst)[OZ_BN / 16][1 + OZ_PLAN_MAX]) {
  static uint32_t plans[OZ_BN / 16][1 + OZ_PLAN_MAX];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int i = 0; i < OZ_BN / 16; ++i) plan::mma_plan(16 * (i + 1), plans[i]);
  });
  memcpy(dst, plans, sizeof plans);
}

// B maps for the widths in `used` (bit i: 16 (i + 1) rows); the others stay zero
static int make_bmaps(BMaps *bm, const void *base, int64_t rows, int Kpad, unsigned used) {
  memset(bm, 0, sizeof *bm);
  for (int i = 0; i < OZ_BN / 16; ++i)
    if ((used >> i) & 1u)
      if (int r = make_slices_map(&bm->m[i], base, rows, Kpad, 16 * (i + 1))) return r;
  return MODAL_OK;
}

static size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch layout (fixed order, sized for the largest radial chunk):
//   [status words 1 KB][A slices][A exponents][B slices][B exponents][triple]
struct LScratch {
  int *words;
  __nv_bfloat16 *As, *Bs;
  int *eA, *eB;
  char *end;
};
static LScratch l_scratch(void *scratch, const SepShape &s, int nxc) {
  const int Kpad = cdiv(s.L, OZ_BK) * OZ_BK;
  const int nch = cdiv(s.L, OZ_KC);
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl, rowsB = (int64_t)nxc * s.nbp;
  LScratch r;
  char *w = (char *)scratch;
  r.words = (int *)w; w += 256 * 4;
  r.As = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * rowsA * Kpad * 2);
  r.eA = (int *)w; w += up256((size_t)nch * rowsA * 4);
  r.Bs = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * rowsB * Kpad * 2);
  r.eB = (int *)w; w += up256((size_t)nch * rowsB * 4);
  r.end = w;
  return r;
}

size_t tc_scratch_bytes(const SepShape &s, int nxl, int nxc, int variant) {
  LScratch r = l_scratch(nullptr, s, nxl);
  return (size_t)(r.end - (char *)nullptr) + tc_triple_scratch_bytes(s, nxc, variant) + 1024;
}

// Split the A operand of the l contraction (rows (j, a): w_l P_l(mu_j) q_a(l)),
// which does not depend on x: once per call.
int tc_prepare_l(const SepShape &s, const double *A, const double *q, void *scratch, int nxc_max, cudaStream_t st,
                 Profiler *prof, bool reset_status) {
  LScratch r = l_scratch(scratch, s, nxc_max);
  const int Kpad = cdiv(s.L, OZ_BK) * OZ_BK;
  const int nch = cdiv(s.L, OZ_KC);
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl;
  cudaError_t e;
  {
    ProfScope ps(prof, "tc_init", st);
    k_init_words<<<1, 32, 0, st>>>(r.words, reset_status ? 1 : 2);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  {
    ProfScope ps(prof, "tc_split_lA", st);
    k_split_lrows<true><<<(unsigned)cdiv64(rowsA * nch * 32, 256), 256, 0, st>>>(rowsA, s.L, Kpad, A, q, nullptr,
                                                                               s.nbl, s.nbp, 0, r.As, r.eA,
                                                                               r.words + 1, r.words);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  return MODAL_OK;
cuda_fail:
  snprintf(g_tc_err, sizeof g_tc_err, "l-contraction operand split: %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

// l contraction of one radial chunk (A prepared by tc_prepare_l).
int tc_contract_l(const SepShape &s, const double *qt, int x0, int nxc, int nxc_max, double *M, void *scratch,
                  long long wait_cycles, cudaStream_t st, Profiler *prof) {
  LScratch r = l_scratch(scratch, s, nxc_max);
  const int Kpad = cdiv(s.L, OZ_BK) * OZ_BK;
  const int nch = cdiv(s.L, OZ_KC);
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl, rowsB = (int64_t)nxc * s.nbp;
  cudaError_t e;
  {
    ProfScope ps(prof, "tc_init", st);
    k_init_words<<<1, 32, 0, st>>>(r.words, 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  {
    ProfScope ps(prof, "tc_split_lB", st);
    k_split_lrows<false><<<(unsigned)cdiv64(rowsB * nch * 32, 256), 256, 0, st>>>(rowsB, s.L, Kpad, nullptr,
                                                                                nullptr, qt, s.nbl, s.nbp, x0,
                                                                                r.Bs, r.eB, r.words + 2, r.words);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  {
    CUtensorMap ta;
    BMaps tb;
    if (int rr = make_slices_map(&ta, r.As, rowsA, Kpad, OZ_BM)) return rr;
    if (int rr = make_bmaps(&tb, r.Bs, rowsB, Kpad, 1u << (OZ_BN / 16 - 1))) return rr;
    OzParams P{};
    P.rowsA = rowsA;
    P.rowsB = rowsB;
    P.Kpad = Kpad;
    P.nchunks = nch;
    P.eA = r.eA;
    P.eB = r.eB;
    P.emaxA = r.words + 1;
    P.emaxB = r.words + 2;
    P.out = M;
    P.err = r.words;
    P.n_mu = s.n_mu;
    P.nbl = s.nbl;
    P.nbp = s.nbp;
    P.wait_cycles = wait_cycles;
    fill_mma_plans(P.plan);
    if ((e = cudaFuncSetAttribute(k_ozaki_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
        cudaSuccess)
      goto cuda_fail;
    // row tiles per CTA: a few, keeping at least ~4 waves of CTAs
    const int64_t nrt = cdiv64(rowsA, OZ_BM), nct = cdiv64(rowsB, OZ_BN);
    const int rpc = gridp::rows_per_cta(nrt, nct);
    P.rows_per_cta = rpc;
    dim3 grid((unsigned)nct, (unsigned)cdiv64(nrt, rpc));
    ProfScope ps(prof, "tc_gemm_l", st);
    k_ozaki_gemm<0><<<grid, OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  }
  return MODAL_OK;
cuda_fail:
  snprintf(g_tc_err, sizeof g_tc_err, "l contraction: %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

// ===========================================================================
// Triple product (Eq. 2D slice reduction) on the tensor cores.
//   A operand: Y rows (b, a, {u,v}) over all b, Y = w_k (M_au M_bv + M_av M_bu)
//              formed in double-FP32 from the FP64 M of the chunk, split with a
//              per-(row, K chunk) exponent from the bound
//              |Y| <= m_au m_bv + m_av m_bu,  m_au = max_k sqrt(w_k) |M_au(k)|;
//   B operand: M columns (c, t) transposed to K-major, exact per-chunk maxima;
//   output:    G block b (rows (a,{u,v}), columns (c,t) with c >= b), FP64 add.
// ===========================================================================
__device__ __forceinline__ f2 df_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  float s = p + e;
  return {s, e - (s - p)};
}
__device__ __forceinline__ f2 df_addv(f2 a, f2 b) {
  f2 s = df_two_sum(a.h, b.h);
  float e = s.l + a.l + b.l;
  float h = s.h + e;
  return {h, e - (h - s.h)};
}

__device__ __forceinline__ void split_df(f2 y, int e, __nv_bfloat16 (&out)[OZ_SLICES]) {
  split_f2(y.h, y.l, e, out);
}

// Column statistics of one chunk of M (FP64, [k][col]) for the triple product,
// in two passes over blocks of 32 columns:
//  * k_tp_col_max, 128 slices per block: max |M| and max |M~| (M~ = sqrt(w_k) M),
//    both from FP32-rounded values, combined by atomicMax on their bit patterns
//    (non-negative floats order like their bits) into colmax[2][nch][nblp];
//  * k_tp_split_cols, 32 slices per block: the per-(chunk, column) exponents
//    and bounds, M~ in double-FP32 (K-major, zero up to Kpad) for the Y
//    operand, and the five BF16 slices of M (K-major) for the B operand.
// w_k = om_j W_x for slice k = (x - x0) n_mu + j.
constexpr int TP_COLS = 32;
__global__ void __launch_bounds__(256) k_tp_col_max(int64_t K, int nblp, int n_mu, int x0,
                                                    const double *__restrict__ M, const double *__restrict__ om,
                                                    const double *__restrict__ xw, unsigned *__restrict__ colmax) {
  // |M| bounds serve both the projection and its |M| error-scale variant
  __shared__ float sw[128];
  __shared__ float red[2][8][TP_COLS];
  const int c0 = blockIdx.x * TP_COLS;
  const int64_t k0 = (int64_t)blockIdx.y * 128;
  const int tc = threadIdx.x & 31, tk = threadIdx.x >> 5;
  if (threadIdx.x < 128) {
    const int64_t k = k0 + threadIdx.x;
    sw[threadIdx.x] = k < K ? sqrtf(fabsf((float)(om[k % n_mu] * xw[x0 + k / n_mu]))) : 0.f;
  }
  __syncthreads();
  const int col = c0 + tc;
  float m1 = 0.f, m2 = 0.f;
  if (col < nblp) {
#pragma unroll 4
    for (int i = tk; i < 128; i += 8) {
      const int64_t k = k0 + i;
      if (k >= K) break;
      const float v = fabsf(__double2float_rn(M[k * nblp + col]));
      m1 = fmaxf(m1, v);
      m2 = fmaxf(m2, sw[i] * v);
    }
  }
  red[0][tk][tc] = m1;
  red[1][tk][tc] = m2;
  __syncthreads();
  if (tk == 0 && col < nblp) {
    for (int i = 1; i < 8; ++i) {
      m1 = fmaxf(m1, red[0][i][tc]);
      m2 = fmaxf(m2, red[1][i][tc]);
    }
    const int ch = (int)(k0 / OZ_KC), nch = (int)((K + OZ_KC - 1) / OZ_KC);
    // a NaN becomes +inf, which the range check of the next pass rejects
    atomicMax(colmax + (int64_t)ch * nblp + col, __float_as_uint(m1 == m1 ? m1 : INFINITY));
    atomicMax(colmax + ((int64_t)nch + ch) * nblp + col, __float_as_uint(m2 == m2 ? m2 : INFINITY));
  }
}

__global__ void __launch_bounds__(256) k_tp_split_cols(int64_t K, int Kpad, int nblp, int n_mu, int x0,
                                                       const double *__restrict__ M, const double *__restrict__ om,
                                                       const double *__restrict__ xw,
                                                       const unsigned *__restrict__ colmax, f2 *__restrict__ Mdf,
                                                       double *__restrict__ mxW, int *__restrict__ eB,
                                                       __nv_bfloat16 *__restrict__ Bt, int *__restrict__ emaxB,
                                                       int *__restrict__ err, int absM) {
  __shared__ double sw[32];
  __shared__ f2 swf[32];  // sqrt|w_k| as double-FP32
  __shared__ float sgn[32];
  __shared__ __nv_bfloat16 tile[OZ_SLICES][TP_COLS][32 + 8];
  __shared__ f2 mtile[TP_COLS][32 + 1];
  const int c0 = blockIdx.x * TP_COLS;
  const int64_t k0 = (int64_t)blockIdx.y * 32;
  const int ch = (int)(k0 / OZ_KC), nch = (int)((K + OZ_KC - 1) / OZ_KC);
  const int tc = threadIdx.x & 31, tk = threadIdx.x >> 5;  // 32 columns x 8 k-lanes (4 slices each)
  const int col = c0 + tc;
  if (threadIdx.x < 32) {
    // M~ = sqrt(|w_k|) M; the sign of w_k goes with the B slices of M, so that
    // Y B = |w| M M M sign(w) (absM: every M and weight by its magnitude)
    const int64_t k = k0 + threadIdx.x;
    const double w = k < K ? om[k % n_mu] * xw[x0 + k / n_mu] : 0.0;
    sw[threadIdx.x] = sqrt(fabs(w));
    swf[threadIdx.x] = df_from_d(sw[threadIdx.x]);
    sgn[threadIdx.x] = (w < 0.0 && !absM) ? -1.f : 1.f;
  }
  // the column's exponent for this chunk
  float m1 = 0.f, m2 = 0.f;
  if (col < nblp) {
    m1 = __uint_as_float(colmax[(int64_t)ch * nblp + col]);
    m2 = __uint_as_float(colmax[((int64_t)nch + ch) * nblp + col]);
  }
  // Y = M~ M~ + M~ M~ must stay inside the FP32 range of the double-FP32 form
  const bool bad = !(m1 < 1e37f) || !(m2 < 1e18f);
  if (bad) m1 = m2 = 0.f;
  const int e = exp_bound((double)m1);
  if ((k0 % OZ_KC) == 0 && tk == 0 && col < nblp) {
    if (bad) atomicOr(err, ERR_RANGE);
    // room for the FP32 roundings of the maxima (sqrt, product) and the low part of M~
    const double mw = (double)m2 * (1.0 + 1.0 / 262144.0);
    eB[(int64_t)ch * nblp + col] = e;
    mxW[(int64_t)ch * nblp + col] = mw;
    if (e > -99999) atomicMax(emaxB, e);
    const int ew = exp_bound(mw);
    if (ew > -99999) atomicMax(emaxB + 2, ew);  // words[5]: bound of max |M~|
  }
  __syncthreads();
  const SplitScale sc = split_scale(e);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int kk = tk * 4 + i;
    const int64_t k = k0 + kk;
    double v = (col < nblp && k < K) ? M[k * nblp + col] : 0.0;
    if (absM) v = fabs(v);
    const f2 vd = df_from_d_fast(v);
    __nv_bfloat16 o[OZ_SLICES];
    split_scaled(sgn[kk] * vd.h, sgn[kk] * vd.l, sc, o);
#pragma unroll
    for (int s = 0; s < OZ_SLICES; ++s) tile[s][tc][kk] = o[s];
    // M~ = sqrt|w| M in double-FP32 arithmetic (relative error ~2^-46, far
    // below the 2^-36 of the BF16 slicing)
    mtile[tc][kk] = df_mul(vd, swf[kk]);
  }
  __syncthreads();
  // B slices: per (slice, column) 64 contiguous bytes; M~: per column 256 bytes
  for (int idx = threadIdx.x; idx < OZ_SLICES * TP_COLS * 4; idx += 256) {
    const int part = idx & 3, cc = (idx >> 2) % TP_COLS, s = idx / (4 * TP_COLS);
    if (c0 + cc < nblp && k0 + part * 8 < Kpad) {
      const uint4 *src = reinterpret_cast<const uint4 *>(&tile[s][cc][part * 8]);
      uint4 *dst = reinterpret_cast<uint4 *>(Bt + ((int64_t)s * nblp + c0 + cc) * Kpad + k0 + part * 8);
      *dst = *src;
    }
  }
  for (int idx = threadIdx.x; idx < TP_COLS * 32; idx += 256) {
    const int kk = idx & 31, cc = idx >> 5;
    if (c0 + cc < nblp && k0 + kk < Kpad) Mdf[(int64_t)(c0 + cc) * Kpad + k0 + kk] = mtile[cc][kk];
  }
}

// Y rows: global row r -> (b, a, uv) with rows ordered by b, then a, then uv.
__device__ __forceinline__ void y_row_decode(int64_t r, int P2, int &b, int &a, int &u, int &v) {
  pair_decode((int)(r / P2), a, b);
  pair_decode((int)(r % P2), u, v);
}

// Per-(row, K chunk) exponents of the Y operand, from the bound
// |Y| <= m_au m_bv + m_av m_bu (FP64, once per row and chunk), and their
// maximum.  Rows are ordered by the layout's Y pairs (GLayout::y_pair), then
// by {u, v}.
__global__ void __launch_bounds__(256) k_tp_y_exp(GLayout g, int64_t rowsY, int nbp, int nblp, int P2,
                                                  const double *__restrict__ mxW, int *__restrict__ eY,
                                                  int *__restrict__ emaxY) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = blockIdx.y;
  int e = -100000;
  if (r < rowsY) {
    int a, b, u, v;
    g.y_pair((int)(r / P2), a, b);
    pair_decode((int)(r % P2), u, v);
    const double *mw = mxW + (int64_t)ch * nblp;
    e = exp_bound(mw[a * nbp + u] * mw[b * nbp + v] + mw[a * nbp + v] * mw[b * nbp + u]);
    eY[(int64_t)ch * rowsY + r] = e;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0 && e > -99999) atomicMax(emaxY, e);
}

// Y operand.  A block takes one pair a <= b and TY_K = 128 slices k (inside
// one chunk): it stages M~_a. and M~_b. for those k in shared memory, and
// warp w forms the rows (a, b, {u, v}) for u = w and u = 2W - 1 - w, ...
// (balanced: rows with u <= v).  Lane i holds k = 4i .. 4i + 3: per row it
// forms four values of Y = M~_au M~_bv + M~_av M~_bu in double-FP32 (w_k is
// folded into M~), splits them with the row's per-chunk scale and stores
// 8 bytes (four BF16) per slice: 256 contiguous bytes per warp and slice.
// The arithmetic runs on pairs of slices with the packed FP32x2 operations
// of sm_100+ (each component rounds exactly as its scalar counterpart).
// Shared layout per column: [k % 4 >= 2][k / 4][h, h', l, l'] (h, l of two
// consecutive k), so each 16-byte load of a lane is conflict-free and gives
// the high and low parts as register pairs.
constexpr int TY_K = 128, TY_WARPS = 10;
constexpr int TY_LD = 2 * TY_K + 4;  // floats per staged column (+ pad)
static_assert(OZ_KC % TY_K == 0, "a Y block stays inside one exact chunk");
__host__ __device__ inline size_t ty_smem_bytes(int nbp) {
  return (size_t)2 * nbp * TY_LD * sizeof(float) + (size_t)(nbp * (nbp + 1) / 2) * sizeof(float2);
}

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }

// double-FP32 values of M~_au M~_bv + M~_av M~_bu for two slices (high parts
// and unnormalised low parts)
__device__ __forceinline__ void y_value2(float2 auh, float2 aul, float2 bvh, float2 bvl, float2 avh, float2 avl,
                                         float2 buh, float2 bul, float2 &hsum, float2 &lsum) {
  const float2 p1 = __fmul2_rn(auh, bvh);
  float2 e1 = __ffma2_rn(auh, bvh, f2neg(p1));
  e1 = __ffma2_rn(auh, bvl, e1);
  e1 = __ffma2_rn(aul, bvh, e1);
  const float2 p2 = __fmul2_rn(avh, buh);
  float2 e2 = __ffma2_rn(avh, buh, f2neg(p2));
  e2 = __ffma2_rn(avh, bul, e2);
  e2 = __ffma2_rn(avl, buh, e2);
  hsum = __fadd2_rn(p1, p2);
  const float2 bb = f2sub(hsum, p1);
  const float2 t = __fadd2_rn(f2sub(p1, f2sub(hsum, bb)), f2sub(p2, bb));
  lsum = __fadd2_rn(t, __fadd2_rn(e1, e2));
}

// split_hl for two values at once
__device__ __forceinline__ void split_hl2(float2 H, float2 L, float2 (&q)[OZ_SLICES]) {
  float2 r = H;
#pragma unroll
  for (int s = 0; s < OZ_SLICES; ++s) {
    const float m = 1.5f * oz_pow2c(23 - OZ_BETA * s);
    const float2 m2 = make_float2(m, m);
    if (s == OZ_FOLD) r = __fadd2_rn(r, L);
    q[s] = f2sub(__fadd2_rn(r, m2), m2);
    if (s + 1 < OZ_SLICES) r = f2sub(r, q[s]);  // exact
  }
}

__device__ __forceinline__ uint32_t bf16x2_bits(float2 v) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t *>(&p);
}

__global__ void __launch_bounds__(32 * TY_WARPS) k_tp_make_y(GLayout g, int pair0, int64_t rowsY, int64_t K, int Kpad, int nbp, int nblp,
                                                         int P2, const f2 *__restrict__ Mdf,
                                                         const int *__restrict__ eY, __nv_bfloat16 *__restrict__ Ysl) {
  extern __shared__ __align__(16) unsigned char ty_sm[];
  float *Ms = reinterpret_cast<float *>(ty_sm);  // [2 nbp][TY_LD]: columns a*nbp+c, then b*nbp+c
  // per row of the pair: the scale 2^(BETA - e) as (2^k, 1) when it is a
  // normal float, else as two exact factors; (0, 0) for an all-zero row
  float2 *Fs = reinterpret_cast<float2 *>(ty_sm + (size_t)2 * nbp * TY_LD * sizeof(float));
  int a, b;
  const int jp = pair0 + (int)blockIdx.x;  // the block's Y pair of the layout
  g.y_pair(jp, a, b);
  const int64_t row0 = (int64_t)jp * P2;
  const int64_t kb = (int64_t)blockIdx.y * TY_K;
  const int ch = (int)(kb / OZ_KC);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  (void)K;
  (void)nblp;
  const int nc2 = 2 * nbp;
  // staging: thread (column cc, lane group g) moves the four slices 4g .. 4g + 3
  // (M~ is K-major and zero beyond K up to Kpad)
  for (int idx = threadIdx.x; idx < nc2 * 32; idx += blockDim.x) {
    const int g = idx & 31, cc = idx >> 5;
    const int col = cc < nbp ? a * nbp + cc : b * nbp + (cc - nbp);
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (kb + 4 * g < Kpad) {
      const float4 *src = reinterpret_cast<const float4 *>(Mdf + (int64_t)col * Kpad + kb + 4 * g);
      lo = src[0];  // (h0, l0, h1, l1)
      hi = src[1];  // (h2, l2, h3, l3)
    }
    *reinterpret_cast<float4 *>(&Ms[cc * TY_LD + 4 * g]) = make_float4(lo.x, lo.z, lo.y, lo.w);
    *reinterpret_cast<float4 *>(&Ms[cc * TY_LD + TY_K + 4 * g]) = make_float4(hi.x, hi.z, hi.y, hi.w);
  }
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    const int e = eY[(int64_t)ch * rowsY + row0 + i];
    const int k = OZ_BETA - e;
    float2 f;
    if (e < -99999) f = make_float2(0.f, 0.f);
    else if (k >= -126 && k <= 127) f = make_float2(pow2f(k), 1.f);
    else f = make_float2(pow2f(k / 2), pow2f(k - k / 2));
    Fs[i] = f;
  }
  __syncthreads();
  const bool kvalid = kb + 4 * lane < Kpad;  // Kpad is a multiple of 64, not of 128
  const int64_t sstride = rowsY * (int64_t)Kpad / 4;  // 8-byte words per slice
  uint2 *Yq = reinterpret_cast<uint2 *>(Ysl) + (kb + 4 * lane) / 4;
  const int64_t rstride = Kpad / 4;
  const int tend = (int)cdiv(nbp, TY_WARPS) * TY_WARPS;
  const int o0 = 4 * lane, o1 = TY_K + 4 * lane;
  for (int t = warp; t < tend; t += TY_WARPS) {
    // balanced pairing of u: w, 2W-1-w, 2W+w, ...
    const int blk = t / TY_WARPS, wi = t % TY_WARPS;
    const int u = blk * TY_WARPS + ((blk & 1) ? (TY_WARPS - 1 - wi) : wi);
    if (u >= nbp) continue;
    // (h, h', l, l') of slices (k0, k1) and (k2, k3) of the lane
    const float4 au0 = *reinterpret_cast<const float4 *>(&Ms[u * TY_LD + o0]);
    const float4 au1 = *reinterpret_cast<const float4 *>(&Ms[u * TY_LD + o1]);
    const float4 bu0 = *reinterpret_cast<const float4 *>(&Ms[(nbp + u) * TY_LD + o0]);
    const float4 bu1 = *reinterpret_cast<const float4 *>(&Ms[(nbp + u) * TY_LD + o1]);
    for (int v = u; v < nbp; ++v) {
      const float4 av0 = *reinterpret_cast<const float4 *>(&Ms[v * TY_LD + o0]);
      const float4 av1 = *reinterpret_cast<const float4 *>(&Ms[v * TY_LD + o1]);
      const float4 bv0 = *reinterpret_cast<const float4 *>(&Ms[(nbp + v) * TY_LD + o0]);
      const float4 bv1 = *reinterpret_cast<const float4 *>(&Ms[(nbp + v) * TY_LD + o1]);
      const int uv = v * (v + 1) / 2 + u;
      const float2 f = Fs[uv];
      float2 h01, l01, h23, l23;
      y_value2(make_float2(au0.x, au0.y), make_float2(au0.z, au0.w), make_float2(bv0.x, bv0.y),
               make_float2(bv0.z, bv0.w), make_float2(av0.x, av0.y), make_float2(av0.z, av0.w),
               make_float2(bu0.x, bu0.y), make_float2(bu0.z, bu0.w), h01, l01);
      y_value2(make_float2(au1.x, au1.y), make_float2(au1.z, au1.w), make_float2(bv1.x, bv1.y),
               make_float2(bv1.z, bv1.w), make_float2(av1.x, av1.y), make_float2(av1.z, av1.w),
               make_float2(bu1.x, bu1.y), make_float2(bu1.z, bu1.w), h23, l23);
      const float2 fx = make_float2(f.x, f.x);
      h01 = __fmul2_rn(h01, fx);
      l01 = __fmul2_rn(l01, fx);
      h23 = __fmul2_rn(h23, fx);
      l23 = __fmul2_rn(l23, fx);
      if (f.y != 1.f) {  // second factor (warp-uniform: every lane has the same row)
        const float2 fy = make_float2(f.y, f.y);
        h01 = __fmul2_rn(h01, fy);
        l01 = __fmul2_rn(l01, fy);
        h23 = __fmul2_rn(h23, fy);
        l23 = __fmul2_rn(l23, fy);
      }
      float2 q01[OZ_SLICES], q23[OZ_SLICES];
      split_hl2(h01, l01, q01);
      split_hl2(h23, l23, q23);
      if (kvalid) {
        uint2 *dst = Yq + (row0 + uv) * rstride;
#pragma unroll
        for (int sl = 0; sl < OZ_SLICES; ++sl) dst[sl * sstride] = make_uint2(bf16x2_bits(q01[sl]), bf16x2_bits(q23[sl]));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fused triple product: the eight producer/epilogue warps form the Y operand
// (double-FP32 products of M entries, split into BF16 slices) directly in
// the 64-byte-swizzled shared-memory stage that the tensor core reads, so Y
// never goes through HBM; the B operand (M slices) comes by TMA.
//   warp 0: TMA for B;  warp 1: TMEM allocation and MMA issue;
//   warps 2-9: produce Y stages, and drain the accumulators of chunk c while
//              producing chunk c+1 (after OZ_STAGES stages of it).
// ---------------------------------------------------------------------------
struct FusedParams {
  int64_t rowsB;  // B operand rows (nb_late * nb_prim)
  int Kpad;
  int64_t K;      // valid slices of this launch
  int nchunks, nbp, nblp, P2;
  const f2 *Mdf;     // [nblp][Kpad]: sqrt(w_k) M in double-FP32, K-major
  const double *mxW; // [nchunks][nblp]
  const int *eB;     // [nchunks][nblp]
  const int *emaxB;  // max of eB
  const int *emaxW;  // exponent bound of max mxW
  double *G;
  GLayout g;
  int *err;
  long long wait_cycles;
  int chunks_per_split;  // K chunks per CTA along blockIdx.y (split-K)
  int split_k;           // number of K splits (> 1: FP64 atomic adds into G)
};

__device__ __forceinline__ int y_exp(const double *mw, int nbp, int a, int b, int u, int v) {
  return exp_bound(mw[a * nbp + u] * mw[b * nbp + v] + mw[a * nbp + v] * mw[b * nbp + u]);
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_triple_fused(const __grid_constant__ CUtensorMap tmB, FusedParams P) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  float *lo_s = (float *)(sm + OZ_STAGES * OZ_STAGE_BYTES);  // [col][row]
  uint64_t *full = (uint64_t *)(sm + OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES);
  uint64_t *empty = full + OZ_STAGES;
  uint64_t *acc_full = empty + OZ_STAGES;
  uint64_t *acc_empty = acc_full + 1;
  uint64_t *mma_done = acc_empty + 1;
  uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NPROD = 32 * OZ_EPI_WARPS;  // 256 producer threads

  // ---- tile of the G block ----
  int t = blockIdx.x, rt = 0, ct = 0, bblk;
  int64_t rowoff = 0;
  for (bblk = 0; bblk < P.g.nbl; ++bblk) {
    const int nrt = (int)cdiv64(P.g.rows(bblk), OZ_BM), nct = (int)cdiv64(P.g.cols(bblk), OZ_BN);
    if (t < nrt * nct) {
      rt = t / nct;
      ct = t % nct;
      break;
    }
    t -= nrt * nct;
    rowoff += P.g.rows(bblk);
  }
  if (bblk >= P.g.nbl) return;
  const int64_t a_row0 = rowoff + (int64_t)rt * OZ_BM;  // global Y row of the tile start
  const int64_t b_row0 = P.g.colstart(bblk) + (int64_t)ct * OZ_BN;
  const int64_t R = min((int64_t)OZ_BM, P.g.rows(bblk) - (int64_t)rt * OZ_BM);
  const int64_t C = min((int64_t)OZ_BN, P.g.cols(bblk) - (int64_t)ct * OZ_BN);
  const int64_t out_base = P.g.offset(bblk) + (int64_t)rt * OZ_BM * P.g.cols(bblk) + (int64_t)ct * OZ_BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1 + NPROD);  // TMA expect_tx arrival + every producer
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, NPROD);
    ptx::mbar_init(mma_done, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int steps_per_chunk = OZ_KC / OZ_BK;
  // this CTA's K range: chunks [c_lo, c_hi), stages [i_lo, i_hi)
  const int c_lo = blockIdx.y * P.chunks_per_split;
  const int c_hi = min(P.nchunks, c_lo + P.chunks_per_split);
  const int i_lo = c_lo * steps_per_chunk;
  const int i_hi = min(P.Kpad / OZ_BK, c_hi * steps_per_chunk);
  const int nloc = c_hi - c_lo;  // chunks of this CTA

  if (warp == 0) {
    // ================= TMA producer (B operand) =================
    if (lane == 0) {
      ptx::prefetch_tmap(&tmB);
      int issued = 0;
      for (int i = i_lo; i < i_hi; ++i) {
        const int s = (i - i_lo) % OZ_STAGES;
        const uint32_t ph = (uint32_t)(((i - i_lo) / OZ_STAGES) & 1);
        if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) break;
        ptx::mbar_arrive_expect_tx(&full[s], OZ_B_BYTES);
        ptx::tma_load_3d(sm + s * OZ_STAGE_BYTES + OZ_A_BYTES, &tmB, &full[s], i * OZ_BK, (int)b_row0, 0);
        ++issued;
      }
      if (*abort_flag) {  // let the copies in flight land before the CTA ends
        for (int j = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); j < issued; ++j) {
          volatile int dummy = 0;
          ptx::mbar_wait(&full[j % OZ_STAGES], (uint32_t)((j / OZ_STAGES) & 1), &dummy, OZ_WAIT_CYCLES);
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(OZ_BM, OZ_BN);
      const uint32_t sbase = ptx::smem_u32(sm);
      int chunk = 0;  // local chunk count
      for (int i = i_lo; i < i_hi; ++i) {
        const int s = (i - i_lo) % OZ_STAGES;
        const uint32_t ph = (uint32_t)(((i - i_lo) / OZ_STAGES) & 1);
        const bool chunk_start = (i % steps_per_chunk) == 0;
        if (chunk_start && chunk > 0) {
          if (!ptx::mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), abort_flag, P.wait_cycles)) break;
        }
        if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) break;
        ptx::tc_fence_after();
        const uint32_t a0 = sbase + s * OZ_STAGE_BYTES;
        const uint64_t ad0 = ptx::smem_desc(a0, 16, 8 * OZ_ROWB, ptx::SW_64B);
        const uint64_t bd0 = ptx::smem_desc(a0 + OZ_A_BYTES, 16, 8 * OZ_ROWB, ptx::SW_64B);
        bool fresh[3] = {chunk_start, chunk_start, chunk_start};
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
          for (int sa = 0; sa < OZ_SLICES; ++sa) {
#pragma unroll
            for (int sb = 0; sb < OZ_SLICES; ++sb) {
              if (sa + sb > OZ_MAXLEV) continue;
              const int lev = sa + sb < 2 ? sa + sb : 2;
              const uint64_t ad = ad0 + (uint64_t)((sa * OZ_BM * OZ_ROWB + kk * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((sb * OZ_BN * OZ_ROWB + kk * 32) >> 4);
              ptx::mma_bf16(tmem + lev * OZ_BN, ad, bd, idesc, fresh[lev] ? 0u : 1u);
              fresh[lev] = false;
            }
          }
        }
        ptx::mma_commit(&empty[s]);
        const bool chunk_end = ((i + 1) % steps_per_chunk) == 0 || i + 1 == i_hi;
        if (chunk_end) {
          ptx::mma_commit(acc_full);
          ++chunk;
        }
      }
      ptx::mma_commit(mma_done);
      volatile int dummy = 0;
      ptx::mbar_wait(mma_done, 0, &dummy, OZ_WAIT_CYCLES);
    }
  } else {
    // ================= Y producers + accumulator drains =================
    const int tp = threadIdx.x - 64;  // 0..255
    // production role: row prow of the tile, 16 of the 32 k of each stage
    const int prow = tp & (OZ_BM - 1), khalf = tp >> 7;
    const bool pvalid = prow < R;
    int pa = 0, pb = 0, pu = 0, pv = 0;
    if (pvalid) y_row_decode(a_row0 + prow, P.P2, pb, pa, pu, pv);
    const int o_au = pa * P.nbp + pu, o_bv = pb * P.nbp + pv, o_av = pa * P.nbp + pv, o_bu = pb * P.nbp + pu;
    const uint32_t swz = (uint32_t)((prow >> 1) & 3);
    // drain role: TMEM lane quarter of this warp, one half of the columns
    const int quarter = warp & 3, chalf = (warp - 2) >> 2;
    const int erow = quarter * 32 + lane, col0 = chalf * 64;
    const bool evalid = erow < R;
    int ea_a = 0, ea_b = 0, ea_u = 0, ea_v = 0;
    if (evalid) y_row_decode(a_row0 + erow, P.P2, ea_b, ea_a, ea_u, ea_v);
    const int ebias = 2 * (*P.emaxW) + 1 + (*P.emaxB) + 40;
    float hi[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) {
      hi[c] = 0.f;
      lo_s[(col0 + c) * OZ_BM + erow] = 0.f;
    }
    const uint32_t sbase = ptx::smem_u32(sm);
    int drained = 0, e_row = -100000;
    bool ok = true;

    // drain local chunk lc (global chunk c_lo + lc)
    auto drain = [&](int lc) -> bool {
      const int ch = c_lo + lc;
      if (!ptx::mbar_wait(acc_full, (uint32_t)(lc & 1), abort_flag, P.wait_cycles)) return false;
      ptx::tc_fence_after();
      const int ea = evalid ? y_exp(P.mxW + (int64_t)ch * P.nblp, P.nbp, ea_a, ea_b, ea_u, ea_v) : -100000;
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < 16; ++cb) {
        float v0[4], v1[4], v2[4];
        const uint32_t cc = (uint32_t)(col0 + cb * 4);
        ptx::tmem_ld4(tl + cc, v0);
        ptx::tmem_ld4(tl + OZ_BN + cc, v1);
        ptx::tmem_ld4(tl + 2 * OZ_BN + cc, v2);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = cb * 4 + k;
          const int64_t bcol = b_row0 + col0 + c;
          const int eb = (bcol < P.rowsB) ? __ldg(P.eB + (int64_t)ch * P.rowsB + bcol) : -100000;
          if (ea < -99999 || eb < -99999) continue;
          float sv = v0[k] + v1[k];
          float bb = sv - v0[k];
          float ev = (v0[k] - (sv - bb)) + (v1[k] - bb);
          ev += v2[k];
          const int sh = ea + eb - 2 * OZ_BETA - ebias;
          const float f1 = pow2f(sh / 2), f2v = pow2f(sh - sh / 2);
          float lo = lo_s[(col0 + c) * OZ_BM + erow];
          df_add(hi[c], lo, (sv * f1) * f2v, (ev * f1) * f2v);
          lo_s[(col0 + c) * OZ_BM + erow] = lo;
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(acc_empty);
      return true;
    };

    for (int i = i_lo; i < i_hi && ok; ++i) {
      const int ch = i / steps_per_chunk, lc = ch - c_lo;
      if (i % steps_per_chunk == 0) {
        e_row = pvalid ? y_exp(P.mxW + (int64_t)ch * P.nblp, P.nbp, pa, pb, pu, pv) : -100000;
      }
      if (lc >= 1 && i % steps_per_chunk == OZ_STAGES && drained == lc - 1) {
        if (!drain(lc - 1)) { ok = false; break; }
        drained = lc;
      }
      const int s = (i - i_lo) % OZ_STAGES;
      const uint32_t ph = (uint32_t)(((i - i_lo) / OZ_STAGES) & 1);
      if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) { ok = false; break; }
      const uint32_t abase = sbase + s * OZ_STAGE_BYTES + prow * OZ_ROWB;
#pragma unroll
      for (int g = 0; g < 2; ++g) {  // two 16-byte granules (8 k each) of this thread
        uint32_t pk[OZ_SLICES][4];
#pragma unroll
        for (int kk = 0; kk < 8; kk += 2) {
          __nv_bfloat16 o0[OZ_SLICES], o1[OZ_SLICES];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int64_t kg = (int64_t)i * OZ_BK + khalf * 16 + g * 8 + kk + h2;
            f2 y = {0.f, 0.f};
            if (pvalid && kg < P.K) {
              const f2 *Mk = P.Mdf + kg;  // K-major: column o at Mk[o * Kpad]
              const int64_t ld = P.Kpad;
              // M~ = sqrt(w) M already carries the slice weight
              y = df_addv(df_mul(Mk[o_au * ld], Mk[o_bv * ld]), df_mul(Mk[o_av * ld], Mk[o_bu * ld]));
            }
            if (h2 == 0) split_f2(y.h, y.l, e_row, o0);
            else split_f2(y.h, y.l, e_row, o1);
          }
#pragma unroll
          for (int sl = 0; sl < OZ_SLICES; ++sl)
            pk[sl][kk / 2] = (uint32_t)__bfloat16_as_ushort(o0[sl]) | ((uint32_t)__bfloat16_as_ushort(o1[sl]) << 16);
        }
        const uint32_t gran = (uint32_t)(khalf * 2 + g) ^ swz;
#pragma unroll
        for (int sl = 0; sl < OZ_SLICES; ++sl)
          ptx::st_shared_v4(abase + sl * OZ_BM * OZ_ROWB + (gran << 4), pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
      }
      ptx::fence_proxy_async_smem();
      ptx::mbar_arrive(&full[s]);
    }
    // chunks not drained inside the loop (the last one or two)
    for (int lc = drained; ok && lc < nloc; ++lc) {
      if (!drain(lc)) { ok = false; break; }
    }
    if (ok && !*abort_flag && evalid) {
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        const int col = col0 + c;
        if (col >= C) continue;
        const double v = f32_scaled_f64(hi[c], ebias) + f32_scaled_f64(lo_s[col * OZ_BM + erow], ebias);
        double *d = P.G + out_base + (int64_t)erow * P.g.cols(bblk) + col;
        if (P.split_k > 1) atomicAdd(d, v);
        else *d += v;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.err, ERR_TIMEOUT);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// Fused triple product, second form.  Sixteen warps form the Y operand of
// each K step in the GEMM's own shared-memory stage, from a TMA-staged tile of
// the M~ rows the tile needs (groups a_first..a_last and b, K-major), and
// drain the accumulators with their double-FP32 running sums in registers
// (32 columns per thread), which leaves room for two 96 KB stages.
//   warp 0: TMA (B slices of M, M~ groups);  warp 1: TMEM and MMA issue;
//   warps 2-17: Y production (4 (row, slice pair) tasks per thread and K
//   step, packed FP32x2 arithmetic) and the chunk drains.
// Y rows of the tile whose pair lies outside the block are written as zero.
// ---------------------------------------------------------------------------
constexpr int F2_WARPS = 16;
constexpr int F2_THREADS = 64 + 32 * F2_WARPS;
constexpr int F2_MT_BYTES = 16 * 1024;            // M~ groups of one stage: <= 64 columns x 32 slices x 8 B
constexpr int F2_MAX_COLS = F2_MT_BYTES / 256;
constexpr int F2_STAGE = OZ_A_BYTES + OZ_B_BYTES + F2_MT_BYTES;
constexpr int F2_SMEM = OZ_STAGES * F2_STAGE + 1024 /*align*/ + 256 /*barriers*/;
static_assert(F2_SMEM <= 232448, "shared memory per CTA");
static_assert(OZ_BK == 32, "one K step = 32 slices = 16 slice pairs");

struct Fused2Params {
  uint32_t plan[OZ_BN / 16][1 + OZ_PLAN_MAX];
  int64_t rowsB;      // nb_late * nb_prim (columns of M)
  int64_t rowsY;      // rows of the full Y operand (for eY)
  int Kpad, nchunks, nbp;
  const int *eY;      // [nchunks][rowsY] row exponents of Y
  const int *eB;      // [nchunks][rowsB]
  const int *emaxY, *emaxB;
  double *G;
  GLayout g;
  int *err;
  long long wait_cycles;
};

// Number of M~ groups of the tile (distinct a of its rows, plus b).
__host__ __device__ inline int f2_groups(const GLayout &g, int b, int rt) {
  const int64_t r0 = (int64_t)rt * OZ_BM;
  const int64_t r1 = min(g.rows(b), r0 + OZ_BM) - 1;
  return (int)(r1 / g.P2 - r0 / g.P2) + 2;
}

__global__ void __launch_bounds__(F2_THREADS, 1)
    k_ozaki_triple_fused2(const __grid_constant__ CUtensorMap tmM, const __grid_constant__ BMaps bmaps,
                          Fused2Params P) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(sm + OZ_STAGES * F2_STAGE);  // TMA: B and M~ landed
  uint64_t *fullA = full + OZ_STAGES;                         // producers: Y written
  uint64_t *empty = fullA + OZ_STAGES;                        // MMAs of the stage retired
  uint64_t *acc_full = empty + OZ_STAGES;
  uint64_t *acc_empty = acc_full + 1;
  uint64_t *mma_done = acc_empty + 1;
  uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NPROD = 32 * F2_WARPS;

  // ---- tile of the G block (as in k_ozaki_gemm<1>) ----
  int t = blockIdx.x, rt = 0, ct = 0, bblk;
  int64_t rowoff = 0;
  for (bblk = 0; bblk < P.g.nbl; ++bblk) {
    const int nrt = (int)cdiv64(P.g.rows(bblk), OZ_BM), nct = (int)cdiv64(P.g.cols(bblk), OZ_BN);
    if (t < nrt * nct) {
      rt = t / nct;
      ct = t % nct;
      break;
    }
    t -= nrt * nct;
    rowoff += P.g.rows(bblk);
  }
  if (bblk >= P.g.nbl) return;
  const int ntile = g_tile_width(P.g.cols(bblk));
  const int64_t lrow0 = (int64_t)rt * OZ_BM;       // first row of the tile inside block b
  const int64_t a_row0 = rowoff + lrow0;           // ... in the full Y row order
  const int64_t b_row0 = P.g.colstart(bblk) + (int64_t)ct * ntile;
  const int64_t R = min((int64_t)OZ_BM, P.g.rows(bblk) - lrow0);
  const int64_t C = min((int64_t)ntile, P.g.cols(bblk) - (int64_t)ct * ntile);
  const int64_t out_base = P.g.offset(bblk) + lrow0 * P.g.cols(bblk) + (int64_t)ct * ntile;
  const int nbp = P.nbp, P2 = P.g.P2;
  const int a_first = (int)(lrow0 / P2);
  const int ngrp = f2_groups(P.g, bblk, rt);     // groups a_first .. a_first + ngrp - 2, then b
  const CUtensorMap *tmB = &bmaps.m[ntile / 16 - 1];
  const uint32_t stage_bytes = (uint32_t)(OZ_SLICES * ntile * OZ_ROWB + ngrp * nbp * 256);

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&fullA[s], NPROD);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, NPROD);
    ptx::mbar_init(mma_done, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksteps = P.Kpad / OZ_BK;
  const int steps_per_chunk = OZ_KC / OZ_BK;

  if (warp == 0) {
    // ================= TMA: B slices and the M~ groups =================
    if (lane == 0) {
      ptx::prefetch_tmap(tmB);
      ptx::prefetch_tmap(&tmM);
      int issued = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % OZ_STAGES;
        const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
        if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) break;
        unsigned char *st = sm + s * F2_STAGE;
        ptx::mbar_arrive_expect_tx(&full[s], stage_bytes);
        ptx::tma_load_3d(st + OZ_A_BYTES, tmB, &full[s], i * OZ_BK, (int)b_row0, 0);
        unsigned char *mt = st + OZ_A_BYTES + OZ_B_BYTES;
        for (int gidx = 0; gidx < ngrp; ++gidx) {
          const int grow = (gidx == ngrp - 1 ? bblk : a_first + gidx) * nbp;
          ptx::tma_load_2d(mt + gidx * nbp * 256, &tmM, &full[s], i * OZ_BK, grow);
        }
        ++issued;
      }
      if (*abort_flag) {  // let the copies in flight land before the CTA ends
        for (int j = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); j < issued; ++j) {
          volatile int dummy = 0;
          ptx::mbar_wait(&full[j % OZ_STAGES], (uint32_t)((j / OZ_STAGES) & 1), &dummy, OZ_WAIT_CYCLES);
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issue (runs of slice products, see mma_plans) =================
    if (lane == 0) {
      const uint32_t idesc0 = ptx::idesc_bf16_f32(OZ_BM, 0);
      const uint32_t *plan = P.plan[ntile / 16 - 1];  // read from the parameter space per MMA
      const int nruns = (int)(plan[0] & 0xffu);
      const uint32_t sbase = ptx::smem_u32(sm);
      int chunk = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % OZ_STAGES;
        const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
        const bool chunk_start = (i % steps_per_chunk) == 0;
        if (chunk_start && chunk > 0) {
          if (!ptx::mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), abort_flag, P.wait_cycles)) break;
        }
        if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) break;
        if (!ptx::mbar_wait(&fullA[s], ph, abort_flag, P.wait_cycles)) break;
        ptx::tc_fence_after();
        const uint32_t a0 = sbase + s * F2_STAGE;
        const uint64_t ad0 = ptx::smem_desc(a0, 16, 8 * OZ_ROWB, ptx::SW_64B);
        const uint64_t bd0 = ptx::smem_desc(a0 + OZ_A_BYTES, 16, 8 * OZ_ROWB, ptx::SW_64B);
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
          for (int r = 0; r < nruns; ++r) {
            const uint32_t e = plan[1 + r];
            const uint32_t sa = e & 15u, sb = (e >> 4) & 15u, n = (e >> 8) & 15u, acc = (e >> 12) & 15u;
            const bool first = chunk_start && kk == 0 && ((e >> 16) & 1u);
            const uint32_t N = n * (uint32_t)ntile;
            const uint64_t ad = ad0 + (uint64_t)((sa * OZ_BM * OZ_ROWB + kk * 32) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((sb * (uint32_t)ntile * OZ_ROWB + kk * 32) >> 4);
            ptx::mma_bf16(tmem + acc * (uint32_t)ntile, ad, bd, idesc0 | ((N >> 3) << 17), first ? 0u : 1u);
          }
        }
        ptx::mma_commit(&empty[s]);
        const bool chunk_end = ((i + 1) % steps_per_chunk) == 0 || i + 1 == ksteps;
        if (chunk_end) {
          ptx::mma_commit(acc_full);
          ++chunk;
        }
      }
      ptx::mma_commit(mma_done);
      volatile int dummy = 0;
      ptx::mbar_wait(mma_done, 0, &dummy, OZ_WAIT_CYCLES);
    }
  } else {
    // ================= Y production and drains =================
    const int pw = warp - 2;                    // producer warp 0..15
    const int kp = lane & 15;                   // slice pair of the K step (slices 2kp, 2kp+1)
    // rows of this thread: 32 j + 2 pw + (lane >> 4), j = 0..3; per row the
    // M~ tile columns of (a,u), (b,v), (a,v), (b,u), one byte each
    uint32_t cols4[4];
    unsigned rmask = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = 32 * j + 2 * pw + (lane >> 4);
      const int64_t lr = lrow0 + r;
      int a = a_first, u = 0, v = 0;
      if (r < R) {
        rmask |= 1u << j;
        a = (int)(lr / P2);
        pair_decode((int)(lr % P2), u, v);
      }
      const int ga = (a - a_first) * nbp, gb = (ngrp - 1) * nbp;
      cols4[j] = (uint32_t)(ga + u) | (uint32_t)(gb + v) << 8 | (uint32_t)(ga + v) << 16 | (uint32_t)(gb + u) << 24;
    }
    // drain role: TMEM lane quarter of this warp, one quarter of the columns
    const int quarter = warp & 3, cq = pw >> 2;
    const int erow = quarter * 32 + lane, col0 = cq * 32;
    const int emA = *P.emaxY, emB = *P.emaxB;
    const int ebias = emA + emB + 40;
    const int nacc = (int)((P.plan[ntile / 16 - 1][0] >> 8) & 0xffu);
    float hi[32], lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.f;
    int rexp[4];  // per-row exponent of the current chunk
    const uint32_t sbase = ptx::smem_u32(sm);
    int drained = 0;
    bool ok = true;

    auto drain = [&](int ch) -> bool {
      const bool got = ptx::mbar_wait(acc_full, (uint32_t)(ch & 1), abort_flag, P.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) return false;
      ptx::tc_fence_after();
      const int ea = (erow < R) ? P.eY[(int64_t)ch * P.rowsY + a_row0 + erow] : -100000;
      const float fa = pow2f_or0(ea - emA);
      const int64_t bcol = b_row0 + col0 + lane;
      const int eb = (col0 + lane < ntile && bcol < P.rowsB) ? __ldg(P.eB + (int64_t)ch * P.rowsB + bcol)
                                                             : -100000;
      const float fbl = pow2f_or0(eb - emB - 2 * OZ_BETA - 40);
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < 8; ++cb) {
        if (col0 + cb * 4 >= ntile) break;  // warp-uniform
        float v0[4], v1[4], v2[4], v3[4], v4[4];
        const uint32_t cc = (uint32_t)(col0 + cb * 4);
        const uint32_t w = (uint32_t)ntile;
        ptx::tmem_ld4(tl + cc, v0);
        ptx::tmem_ld4(tl + w + cc, v1);
        ptx::tmem_ld4(tl + 2 * w + cc, v2);
        if (nacc > 3) ptx::tmem_ld4(tl + 3 * w + cc, v3);
        if (nacc > 4) ptx::tmem_ld4(tl + 4 * w + cc, v4);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = cb * 4 + k;
          float rest = v2[k];
          if (nacc > 3) rest += v3[k];
          if (nacc > 4) rest += v4[k];
          const float f = fa * __shfl_sync(0xffffffffu, fbl, c);
          float s = v0[k] + v1[k];
          float bb = s - v0[k];
          float e = (v0[k] - (s - bb)) + (v1[k] - bb);
          e += rest;
          df_add(hi[c], lo[c], s * f, e * f);
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(acc_empty);
      return true;
    };

    for (int i = 0; i < ksteps && ok; ++i) {
      const int ch = i / steps_per_chunk, ic = i % steps_per_chunk;
      if (ch >= 1 && ic == OZ_STAGES && drained == ch - 1) {
        if (!drain(ch - 1)) { ok = false; break; }
        drained = ch;
      }
      if (ic == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = 32 * j + 2 * pw + (lane >> 4);
          rexp[j] = ((rmask >> j) & 1u) ? P.eY[(int64_t)ch * P.rowsY + a_row0 + r] : -100000;
        }
      }
      const int s = i % OZ_STAGES;
      const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
      bool got = ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles);
      if (got) got = ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }  // the warp goes on or stops together
      const float4 *mt = reinterpret_cast<const float4 *>(sm + s * F2_STAGE + OZ_A_BYTES + OZ_B_BYTES);
      const uint32_t abase = sbase + s * F2_STAGE;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 32 * j + 2 * pw + (lane >> 4);
        float2 q[OZ_SLICES];
        if ((rmask >> j) & 1u) {
          // (h, l, h', l') of slices 2kp and 2kp+1 of each factor
          const uint32_t cj = cols4[j];
          const float4 au = mt[(cj & 255u) * 16 + kp], bv = mt[((cj >> 8) & 255u) * 16 + kp];
          const float4 av = mt[((cj >> 16) & 255u) * 16 + kp], bu = mt[(cj >> 24) * 16 + kp];
          float2 hy, ly;
          y_value2(make_float2(au.x, au.z), make_float2(au.y, au.w), make_float2(bv.x, bv.z),
                   make_float2(bv.y, bv.w), make_float2(av.x, av.z), make_float2(av.y, av.w),
                   make_float2(bu.x, bu.z), make_float2(bu.y, bu.w), hy, ly);
          // scale 2^(BETA - e) as two exact factors (0 for an all-zero row)
          const int e = rexp[j], k = OZ_BETA - e;
          const float f1 = e < -99999 ? 0.f : pow2f(k / 2), f2v = e < -99999 ? 0.f : pow2f(k - k / 2);
          const float2 fx = make_float2(f1, f1), fy = make_float2(f2v, f2v);
          hy = __fmul2_rn(__fmul2_rn(hy, fx), fy);
          ly = __fmul2_rn(__fmul2_rn(ly, fx), fy);
          split_hl2(hy, ly, q);
        } else {
#pragma unroll
          for (int sl = 0; sl < OZ_SLICES; ++sl) q[sl] = make_float2(0.f, 0.f);
        }
        // 64-byte swizzled row of each slice: granule kp/4 ^ ((r >> 1) & 3)
        const uint32_t gran = (uint32_t)((kp >> 2) ^ ((r >> 1) & 3));
        const uint32_t addr = abase + (uint32_t)r * OZ_ROWB + (gran << 4) + (uint32_t)(kp & 3) * 4;
#pragma unroll
        for (int sl = 0; sl < OZ_SLICES; ++sl)
          asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr + sl * OZ_BM * OZ_ROWB), "r"(bf16x2_bits(q[sl]))
                       : "memory");
      }
      ptx::fence_proxy_async_smem();
      ptx::mbar_arrive(&fullA[s]);
    }
    const int nch = P.nchunks;
    for (int c = drained; ok && c < nch; ++c) {
      if (!drain(c)) { ok = false; break; }
    }
    if (ok && !*abort_flag && erow < R) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = col0 + c;
        if (col >= C) continue;
        double *d = P.G + out_base + (int64_t)erow * P.g.cols(bblk) + col;
        *d += f32_scaled_f64(hi[c], ebias) + f32_scaled_f64(lo[c], ebias);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.err, ERR_TIMEOUT);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

static constexpr int TRIPLE_KSPLIT_MAX = 4;  // K splits of the one-CTA-per-tile triple GEMM

// Y rows of every pair a <= b (the most any layout uses: scratch sizes)
static int64_t y_rows(const SepShape &s) {
  const int64_t P2 = (int64_t)s.nbp * (s.nbp + 1) / 2;
  return P2 * s.nbl * (s.nbl + 1) / 2;
}

// Layout of G for a triple-product variant: the split expansion (every block
// wide, Y rows of about half of the pairs) for the forms that read Y from
// device memory; the row-of-c expansion throughout for the forms that build
// Y inside the GEMM.
GLayout tc_triple_glayout(const SepShape &s, int variant) {
  const bool y_hbm = variant == TC_TRIPLE_MATERIALISED || variant == TC_TRIPLE_PAIR || variant == TC_TRIPLE_QUEUE;
  return y_hbm ? make_glayout_split(s.nbl, s.nbp) : make_glayout(s.nbl, s.nbp);
}

static size_t triple_bytes(const SepShape &s, int nxc, int variant, bool parts);
size_t tc_triple_scratch_bytes(const SepShape &s, int nxc, int variant) { return triple_bytes(s, nxc, variant, true); }
// parts: room for the partial sums of K splits, which the forms that read Y
// from device memory may use (the tile autotuner switches between them)
static size_t triple_bytes(const SepShape &s, int nxc, int variant, bool parts) {
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int64_t nblp = (int64_t)s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  size_t b = 0;
  b += up256((size_t)Kpad * nblp * 8) + up256((size_t)nch * nblp * 8); // Mdf, column maxima
  b += up256((size_t)nch * nblp * 8) + up256((size_t)nch * nblp * 4);  // mxW, eB
  b += up256((size_t)OZ_SLICES * nblp * Kpad * 2);                     // Bt
  const bool y_hbm = variant == TC_TRIPLE_MATERIALISED || variant == TC_TRIPLE_PAIR || variant == TC_TRIPLE_QUEUE;
  if (y_hbm || variant == TC_TRIPLE_FUSED2)
    b += up256((size_t)nch * y_rows(s) * 4);                            // eY
  if (y_hbm)
    b += up256((size_t)OZ_SLICES * y_rows(s) * Kpad * 2);               // Y slices
  if (y_hbm && parts)                                                    // partial sums of K splits
    b += up256((size_t)(TRIPLE_KSPLIT_MAX - 1) * make_glayout(s.nbl, s.nbp).size() * 8);
  return b;
}

bool tc_fused2_fits(int nbl, int nbp) {
  const GLayout g = make_glayout(nbl, nbp);
  for (int b = 0; b < nbl; ++b)
    for (int rt = 0; rt < (int)cdiv64(g.rows(b), OZ_BM); ++rt)
      if (f2_groups(g, b, rt) * nbp > F2_MAX_COLS) return false;
  return true;
}

// 2-D map over M~ ([nblp][Kpad] double-FP32 pairs as 8-byte elements), box of
// 32 slices x nbp columns: one group of columns (a, 0..nbp-1) per load.
static int make_mt_map(CUtensorMap *m, const void *base, int64_t rows, int Kpad, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    snprintf(g_tc_err, sizeof g_tc_err, "cuTensorMapEncodeTiled unavailable");
    return MODAL_EUNSUPPORTED;
  }
  cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kpad * 8};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(g_tc_err, sizeof g_tc_err, "cuTensorMapEncodeTiled (M~) failed (%d)", (int)r);
    return MODAL_EINVAL;
  }
  return MODAL_OK;
}

// Modelled issue cost (clocks) of one 16-deep K step of a tile of width w:
// max(80, N/2) per MMA of its schedule (mma_plan.h).
static double plan_step_cost(const uint32_t (&plan)[1 + OZ_PLAN_MAX], int w) {
  double c = 0.0;
  for (int r = 0; r < (int)(plan[0] & 0xffu); ++r) {
    const double N = (double)(((plan[1 + r] >> 8) & 15u) * (uint32_t)w);
    c += N / 2.0 > 80.0 ? N / 2.0 : 80.0;
  }
  return c;
}

// K splits of the one-CTA-per-tile triple GEMM: tiles run in launch order on
// the SMs as they free up (one CTA per SM), each costing its schedule's
// modelled step cost per K step; a split cuts every tile into ks consecutive
// CTAs of whole exact chunks (partial sums added in a fixed order after the
// GEMM), which levels the last wave when the tiles are few and large.  Chooses ks = 1 .. 4 of least
// modelled makespan (each CTA also pays half a chunk of set-up and drain).
// G += part 0 + part 1 + ... (the K splits beyond the first, in order)
__global__ void k_add_parts(double *__restrict__ G, const double *__restrict__ parts, int nparts, int64_t n,
                            int64_t stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = G[i];
  for (int k = 0; k < nparts; ++k) v += parts[(int64_t)k * stride + i];
  G[i] = v;
}
static void triple_ksplit_choice(OzParams &P, int num_sms) {
  std::vector<double> cost;
  for (int b = 0; b < P.g.nbl; ++b) {
    const int w = g_tile_width(P.g.cols(b));
    const double c = plan_step_cost(P.plan[w / 16 - 1], w) * (OZ_KC / 16);  // one exact chunk
    const int64_t n = cdiv64(P.g.rows(b), OZ_BM) * cdiv64(P.g.cols(b), OZ_BN);
    for (int64_t i = 0; i < n; ++i) cost.push_back(c);
  }
  int best = 1;
  double best_t = 0.0;
  const int sms = num_sms > 0 ? num_sms : 1;
  for (int ks = 1; ks <= TRIPLE_KSPLIT_MAX && ks <= P.nchunks; ++ks) {
    const int cpk = (int)cdiv64(P.nchunks, ks);
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int i = 0; i < sms; ++i) free_at.push(0.0);
    double end = 0.0;
    for (const double c : cost)
      for (int k = 0; k < ks; ++k) {
        const int nc = std::min(cpk, P.nchunks - k * cpk);
        if (nc <= 0) continue;
        const double t = free_at.top() + c * (nc + 0.5);
        free_at.pop();
        free_at.push(t);
        end = std::max(end, t);
      }
    if (ks == 1 || end < best_t * 0.98) {  // a split must gain at least 2 %
      best = ks;
      best_t = end;
    }
  }
  P.chunks_per_split = (int)cdiv64(P.nchunks, best);
  P.ksplit = (int)cdiv64(P.nchunks, P.chunks_per_split);  // no part with an empty K range
}

// The persistent queue GEMM: items (tile, K range) in order of decreasing
// modelled cost; tiles are split into K ranges when there are too few of
// them to give every SM two; grid = min(items, SMs).  Returns MODAL_EUNSUPPORTED
// (the caller falls back to one CTA per tile) beyond the queue table's size.
static int launch_queue_gemm(OzParams &P, const CUtensorMap &ta, const BMaps &tb, int nbl, int num_sms,
                             int wmax, bool split, int *head, cudaStream_t st, Profiler *prof) {
  static QueueParams Q;  // host staging of the (large) parameter block
  static std::mutex qm;
  std::lock_guard<std::mutex> lock(qm);
  Q.o = P;
  fill_mma_plans(Q.o.plan);
  struct It {
    double cost;
    uint32_t code;
  };
  std::vector<It> tiles;
  Q.wmax = wmax;
  for (int b = 0, t = 0; b < nbl; ++b) {
    const int w = g_tile_width_cap(P.g.cols(b), wmax);
    const double c = plan_step_cost(Q.o.plan[w / 16 - 1], w);
    const int n = (int)(cdiv64(P.g.rows(b), OZ_BM) * cdiv64(P.g.cols(b), wmax));
    for (int i = 0; i < n; ++i, ++t) tiles.push_back({c, (uint32_t)t});
  }
  const int ntiles = (int)tiles.size();
  int nkr = 1;
  if (split && ntiles < 2 * num_sms) nkr = (int)cdiv64(2 * num_sms, ntiles);
  if (nkr > P.nchunks) nkr = P.nchunks;
  if (nkr > 255) nkr = 255;
  if (nkr < 1) nkr = 1;
  const int cpk = (int)cdiv64(P.nchunks, nkr);
  nkr = (int)cdiv64(P.nchunks, cpk);
  if ((int64_t)ntiles * nkr > Q_ITEMS_MAX) return MODAL_EUNSUPPORTED;
  std::vector<It> items;
  for (auto &t : tiles)
    for (int k = 0; k < nkr; ++k) {
      const int nc = (k + 1) * cpk <= P.nchunks ? cpk : P.nchunks - k * cpk;
      items.push_back({t.cost * nc, t.code << 8 | (uint32_t)k});
    }
  std::stable_sort(items.begin(), items.end(), [](const It &a, const It &b) { return a.cost > b.cost; });
  Q.n_items = (int)items.size();
  Q.nkr = nkr;
  Q.chunks_per_kr = cpk;
  Q.head = head;
  for (int i = 0; i < Q.n_items; ++i) Q.item[i] = items[i].code;
  cudaError_t e;
  if ((e = cudaMemsetAsync(head, 0, sizeof(int), st)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_ozaki_gemm_q, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
          cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "queue GEMM set-up: %s", cudaGetErrorString(e));
    return MODAL_ECUDA;
  }
  const int grid = Q.n_items < num_sms ? Q.n_items : num_sms;
  ProfScope ps(prof, "tc_gemm_triple", st);
  k_ozaki_gemm_q<<<grid, OZ_THREADS, OZ_SMEM, st>>>(ta, tb, Q);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "queue GEMM launch: %s", cudaGetErrorString(e));
    return MODAL_ECUDA;
  }
  return MODAL_OK;
}

int tc_triple_chunk(const SepShape &s, const double *M, const double *om, const double *xw, int x0, int nxc,
                    int nxl_max, double *G, bool accumulate, void *scratch, long long wait_cycles, int num_sms,
                    int variant, int split_k, cudaStream_t st, Profiler *prof, bool absM, int tune) {
  LScratch ls = l_scratch(scratch, s, nxl_max);
  char *w = ls.end;
  int *words = ls.words;
  cudaError_t e;
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int nblp = s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  const int P2 = s.nbp * (s.nbp + 1) / 2;
  f2 *Mdf = (f2 *)w; w += up256((size_t)Kpad * nblp * 8);
  unsigned *colmax = (unsigned *)w; w += up256((size_t)nch * nblp * 8);
  double *mxW = (double *)w; w += up256((size_t)nch * nblp * 8);
  int *eB = (int *)w; w += up256((size_t)nch * nblp * 4);
  __nv_bfloat16 *Bt = (__nv_bfloat16 *)w;
  if (!accumulate) {
    ProfScope ps(prof, "zero_G", st);
    GLayout g = make_glayout(s.nbl, s.nbp);
    if ((e = launch_zero(G, (size_t)g.size(), st)) != cudaSuccess) goto cuda_fail;
  }
  {
    ProfScope ps(prof, "tc_prep_M", st, 2);
    if ((e = cudaMemsetAsync(colmax, 0, (size_t)nch * nblp * 8, st)) != cudaSuccess) goto cuda_fail;
    k_tp_col_max<<<dim3((unsigned)cdiv(nblp, TP_COLS), (unsigned)cdiv64(K, 128)), 256, 0, st>>>(
        K, nblp, s.n_mu, x0, M, om, xw, colmax);
    k_tp_split_cols<<<dim3((unsigned)cdiv(nblp, TP_COLS), (unsigned)(Kpad / 32)), 256, 0, st>>>(
        K, Kpad, nblp, s.n_mu, x0, M, om, xw, colmax, Mdf, mxW, eB, Bt, words + 3, words, absM ? 1 : 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  if (variant == TC_TRIPLE_FUSED2) {
    // Y formed in the GEMM's shared-memory stages; only the row exponents first
    const int64_t rowsY = y_rows(s);
    int *eY = (int *)((char *)Bt + up256((size_t)OZ_SLICES * nblp * Kpad * 2));
    {
      ProfScope ps(prof, "tc_y_exp", st);
      k_tp_y_exp<<<dim3((unsigned)cdiv64(rowsY, 256), (unsigned)nch), 256, 0, st>>>(
          make_glayout(s.nbl, s.nbp), rowsY, s.nbp, nblp, P2, mxW, eY, words + 4);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
    CUtensorMap tm;
    BMaps tb;
    const GLayout gl = make_glayout(s.nbl, s.nbp);
    unsigned used = 0;
    for (int b = 0; b < s.nbl; ++b) used |= 1u << (g_tile_width(gl.cols(b)) / 16 - 1);
    if (int r = make_mt_map(&tm, Mdf, nblp, Kpad, s.nbp)) return r;
    if (int r = make_bmaps(&tb, Bt, nblp, Kpad, used)) return r;
    Fused2Params F{};
    fill_mma_plans(F.plan);
    F.rowsB = nblp;
    F.rowsY = rowsY;
    F.Kpad = Kpad;
    F.nchunks = nch;
    F.nbp = s.nbp;
    F.eY = eY;
    F.eB = eB;
    F.emaxY = words + 4;
    F.emaxB = words + 3;
    F.G = G;
    F.g = gl;
    F.err = words;
    F.wait_cycles = wait_cycles;
    int64_t tiles = 0;
    for (int b = 0; b < s.nbl; ++b) tiles += cdiv64(gl.rows(b), OZ_BM) * cdiv64(gl.cols(b), OZ_BN);
    if ((e = cudaFuncSetAttribute(k_ozaki_triple_fused2, cudaFuncAttributeMaxDynamicSharedMemorySize, F2_SMEM)) !=
        cudaSuccess)
      goto cuda_fail;
    ProfScope ps(prof, "tc_gemm_triple", st);
    k_ozaki_triple_fused2<<<(unsigned)tiles, F2_THREADS, F2_SMEM, st>>>(tm, tb, F);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
    return MODAL_OK;
  }
  if (variant == TC_TRIPLE_MATERIALISED || variant == TC_TRIPLE_PAIR || variant == TC_TRIPLE_QUEUE) {
    // Y slices through HBM, then the TMA-fed GEMM for both operands (single
    // CTAs, or CTA pairs with the 2-SM MMA)
    const GLayout gl = tc_triple_glayout(s, variant);
    const int64_t rowsY = (int64_t)gl.ypairs_total() * P2;
    char *wy = (char *)Bt + up256((size_t)OZ_SLICES * nblp * Kpad * 2);
    int *eY = (int *)wy;
    wy += up256((size_t)nch * rowsY * 4);
    __nv_bfloat16 *Ysl = (__nv_bfloat16 *)wy;
    {
      ProfScope ps(prof, "tc_make_Y", st, 2);  // exponents + slices
      k_tp_y_exp<<<dim3((unsigned)cdiv64(rowsY, 256), (unsigned)nch), 256, 0, st>>>(gl, rowsY, s.nbp, nblp, P2,
                                                                                  mxW, eY, words + 4);
      const size_t smy = ty_smem_bytes(s.nbp);
      if ((e = cudaFuncSetAttribute(k_tp_make_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy)) !=
          cudaSuccess)
        goto cuda_fail;
      k_tp_make_y<<<dim3((unsigned)gl.ypairs_total(), (unsigned)cdiv64(Kpad, TY_K)), 32 * TY_WARPS, smy, st>>>(
          gl, 0, rowsY, K, Kpad, s.nbp, nblp, P2, Mdf, eY, Ysl);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
    CUtensorMap ta;
    BMaps tb;
    unsigned used = 0;
    for (int b = 0; b < s.nbl; ++b) used |= 1u << (g_tile_width(gl.cols(b)) / 16 - 1);
    if (int r = make_slices_map(&ta, Ysl, rowsY, Kpad, OZ_BM)) return r;
    if (int r = make_bmaps(&tb, Bt, nblp, Kpad, used)) return r;
    OzParams P{};
    P.rowsA = rowsY;
    P.rowsB = nblp;
    P.Kpad = Kpad;
    P.nchunks = nch;
    P.eA = eY;
    P.eB = eB;
    P.emaxA = words + 4;
    P.emaxB = words + 3;
    P.out = G;
    P.err = words;
    P.g = gl;
    P.wait_cycles = wait_cycles;
    if (variant == TC_TRIPLE_QUEUE) {
      const int wmax = tune_wmax(tune);
      if (wmax != OZ_BN) {  // B maps for the capped widths
        unsigned used2 = 0;
        for (int b = 0; b < s.nbl; ++b) used2 |= 1u << (g_tile_width_cap(P.g.cols(b), wmax) / 16 - 1);
        if (int r = make_bmaps(&tb, Bt, nblp, Kpad, used2)) return r;
      }
      const int r = launch_queue_gemm(P, ta, tb, s.nbl, num_sms, wmax, tune_split(tune), words + 16, st, prof);
      if (r != MODAL_EUNSUPPORTED) return r;  // else (more items than the table holds): one CTA per tile
    }
    if (variant == TC_TRIPLE_PAIR) {
      // one schedule for every width (pair_plan), two 128-row tiles per cluster
      for (int i = 0; i < OZ_BN / 16; ++i) plan::pair_plan(P.plan[i]);
      int64_t pairs = 0;
      for (int b = 0; b < s.nbl; ++b) pairs += cdiv64(cdiv64(P.g.rows(b), OZ_BM), 2) * cdiv64(P.g.cols(b), OZ_BN);
      if ((e = cudaFuncSetAttribute(k_ozaki_gemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
          cudaSuccess)
        goto cuda_fail;
      ProfScope ps(prof, "tc_gemm_triple", st);
      k_ozaki_gemm_pair<<<(unsigned)(2 * pairs), OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
      if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
      return MODAL_OK;
    }
    fill_mma_plans(P.plan);
    int64_t tiles = 0;
    for (int b = 0; b < s.nbl; ++b) tiles += cdiv64(P.g.rows(b), OZ_BM) * cdiv64(P.g.cols(b), OZ_BN);
    triple_ksplit_choice(P, num_sms);
    if (split_k > 0) {  // a caller's choice (MODAL_OPT_TC_SPLIT_K)
      P.chunks_per_split = (int)cdiv64(P.nchunks, std::min(split_k, TRIPLE_KSPLIT_MAX));
      P.ksplit = (int)cdiv64(P.nchunks, P.chunks_per_split);
    }
    P.part_stride = gl.size();
    P.out_part = (double *)((char *)Ysl + up256((size_t)OZ_SLICES * y_rows(s) * Kpad * 2));
    if ((e = cudaFuncSetAttribute(k_ozaki_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
        cudaSuccess)
      goto cuda_fail;
    {
      ProfScope ps(prof, "tc_gemm_triple", st);
      k_ozaki_gemm<1><<<(unsigned)(tiles * P.ksplit), OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
      if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
    }
    if (P.ksplit > 1) {
      ProfScope ps(prof, "tc_add_parts", st);
      k_add_parts<<<(unsigned)cdiv64(gl.size(), 256), 256, 0, st>>>(G, P.out_part, P.ksplit - 1, gl.size(),
                                                                      gl.size());
      if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
    }
    return MODAL_OK;
  }
  {
    CUtensorMap tb;
    if (int r = make_slices_map(&tb, Bt, nblp, Kpad, OZ_BN)) return r;
    FusedParams F{};
    F.rowsB = nblp;
    F.Kpad = Kpad;
    F.K = K;
    F.nchunks = nch;
    F.nbp = s.nbp;
    F.nblp = nblp;
    F.P2 = P2;
    F.Mdf = Mdf;
    F.mxW = mxW;
    F.eB = eB;
    F.emaxB = words + 3;
    F.emaxW = words + 5;
    F.G = G;
    F.g = make_glayout(s.nbl, s.nbp);
    F.err = words;
    F.wait_cycles = wait_cycles;
    int64_t tiles = 0;
    for (int b = 0; b < s.nbl; ++b) tiles += cdiv64(F.g.rows(b), OZ_BM) * cdiv64(F.g.cols(b), OZ_BN);
    // split K when the tiles alone cannot fill two waves of one CTA per SM,
    // keeping at least 4 exact chunks per split
    int ks = (int)cdiv64(2LL * num_sms, tiles);
    ks = ks < nch / 4 ? ks : nch / 4;
    if (split_k > 0) ks = split_k < nch ? split_k : nch;
    if (ks < 1) ks = 1;
    F.chunks_per_split = (int)cdiv64(nch, ks);
    F.split_k = (int)cdiv64(nch, F.chunks_per_split);
    if ((e = cudaFuncSetAttribute(k_ozaki_triple_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
        cudaSuccess)
      goto cuda_fail;
    ProfScope ps(prof, "tc_gemm_triple", st);
    k_ozaki_triple_fused<<<dim3((unsigned)tiles, (unsigned)F.split_k), OZ_THREADS, OZ_SMEM, st>>>(tb, F);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  }
  return MODAL_OK;
cuda_fail:
  snprintf(g_tc_err, sizeof g_tc_err, "triple product: %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

// ===========================================================================
// The adjoint (row a9) on the tensor cores.
//
// dL/dM through the permanent of Eq. 2D: the derivative of perm(M[L; C])
// with respect to the entry (x, y) is the sum, over the positions i of x in
// the late triple L and j of y in the primordial triple C, of the permanent
// of the 2 x 2 minor left when row i and column j are struck out.  So
//   dL/dM_{xy}(s) = sum_rows Gfull[row][(x, y)] Y_row(s),
//   Y_row(s) = w_s (M_{a u} M_{b v} + M_{a v} M_{b u}),  row = (a <= b, {u, v}),
// where Gfull collects gbar / (48 pi) over every (n, n') and all nine
// (i, j): one GEMM over the Y rows per radial chunk (every row pairs with
// every (x, y), unlike the forward's b <= c blocks).  Then
//   T[(x, a, p)][l] = sum_j dM_{ap}(x, j) w_l P_l(mu_j)      (a second GEMM),
//   dL/dq~_p(l, x) = sum_a q_a(l) T[(x, a, p)][l],
//   dL/dq_a(l)     = sum_{x,p} q~_p(l, x) T[(x, a, p)][l]      (FP64 sums).
// Both GEMMs run as A B^T on the exact-slicing GEMM kernel (dense output),
// operands split into five exponent-aligned BF16 slices.
// ===========================================================================

// Operand rows for the slicing: value (r, k) as FP64 of a [rows][K] operand.
struct OpGfullT {  // rows (x, y) over nblp, K = Y rows: Gfull^T stored [nblp][rowsY]
  const double *g;
  int64_t rowsY;
  __device__ bool empty() const { return false; }
  __device__ double val(int64_t r, int64_t k) const { return g[r * rowsY + k]; }
};
struct OpAt {  // rows l, K = j: the weighted Legendre table A[j][l] = w_l P_l(mu_j)
  const double *A;
  int L;
  __device__ bool empty() const { return false; }
  __device__ double val(int64_t r, int64_t k) const { return A[k * L + r]; }
};
struct OpDmT {  // rows (xl, a, p), K = j: dM[(xl n_mu + j) nblp + (a nbp + p)]
  const double *dM;
  int n_mu, nblp;
  __device__ bool empty() const { return false; }
  __device__ double val(int64_t r, int64_t k) const {
    const int64_t xl = r / nblp, ap = r % nblp;
    return dM[(xl * n_mu + k) * nblp + ap];
  }
};

struct OpBatch {  // rows r, K = t: P[r * T + t] for t0 + t < *count, else 0 (a batch of the direct form)
  const double *P;
  int64_t T;
  const int64_t *count;
  int64_t t0;
  __device__ bool empty() const { return *count <= t0; }
  __device__ double val(int64_t r, int64_t k) const { return t0 + k < *count ? P[r * T + k] : 0.0; }
};

// One warp per (row, K chunk of OZ_KC): the chunk's max |x| (FP32-rounded),
// then the five BF16 slices with that exponent; out [5][rows][Kpad], ex
// [chunks][rows], emax = max exponent.  Zero for k in [K, Kpad).
template <class Op>
__global__ void k_split_op(int64_t rows, int64_t K, int Kpad, Op op, __nv_bfloat16 *__restrict__ out,
                           int *__restrict__ ex, int *__restrict__ emax, int *__restrict__ err) {
  if (op.empty()) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nch = (int)cdiv64(Kpad, OZ_KC);
  if (w >= rows * nch) return;
  const int64_t r = w / nch;
  const int ch = (int)(w % nch);
  const int64_t k0 = (int64_t)ch * OZ_KC, k1 = min(K, k0 + OZ_KC);
  // max |x| on the bits (non-negative doubles order as their bit patterns; a
  // NaN sorts above infinity), rounded to FP32 once: the same value as the
  // maximum of the rounded magnitudes, without a conversion per element
  unsigned long long mb = 0ull;
  for (int64_t k = k0 + lane; k < k1; k += 32)
    mb = max(mb, (unsigned long long)fpb::d_bits(op.val(r, k)) & 0x7fffffffffffffffull);
#pragma unroll
  for (int o = 16; o; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  float m = __double2float_rn(fpb::d_from(mb));
  if (!(m < 1e37f)) {
    if (lane == 0) atomicOr(err, ERR_RANGE);
    m = 0.f;
  }
  const int e = exp_bound_f(m);
  const int64_t sstride = rows * (int64_t)Kpad;
  const int64_t kend = min((int64_t)Kpad, k0 + OZ_KC);
  for (int64_t k = k0 + lane; k < kend; k += 32) {
    const double v = k < K ? op.val(r, k) : 0.0;
    const f2 vd = df_from_d_fast(v);
    __nv_bfloat16 o[OZ_SLICES];
    split_f2(vd.h, vd.l, e, o);
#pragma unroll
    for (int sl = 0; sl < OZ_SLICES; ++sl) out[sl * sstride + r * Kpad + k] = o[sl];
  }
  if (lane == 0) {
    ex[(int64_t)ch * rows + r] = e;
    if (e > -99999) atomicMax(emax, e);
  }
}

// A operand of the dL/dM GEMM: rows = the chunk's slices s = (xl, j), K = the
// Y rows (a <= b, {u, v}); Y_row(s) = sign(w_s) (M~_au M~_bv + M~_av M~_bu)
// with M~ = sqrt|w_s| M in double-FP32 (as the forward's Y).  One block per
// slice: its M~ row, the per-a maxima m_a = max_u |M~_au| and the decoding
// tables of the pair indices in shared memory; warp w takes the row chunks
// w, w + 8, ... of OZ_KC rows.  A chunk's exponent comes from the bound
// |Y| <= 2 m_a m_b over the pairs (a, b) it spans (no pass over the values,
// as for the forward's Y rows); lane i forms rows 4i .. 4i + 3 of each
// 128-row group and stores four BF16 per slice (8 bytes).
constexpr int AY_MAXNB = 64;
__host__ __device__ inline size_t ay_smem_bytes(int nbl, int nbp) {
  return sizeof(f2) * (size_t)nbl * nbp + sizeof(float) * AY_MAXNB +
         sizeof(int) * ((size_t)nbp * (nbp + 1) / 2 + (size_t)nbl * (nbl + 1) / 2);
}
__global__ void __launch_bounds__(256) k_adj_split_y(int64_t S, int nbl, int nbp, int n_mu, int x0,
                                                     const double *__restrict__ M, const double *__restrict__ om,
                                                     const double *__restrict__ xw, int64_t rowsY, int KpadY,
                                                     __nv_bfloat16 *__restrict__ out, int *__restrict__ ex,
                                                     int *__restrict__ emax, int *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char ay_sm[];
  const int nblp = nbl * nbp, P2 = nbp * (nbp + 1) / 2, P2l = nbl * (nbl + 1) / 2;
  f2 *Ms = reinterpret_cast<f2 *>(ay_sm);                       // [nblp]
  float *rmax = reinterpret_cast<float *>(Ms + nblp);           // [AY_MAXNB]
  int *uvtab = reinterpret_cast<int *>(rmax + AY_MAXNB);        // uv -> u | v << 8
  int *prtab = uvtab + P2;                                       // pair -> a | b << 8
  const int64_t sl = blockIdx.x;
  if (sl >= S) return;
  const double w = om[sl % n_mu] * xw[x0 + sl / n_mu];
  const f2 sw = df_from_d(sqrt(fabs(w)));
  const float sg = w < 0.0 ? -1.f : 1.f;
  for (int c = threadIdx.x; c < nblp; c += blockDim.x) Ms[c] = df_mul(df_from_d_fast(M[sl * nblp + c]), sw);
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    int u, v;
    pair_decode(i, u, v);
    uvtab[i] = u | v << 8;
  }
  for (int i = threadIdx.x; i < P2l; i += blockDim.x) {
    int a, b;
    pair_decode(i, a, b);
    prtab[i] = a | b << 8;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nbl; a += blockDim.x) {
    float m = 0.f;
    for (int u = 0; u < nbp; ++u) m = fmaxf(m, fabsf(Ms[a * nbp + u].h) + fabsf(Ms[a * nbp + u].l));
    rmax[a] = m;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (int)cdiv64(KpadY, OZ_KC);
  const int64_t sstride = S * (int64_t)KpadY;
  uint2 *outq = reinterpret_cast<uint2 *>(out);
  for (int ch = warp; ch < nch; ch += 8) {
    const int64_t k0 = (int64_t)ch * OZ_KC, kend = min((int64_t)KpadY, k0 + OZ_KC);
    const int64_t klast = min(rowsY, k0 + OZ_KC) - 1;
    // bound over the pairs of rows [k0, klast]
    float bnd = 0.f;
    if (k0 <= klast)
      for (int64_t pr = k0 / P2 + lane; pr <= klast / P2; pr += 32) {
        const int ab = prtab[pr];
        bnd = fmaxf(bnd, 2.f * rmax[ab & 255] * rmax[ab >> 8]);
      }
#pragma unroll
    for (int o = 16; o; o >>= 1) bnd = fmaxf(bnd, __shfl_xor_sync(0xffffffffu, bnd, o));
    if (!(bnd < 1e37f)) {
      if (lane == 0) atomicOr(err, ERR_RANGE);
      bnd = 0.f;
    }
    const int e = exp_bound_f(bnd);
    const SplitScale sc = split_scale(e);
    // (pair, {u,v}) of the lane's row, stepped along instead of divided out per row
    int pr = (int)((k0 + 4 * lane) / P2), uvr = (int)((k0 + 4 * lane) % P2);
    for (int64_t r0 = k0 + 4 * lane; r0 < kend; r0 += 128) {
      float q[4][OZ_SLICES];
      int prt = pr, uvt = uvr;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t r = r0 + t;
        float h = 0.f, l = 0.f;
        if (r < rowsY) {
          const int ab = prtab[prt], uv = uvtab[uvt];
          const int oa = (ab & 255) * nbp, ob = (ab >> 8) * nbp, u = uv & 255, v = uv >> 8;
          const f2 y = df_addv(df_mul(Ms[oa + u], Ms[ob + v]), df_mul(Ms[oa + v], Ms[ob + u]));
          h = sg * y.h;
          l = sg * y.l;
        }
        if (++uvt == P2) {
          uvt = 0;
          ++prt;
        }
        const float H = sc.zero ? 0.f : (h * sc.s1) * sc.s2;
        const float L = sc.zero ? 0.f : (l * sc.s1) * sc.s2;
        split_hl(H, L, q[t]);
      }
#pragma unroll
      for (int qq = 0; qq < OZ_SLICES; ++qq)
        outq[(qq * sstride + sl * KpadY + r0) / 4] =
            make_uint2(bf16x2_bits(make_float2(q[0][qq], q[1][qq])), bf16x2_bits(make_float2(q[2][qq], q[3][qq])));
      uvr += 128;
      while (uvr >= P2) {
        uvr -= P2;
        ++pr;
      }
    }
    if (lane == 0) {
      ex[(int64_t)ch * S + sl] = e;
      if (e > -99999) atomicMax(emax, e);
    }
  }
}

// Gfull^T[(x, y)][row] += gbar[n][n'] / (48 pi) for every (n, n') and each of
// the nine positions (i, j) of the late triple L = late[n] and the
// primordial triple C = prim[n']: (x, y) = (L_i, C_j), row = the 2 x 2
// minor's rows (the other two late indices, sorted) and columns (the other
// two primordial indices, unordered).
__global__ void k_adj_scatter_gfull(int nbl, int nbp, const double *__restrict__ gbar, const int *__restrict__ late,
                                    const int *__restrict__ prim, int n_late, int n_prim, double scale,
                                    int64_t rowsY, double *__restrict__ GfT) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_late * n_prim) return;
  const int n = (int)(idx / n_prim), m = (int)(idx % n_prim);
  const int Lt[3] = {late[3 * n], late[3 * n + 1], late[3 * n + 2]};
  const int Ct[3] = {prim[3 * m], prim[3 * m + 1], prim[3 * m + 2]};
  for (int i = 0; i < 3; ++i)
    if ((unsigned)Lt[i] >= (unsigned)nbl || (unsigned)Ct[i] >= (unsigned)nbp) return;
  const int P2 = nbp * (nbp + 1) / 2;
  const double v = scale * gbar[idx];
  for (int i = 0; i < 3; ++i) {
    const int r1 = Lt[(i + 1) % 3], r2 = Lt[(i + 2) % 3];
    const int64_t pr = pair_index(r1 < r2 ? r1 : r2, r1 < r2 ? r2 : r1);
    for (int j = 0; j < 3; ++j) {
      const int c1 = Ct[(j + 1) % 3], c2 = Ct[(j + 2) % 3];
      const int64_t row = pr * P2 + pair_index(c1, c2);
      atomicAdd(GfT + ((int64_t)Lt[i] * nbp + Ct[j]) * rowsY + row, v);
    }
  }
}

// ---------------------------------------------------------------------------
// The Y-through-HBM triple product in two phases on two streams, so that the
// Y pass of one radial chunk runs beside the GEMM of the previous one.  Two
// scratch sets alternate between chunks; each set has its own exponent
// maxima and queue counter (the l contraction's words are not touched):
//   set words: [0] max B exponent, [1] max Y exponent, [2] bound of max |M~|,
//   [3] queue counter.
// ---------------------------------------------------------------------------
constexpr int SET_WORDS_BYTES = 256;

static size_t set_bytes(const SepShape &s, int nxc_max) {
  return SET_WORDS_BYTES + triple_bytes(s, nxc_max, TC_TRIPLE_MATERIALISED, false);
}

// two scratch sets, then the K-split partial sums of the one-CTA-per-tile
// GEMM (one copy: the GEMMs of the chunks run one after the other)
static size_t ovl_parts_bytes(const SepShape &s) {
  return up256((size_t)(TRIPLE_KSPLIT_MAX - 1) * make_glayout(s.nbl, s.nbp).size() * 8);
}
size_t tc_ovl_scratch_bytes(const SepShape &s, int nxl, int nxc) {
  LScratch r = l_scratch(nullptr, s, nxl);
  return (size_t)(r.end - (char *)nullptr) + 2 * set_bytes(s, nxc) + ovl_parts_bytes(s) + 1024;
}

__global__ void k_init_set_words(int *w) {
  if (threadIdx.x < 3) w[threadIdx.x] = -100000;
  else if (threadIdx.x == 3) w[3] = 0;
}

struct SetScratch {
  int *sw;
  f2 *Mdf;
  unsigned *colmax;
  double *mxW;
  int *eB, *eY;
  __nv_bfloat16 *Bt, *Ysl;
};
static SetScratch set_scratch(void *scratch, const SepShape &s, int nxl_max, int nxc_max, int set, int nxc) {
  LScratch ls = l_scratch(scratch, s, nxl_max);
  char *w = ls.end + (size_t)set * set_bytes(s, nxc_max);
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int nblp = s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  SetScratch r;
  r.sw = (int *)w; w += SET_WORDS_BYTES;
  r.Mdf = (f2 *)w; w += up256((size_t)Kpad * nblp * 8);
  r.colmax = (unsigned *)w; w += up256((size_t)nch * nblp * 8);
  r.mxW = (double *)w; w += up256((size_t)nch * nblp * 8);
  r.eB = (int *)w; w += up256((size_t)nch * nblp * 4);
  r.Bt = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * nblp * Kpad * 2);
  r.eY = (int *)w; w += up256((size_t)nch * y_rows(s) * 4);
  r.Ysl = (__nv_bfloat16 *)w;
  return r;
}

int tc_triple_prep(const SepShape &s, const double *M, const double *om, const double *xw, int x0, int nxc,
                   int nxl_max, int nxc_max, void *scratch, int set, int part, cudaStream_t st, Profiler *prof) {
  LScratch ls = l_scratch(scratch, s, nxl_max);
  SetScratch r = set_scratch(scratch, s, nxl_max, nxc_max, set, nxc);
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int nblp = s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  const int P2 = s.nbp * (s.nbp + 1) / 2;
  const GLayout gl = tc_triple_glayout(s, TC_TRIPLE_QUEUE);
  const int64_t rowsY = (int64_t)gl.ypairs_total() * P2;
  // part 0: M~, B slices, Y exponents and the Y rows of the first-form
  // blocks; part 1: the Y rows of the others; part < 0: everything
  const int pmid = gl.ypair0(gl.h < gl.nbl ? gl.h : gl.nbl);
  const int p0 = part == 1 ? pmid : 0, p1 = part == 0 ? pmid : gl.ypairs_total();
  cudaError_t e;
  if (part != 1) {
    ProfScope ps(prof, "tc_prep_M", st, 3);
    k_init_set_words<<<1, 32, 0, st>>>(r.sw);
    if ((e = cudaMemsetAsync(r.colmax, 0, (size_t)nch * nblp * 8, st)) != cudaSuccess) goto cuda_fail;
    k_tp_col_max<<<dim3((unsigned)cdiv(nblp, TP_COLS), (unsigned)cdiv64(K, 128)), 256, 0, st>>>(
        K, nblp, s.n_mu, x0, M, om, xw, r.colmax);
    k_tp_split_cols<<<dim3((unsigned)cdiv(nblp, TP_COLS), (unsigned)(Kpad / 32)), 256, 0, st>>>(
        K, Kpad, nblp, s.n_mu, x0, M, om, xw, r.colmax, r.Mdf, r.mxW, r.eB, r.Bt, r.sw, ls.words, 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  {
    ProfScope ps(prof, "tc_make_Y", st, part == 1 ? 1 : 2);
    if (part != 1)
      k_tp_y_exp<<<dim3((unsigned)cdiv64(rowsY, 256), (unsigned)nch), 256, 0, st>>>(gl, rowsY, s.nbp, nblp, P2,
                                                                                  r.mxW, r.eY, r.sw + 1);
    const size_t smy = ty_smem_bytes(s.nbp);
    if ((e = cudaFuncSetAttribute(k_tp_make_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy)) !=
        cudaSuccess)
      goto cuda_fail;
    if (p1 > p0)
      k_tp_make_y<<<dim3((unsigned)(p1 - p0), (unsigned)cdiv64(Kpad, TY_K)), 32 * TY_WARPS, smy, st>>>(
          gl, p0, rowsY, K, Kpad, s.nbp, nblp, P2, r.Mdf, r.eY, r.Ysl);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  return MODAL_OK;
cuda_fail:
  snprintf(g_tc_err, sizeof g_tc_err, "triple product (operands): %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

int tc_triple_gemm(const SepShape &s, int nxc, int nxl_max, int nxc_max, double *G, bool accumulate,
                   void *scratch, int set, long long wait_cycles, int grid_sms, int tune, bool single,
                   int split_k, int part, cudaStream_t st, Profiler *prof) {
  LScratch ls = l_scratch(scratch, s, nxl_max);
  SetScratch r = set_scratch(scratch, s, nxl_max, nxc_max, set, nxc);
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int nblp = s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  const GLayout gl = tc_triple_glayout(s, TC_TRIPLE_QUEUE);
  const int64_t rowsY = (int64_t)gl.ypairs_total() * (s.nbp * (s.nbp + 1) / 2);
  cudaError_t e;
  if (!accumulate) {
    ProfScope ps(prof, "zero_G", st);
    if ((e = launch_zero(G, (size_t)gl.size(), st)) != cudaSuccess) {
      snprintf(g_tc_err, sizeof g_tc_err, "triple product: %s", cudaGetErrorString(e));
      return MODAL_ECUDA;
    }
  }
  CUtensorMap ta;
  BMaps tb;
  const int wmax = tune_wmax(tune);
  unsigned used = 0;
  for (int b = 0; b < s.nbl; ++b) used |= 1u << (g_tile_width_cap(gl.cols(b), wmax) / 16 - 1);
  if (int rr = make_slices_map(&ta, r.Ysl, rowsY, Kpad, OZ_BM)) return rr;
  if (int rr = make_bmaps(&tb, r.Bt, nblp, Kpad, used)) return rr;
  OzParams P{};
  P.rowsA = rowsY;
  P.rowsB = nblp;
  P.Kpad = Kpad;
  P.nchunks = nch;
  P.eA = r.eY;
  P.eB = r.eB;
  P.emaxA = r.sw + 1;
  P.emaxB = r.sw;
  P.out = G;
  P.err = ls.words;
  P.g = gl;
  P.wait_cycles = wait_cycles;
  if (!single) {
    const int rq = launch_queue_gemm(P, ta, tb, s.nbl, grid_sms, wmax, tune_split(tune), r.sw + 3, st, prof);
    if (rq != MODAL_EUNSUPPORTED) return rq;
  }
  // one CTA per tile, or per K range of one (single), or the queue's
  // fallback when it has more items than its table holds
  unsigned used1 = 0;
  for (int b = 0; b < s.nbl; ++b) used1 |= 1u << (g_tile_width(gl.cols(b)) / 16 - 1);
  if (int rr = make_bmaps(&tb, r.Bt, nblp, Kpad, used1)) return rr;
  fill_mma_plans(P.plan);
  // tiles of the blocks of the part (single form): first-form blocks, the
  // others, or all
  int64_t tiles = 0, tile0 = 0;
  for (int b = 0; b < s.nbl; ++b) {
    const int64_t n = cdiv64(gl.rows(b), OZ_BM) * cdiv64(gl.cols(b), OZ_BN);
    const bool in = part < 0 || (part == 0) == gl.first(b);
    if (in) tiles += n;
    else if (part == 1) tile0 += n;  // the first-form blocks come first
  }
  P.tile0 = (int)tile0;
  if (single) {
    // no K splits by default: here the operand passes of the next chunk
    // fill the SMs that the last wave of whole tiles leaves idle
    P.ksplit = 1;
    P.chunks_per_split = P.nchunks;
    if (split_k > 0) {  // a caller's choice (MODAL_OPT_TC_SPLIT_K)
      P.chunks_per_split = (int)cdiv64(P.nchunks, std::min(split_k, TRIPLE_KSPLIT_MAX));
      P.ksplit = (int)cdiv64(P.nchunks, P.chunks_per_split);
    }
    P.part_stride = gl.size();
    P.out_part = (double *)(ls.end + 2 * set_bytes(s, nxc_max));
  }
  if ((e = cudaFuncSetAttribute(k_ozaki_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) ==
      cudaSuccess) {
    ProfScope ps(prof, "tc_gemm_triple", st);
    const int ks = P.ksplit > 1 ? P.ksplit : 1;
    if (tiles > 0) k_ozaki_gemm<1><<<(unsigned)(tiles * ks), OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && P.ksplit > 1 && tiles > 0) {
    // the part's blocks are contiguous in G: [offset(first), offset(last + 1))
    int bl0 = 0, bl1 = s.nbl;
    if (part == 0) bl1 = gl.h < s.nbl ? gl.h : s.nbl;
    if (part == 1) bl0 = gl.h < s.nbl ? gl.h : s.nbl;
    const int64_t g0 = gl.offset(bl0), n = gl.offset(bl1) - g0;
    ProfScope ps(prof, "tc_add_parts", st);
    k_add_parts<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(G + g0, P.out_part + g0, P.ksplit - 1, n, gl.size());
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "triple product: %s", cudaGetErrorString(e));
    return MODAL_ECUDA;
  }
  return MODAL_OK;
}

// dL/dq~ rows of the chunk and its addition to dL/dq from T (FP64):
//   dqt[x0 + xl][p][l]  = sum_a q_a(l) T[(xl, a, p)][l]           (blocks with a == 0)
//   dq[a][l]           += sum_{xl, p} q~_p(l, x0 + xl) T[(xl, a, p)][l]
// one thread per (l, a).
__global__ void k_adj_reduce_t(int nc, int nbl, int nbp, int L, int x0, const double *__restrict__ T,
                               const double *__restrict__ q, const double *__restrict__ qt, double *__restrict__ dqt,
                               double *__restrict__ dq) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (l >= L) return;
  const int64_t nblp = (int64_t)nbl * nbp;
  double sq = 0.0;
  for (int xl = 0; xl < nc; ++xl)
    for (int p = 0; p < nbp; ++p) {
      if (dq) sq = fma(qt[((int64_t)(x0 + xl) * nbp + p) * L + l], T[((int64_t)xl * nblp + (int64_t)a * nbp + p) * L + l], sq);
      if (a == 0) {
        double st = 0.0;
        for (int aa = 0; aa < nbl; ++aa)
          st = fma(q[(int64_t)aa * L + l], T[((int64_t)xl * nblp + (int64_t)aa * nbp + p) * L + l], st);
        dqt[((int64_t)(x0 + xl) * nbp + p) * L + l] = st;
      }
    }
  if (dq) dq[(int64_t)a * L + l] += sq;
}

// ---------------------------------------------------------------------------
// Host side of the tensor-core adjoint.
// ---------------------------------------------------------------------------
// Dense C = A B^T (out[r ld_r + c ld_c], stored or added) on the exact-slicing
// GEMM kernel from operands already split: A [5][rowsA][Kpad] with exponents
// eA [chunks][rowsA] and their maximum *emaxA, B likewise.
static int dense_gemm(const __nv_bfloat16 *As, const int *eA, const int *emaxA, int64_t rowsA,
                      const __nv_bfloat16 *Bs, const int *eB, const int *emaxB, int64_t rowsB, int Kpad, double *out,
                      int64_t ld_r, int64_t ld_c, bool accumulate, int *err, long long wait_cycles, cudaStream_t st,
                      Profiler *prof, const char *name, const int64_t *kdev = nullptr, int64_t koff = 0) {
  CUtensorMap ta;
  BMaps tb;
  if (int r = make_slices_map(&ta, As, rowsA, Kpad, OZ_BM)) return r;
  if (int r = make_bmaps(&tb, Bs, rowsB, Kpad, 1u << (OZ_BN / 16 - 1))) return r;
  OzParams P{};
  P.rowsA = rowsA;
  P.rowsB = rowsB;
  P.Kpad = Kpad;
  P.nchunks = (int)cdiv64(Kpad, OZ_KC);
  P.eA = eA;
  P.eB = eB;
  P.emaxA = emaxA;
  P.emaxB = emaxB;
  P.out = out;
  P.err = err;
  P.wait_cycles = wait_cycles;
  P.ld_r = ld_r;
  P.ld_c = ld_c;
  P.out_accumulate = accumulate ? 1 : 0;
  P.kdev = kdev;
  P.koff = koff;
  fill_mma_plans(P.plan);
  const int64_t nrt = cdiv64(rowsA, OZ_BM), nct = cdiv64(rowsB, OZ_BN);
  const int rpc = gridp::rows_per_cta(nrt, nct);
  P.rows_per_cta = rpc;
  cudaError_t e = cudaFuncSetAttribute(k_ozaki_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  if (e == cudaSuccess) {
    ProfScope ps(prof, name, st);
    k_ozaki_gemm<2><<<dim3((unsigned)nct, (unsigned)cdiv64(nrt, rpc)), OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "%s: %s", name, cudaGetErrorString(e));
    return MODAL_ECUDA;
  }
  return MODAL_OK;
}

template <class Op>
static int split_op(int64_t rows, int64_t K, int Kpad, const Op &op, __nv_bfloat16 *out, int *ex, int *emax,
                    int *err, cudaStream_t st, Profiler *prof, const char *name) {
  ProfScope ps(prof, name, st);
  const int nch = (int)cdiv64(Kpad, OZ_KC);
  k_split_op<Op><<<(unsigned)cdiv64(rows * nch * 32, 256), 256, 0, st>>>(rows, K, Kpad, op, out, ex, emax, err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "%s: %s", name, cudaGetErrorString(e));
    return MODAL_ECUDA;
  }
  return MODAL_OK;
}

// reset words [first, first + n) of the status block to "no exponent yet"
__global__ void k_reset_emax(int *w, int n) {
  if ((int)threadIdx.x < n) w[threadIdx.x] = -100000;
}

static int64_t pad32(int64_t v) { return cdiv64(v, 32) * 32; }

struct AdjScratch {
  char *lreg;  // the l contraction's scratch (l_scratch layout, status words first)
  double *mu, *om, *A, *M, *GfT, *dM, *T;
  __nv_bfloat16 *GfTs, *AtS, *YTs, *dMTs;
  int *eG, *eAt, *eY, *edMT;
  char *end;
};
static AdjScratch adj_scratch(void *base, const SepShape &s, int nxc) {
  const int64_t nblp = (int64_t)s.nbl * s.nbp, rowsY = y_rows(s), S = (int64_t)nxc * s.n_mu;
  const int64_t KY = pad32(rowsY), Kj = pad32(s.n_mu);
  auto nch = [](int64_t K) { return cdiv64(K, OZ_KC); };
  AdjScratch r;
  char *w = (char *)base;
  r.lreg = w;
  w = l_scratch(w, s, nxc).end;
  w = (char *)(((uintptr_t)w + 255) & ~(uintptr_t)255);
  r.mu = (double *)w; w += up256(8 * (size_t)s.n_mu);
  r.om = (double *)w; w += up256(8 * (size_t)s.n_mu);
  r.A = (double *)w; w += up256(8 * (size_t)s.n_mu * s.L);
  r.M = (double *)w; w += up256(8 * (size_t)S * nblp);
  r.dM = (double *)w; w += up256(8 * (size_t)S * nblp);
  r.T = (double *)w; w += up256(8 * (size_t)nxc * nblp * s.L);
  r.GfT = (double *)w; w += up256(8 * (size_t)nblp * rowsY);
  r.GfTs = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * nblp * KY * 2);
  r.eG = (int *)w; w += up256(4 * (size_t)nch(KY) * nblp);
  r.AtS = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * s.L * Kj * 2);
  r.eAt = (int *)w; w += up256(4 * (size_t)nch(Kj) * s.L);
  r.YTs = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * S * KY * 2);
  r.eY = (int *)w; w += up256(4 * (size_t)nch(KY) * S);
  r.dMTs = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * nxc * nblp * Kj * 2);
  r.edMT = (int *)w; w += up256(4 * (size_t)nch(Kj) * nxc * nblp);
  r.end = w;
  return r;
}

size_t tc_backward_scratch_bytes(const SepShape &s, int nxc) {
  return (size_t)(adj_scratch(nullptr, s, nxc).end - (char *)nullptr) + 1024;
}

// radial points per chunk of the tensor-core adjoint: its per-point buffers
// (Y^T slices, M, dM and its slices, T) within 8 GiB, 1 .. 32; given the SM
// count, the chunk between half and all of that whose dL/dM GEMMs need the
// fewest CTA waves over the call (grid_plan.h)
int tc_backward_nxc(const SepShape &s, int num_sms) {
  const int64_t per_x = (int64_t)s.n_mu * (10 * pad32(y_rows(s)) + 26 * (int64_t)s.nbl * s.nbp) +
                        8 * (int64_t)s.nbl * s.nbp * s.L;
  int64_t c = ((int64_t)8 << 30) / (per_x > 0 ? per_x : 1);
  c = c < 1 ? 1 : (c > 32 ? 32 : c);
  if (c > s.n_x) c = s.n_x > 0 ? s.n_x : 1;
  return gridp::chunk(s.n_x, s.n_mu, (int64_t)s.nbl * s.nbp, c, num_sms);
}

// The adjoint on the tensor cores (see the block comment above k_adj_split_y).
// Status words (the l contraction's block): [0] error bits; adjoint maxima at
// [32] Y^T, [33] Gfull^T, [34] dM^T, [35] A^T.
int tc_backward(const SepShape &s, int nxc, const modal_problem *p, const double *gbar, double *dqt, double *dq,
                void *scratch, long long wc, cudaStream_t st, Profiler *prof) {
  AdjScratch r = adj_scratch(scratch, s, nxc);
  int *words = (int *)r.lreg, *aw = words + 32;
  const int64_t nblp = (int64_t)s.nbl * s.nbp, rowsY = y_rows(s);
  const int KY = (int)pad32(rowsY), Kj = (int)pad32(s.n_mu);
  cudaError_t e;
#define ADJ_CK(x)                                                                      \
  do {                                                                                 \
    if ((e = (x)) != cudaSuccess) {                                                    \
      snprintf(g_tc_err, sizeof g_tc_err, "adjoint: %s: %s", #x, cudaGetErrorString(e)); \
      return MODAL_ECUDA;                                                              \
    }                                                                                  \
  } while (0)
  ADJ_CK(launch_zero(dqt, (size_t)s.n_x * s.nbp * s.L, st));
  if (dq) ADJ_CK(launch_zero(dq, (size_t)s.nbl * s.L, st));
  if (s.n_x == 0 || (int64_t)p->n_late * p->n_prim == 0) return MODAL_OK;
  {
    ProfScope ps(prof, "adj_tables", st, 2);
    ADJ_CK(launch_gl_nodes(s.n_mu, r.mu, r.om, st));
    ADJ_CK(launch_legendre_table(s.n_mu, r.mu, s.l_min, s.l_max, p->w_l, r.A, st));
  }
  // the x-independent operands: Gfull^T (rows (x, y), K = Y rows) and A q (rows l, K = (j, a))
  if (int rr = tc_prepare_l(s, r.A, p->q, r.lreg, nxc, st, prof, true)) return rr;
  {
    ProfScope ps(prof, "adj_gfull", st, 3);
    k_reset_emax<<<1, 32, 0, st>>>(aw, 8);
    ADJ_CK(launch_zero(r.GfT, (size_t)nblp * rowsY, st));
    const int64_t n = (int64_t)p->n_late * p->n_prim;
    k_adj_scatter_gfull<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(s.nbl, s.nbp, gbar, p->late_modes, p->prim_modes,
                                                                   p->n_late, p->n_prim, 1.0 / (48.0 * MODAL_PI),
                                                                   rowsY, r.GfT);
    ADJ_CK(cudaGetLastError());
  }
  if (int rr = split_op(nblp, rowsY, KY, OpGfullT{r.GfT, rowsY}, r.GfTs, r.eG, aw + 1, words, st, prof,
                        "adj_split_gfull"))
    return rr;
  if (int rr = split_op((int64_t)s.L, (int64_t)s.n_mu, Kj, OpAt{r.A, s.L}, r.AtS, r.eAt, aw + 3, words, st, prof,
                        "adj_split_a"))
    return rr;
  const size_t ysm = ay_smem_bytes(s.nbl, s.nbp);
  ADJ_CK(cudaFuncSetAttribute(k_adj_split_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm));
  for (int x0 = 0; x0 < s.n_x; x0 += nxc) {
    const int nc = (s.n_x - x0) < nxc ? (s.n_x - x0) : nxc;
    const int64_t S = (int64_t)nc * s.n_mu;
    if (int rr = tc_contract_l(s, p->qt, x0, nc, nxc, r.M, r.lreg, wc, st, prof)) return rr;  // M (FP64)
    {
      ProfScope ps(prof, "adj_split_y", st, 2);
      k_reset_emax<<<1, 32, 0, st>>>(aw, 1);
      k_adj_split_y<<<(unsigned)S, 256, ysm, st>>>(S, s.nbl, s.nbp, s.n_mu, x0, r.M, r.om, p->x_w, rowsY, KY, r.YTs,
                                                    r.eY, aw, words);
      ADJ_CK(cudaGetLastError());
    }
    // dL/dM [s][(x, y)] = Y^T Gfull over the Y rows
    if (int rr = dense_gemm(r.YTs, r.eY, aw, S, r.GfTs, r.eG, aw + 1, nblp, KY, r.dM, nblp, 1, false, words, wc, st,
                            prof, "adj_gemm_dM"))
      return rr;
    // T[(xl, a, p)][l] = sum_j dM against the Legendre table, then dL/dq~ and dL/dq
    k_reset_emax<<<1, 32, 0, st>>>(aw + 2, 1);
    if (int rr = split_op((int64_t)nc * nblp, (int64_t)s.n_mu, Kj, OpDmT{r.dM, s.n_mu, (int)nblp}, r.dMTs, r.edMT,
                          aw + 2, words, st, prof, "adj_split_dm"))
      return rr;
    if (int rr = dense_gemm(r.dMTs, r.edMT, aw + 2, (int64_t)nc * nblp, r.AtS, r.eAt, aw + 3, s.L, Kj, r.T, s.L, 1,
                            false, words, wc, st, prof, "adj_gemm_t"))
      return rr;
    {
      ProfScope ps(prof, "adj_reduce_t", st);
      k_adj_reduce_t<<<dim3((unsigned)cdiv(s.L, 128), (unsigned)(dq ? s.nbl : 1)), 128, 0, st>>>(nc, s.nbl, s.nbp,
                                                                                                 s.L, x0, r.T,
                                                                                      p->q, p->qt, dqt, dq);
      ADJ_CK(cudaGetLastError());
    }
  }
#undef ADJ_CK
  return MODAL_OK;
}

// C[m][n] += sum_t A[m][t] B[n][t] over the t < *count - t0 of a batch of T
// terms (A [m][T], B [n][T] FP64), on the exact-slicing GEMM; a batch past
// the end does no work.  Scratch: [words 1 KB][A slices, exponents][B ...].
static size_t tc_batch_parts(int m, int n, int T, char *base, int **words, __nv_bfloat16 **As, int **eA,
                             __nv_bfloat16 **Bs, int **eB) {
  const int64_t Kp = pad32(T), nch = cdiv64(Kp, OZ_KC);
  char *w = base;
  *words = (int *)w; w += 1024;
  *As = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * m * Kp * 2);
  *eA = (int *)w; w += up256(4 * (size_t)nch * m);
  *Bs = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * n * Kp * 2);
  *eB = (int *)w; w += up256(4 * (size_t)nch * n);
  return (size_t)(w - base);
}
size_t tc_gemm_batch_scratch_bytes(int m, int n, int T) {
  int *w, *ea, *eb;
  __nv_bfloat16 *a, *b;
  return tc_batch_parts(m, n, T, nullptr, &w, &a, &ea, &b, &eb) + 256;
}
int tc_gemm_batch(int m, int n, int T, const double *A, const double *B, const int64_t *count, int64_t t0, double *C,
                  int64_t ldc, void *scratch, bool reset_status, long long wc, cudaStream_t st, Profiler *prof) {
  int *words, *eA, *eB;
  __nv_bfloat16 *As, *Bs;
  tc_batch_parts(m, n, T, (char *)scratch, &words, &As, &eA, &Bs, &eB);
  const int Kp = (int)pad32(T);
  if (reset_status && cudaMemsetAsync(words, 0, sizeof(int), st) != cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "batch GEMM: status reset failed");
    return MODAL_ECUDA;
  }
  k_reset_emax<<<1, 32, 0, st>>>(words + 1, 2);
  if (int r = split_op((int64_t)m, (int64_t)T, Kp, OpBatch{A, T, count, t0}, As, eA, words + 1, words, st, prof,
                       "direct_split"))
    return r;
  if (int r = split_op((int64_t)n, (int64_t)T, Kp, OpBatch{B, T, count, t0}, Bs, eB, words + 2, words, st, prof,
                       "direct_split"))
    return r;
  return dense_gemm(As, eA, words + 1, m, Bs, eB, words + 2, n, Kp, C, ldc, 1, true, words, wc, st, prof,
                    "direct_gemm_tc", count, t0);
}

// ===========================================================================
// Direct form (Eq. 3D) with the radial integrals on the tensor cores.
//
// For a sorted triple (l1, l2, l3) the radial integral, expanded along l1 as
// in the FP64 kernel, is
//   Z[p][{u,v}] = sum_x q~_p(l1, x) U_uv(x),
//   U_uv(x)     = W_x (q~_u(l2, x) q~_v(l3, x) + q~_v(l2, x) q~_u(l3, x)),
//   X[(p,r,s)]  = Z[p][{r,s}] + Z[r][{p,s}] + Z[s][{p,r}].
// U depends on the pair (l2, l3) only, so the triples are grouped by it.
// The l1 that complete a pair -- grid points with l3 - l2 <= l1 <= l2 and,
// with exact 3j weights, l1 + l2 + l3 even -- are a contiguous run of the
// grid points of one parity class; with the q~ rows of the grid ordered by
// class (A: rows (l1, p), K = x), the Z blocks of all of a pair's triples
// are one product with the pair's U rows (B: rows {u,v}, K = x).  The work
// items of that grouped GEMM (OUT_MODE 3) are tiles of cpt = 128 / nbp
// consecutive l1 of one pair times column tiles of the {u,v} rows.
//
// The late-time side is expanded along l1 as well:
//   sum_perm q_a q_b q_c = q_a(l1) S_bc + q_b(l1) S_ac + q_c(l1) S_ab,
//   S_bc = q_b(l2) q_c(l3) + q_c(l2) q_b(l3)   (a function of the pair),
// so with W_pair[a][n'] = sum over the pair's triples of z q_a(l1) X[n'],
//   Gu[{b,c}][(a, n')] = sum over pairs of S_bc W_pair[a][n'],
//   Gamma'[(a,b,c)][n'] = Gu[{b,c}][(a,n')] + Gu[{a,c}][(b,n')] + Gu[{a,b}][(c,n')]:
// the l1 sum runs at the width of the basis (nb_late x n_prim per triple)
// and the large GEMM runs over pairs, not triples.
//
// Triples are numbered pair by pair (pairs i2 <= i3 in row-major order of
// the grid indices, then l1 ascending) and processed in batches of at most
// DTC_NT tiles and DTC_NP pairs, whose bounds are found on the device (a
// cursor over the tile list); per batch:
//   info, fill   ranges of the batch; (l1, l2, l3) and weight z per triple
//   make_u       the U rows of the batch's pairs, sliced
//   items, GEMM  Z of every triple of the batch
//   X            radial integrals from Z
//   W            the l1 sums of the batch's pairs (double-FP32)
//   Gu          += S^T W over the batch's pairs (exact-slicing GEMM)
// then Gamma' from Gu.  The host bounds the number of batches by the tile
// bound (the pairs plus C(ng + 2, 3) / cpt) and the pair bound; batches
// past the end do no work.
// ===========================================================================
constexpr int DTC_NT = 4096;   // tiles per batch (at most)
constexpr int DTC_NP = 1024;   // pairs per batch (at most)
constexpr int DTC_MAXNB = 32;  // basis functions of this form (Z block of a triple in shared memory; W sums)

using DtcBatch = dtc::Batch;  // index logic of this form: dtc_enum.h
using dtc::find;

// Grid points ordered by class: crow[k] = grid index of class row k; class 0
// (even l with exact 3j weights, every point otherwise) first.  cls = sizes.
__global__ void k_dtc_classes(int ng, const int *__restrict__ grid, int mode, int *__restrict__ crow,
                              int *__restrict__ cls) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const bool par = mode == MODAL_W_EXACT_3J;
  int k = 0;
  for (int i = 0; i < ng; ++i)
    if (!par || !(grid[i] & 1)) crow[k++] = i;
  const int n0 = k;
  if (par)
    for (int i = 0; i < ng; ++i)
      if (grid[i] & 1) crow[k++] = i;
  cls[0] = n0;
  cls[1] = k - n0;
}

// per pair index (i2, i3) (zero unless i2 <= i3): triples, tiles, has-tiles
__global__ void k_dtc_count(int ng, const int *__restrict__ grid, const int *__restrict__ crow,
                            const int *__restrict__ cls, int mode, int cpt, int64_t *__restrict__ tri_cnt,
                            int64_t *__restrict__ tile_cnt, int64_t *__restrict__ nz_cnt) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ng * ng) return;
  const int i2 = (int)(idx / ng), i3 = (int)(idx % ng);
  int64_t n = 0;
  if (i3 >= i2) n = dtc::run(i2, i3, grid, crow, cls, mode == MODAL_W_EXACT_3J).n;
  const int64_t nt = (n + cpt - 1) / cpt;
  tri_cnt[idx] = n;
  tile_cnt[idx] = nt;
  nz_cnt[idx] = nt > 0;
}

// totals {triples, tiles, pairs with tiles}; the batch cursor starts at tile 0
__global__ void k_dtc_totals(int64_t n, const int64_t *__restrict__ tri_cnt, const int64_t *__restrict__ tri_off,
                             const int64_t *__restrict__ tile_cnt, const int64_t *__restrict__ tile_off,
                             const int64_t *__restrict__ nz_cnt, const int64_t *__restrict__ slot_of,
                             int64_t *__restrict__ tot) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  tot[0] = n > 0 ? tri_off[n - 1] + tri_cnt[n - 1] : 0;
  tot[1] = n > 0 ? tile_off[n - 1] + tile_cnt[n - 1] : 0;
  tot[2] = n > 0 ? slot_of[n - 1] + nz_cnt[n - 1] : 0;
  tot[3] = 0;  // cursor: first tile of the next batch
}

__global__ void k_dtc_compact(int64_t n, const int64_t *__restrict__ nz_cnt, const int64_t *__restrict__ slot_of,
                              int *__restrict__ pairs_nz) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n && nz_cnt[idx]) pairs_nz[slot_of[idx]] = (int)idx;
}

// The next batch: from the cursor, at most DTC_NT tiles and DTC_NP pairs.
__global__ void k_dtc_info(int nct, int cpt, int64_t npairs, const int64_t *__restrict__ tile_off,
                           const int64_t *__restrict__ tri_off, const int64_t *__restrict__ slot_of,
                           const int *__restrict__ pairs_nz, int64_t *__restrict__ tot, DtcBatch *__restrict__ info) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t cursor = tot[3];
  *info = dtc::next_batch(cursor, tot, nct, cpt, npairs, tile_off, tri_off, slot_of, pairs_nz, DTC_NT, DTC_NP);
  tot[3] = cursor;
}

// (l1, l2, l3) and the weight z of each triple of the batch
__global__ void k_dtc_fill(const DtcBatch *__restrict__ info, const int64_t *__restrict__ tri_off, int64_t npairs,
                           int ng, const int *__restrict__ grid, const int *__restrict__ crow,
                           const int *__restrict__ cls, int mode, const double *__restrict__ dw,
                           const double *__restrict__ w_l, int l_min, const double *__restrict__ ctab,
                           int *__restrict__ tri, double *__restrict__ z) {
  const int64_t tb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tb >= info->n_tri) return;
  const int64_t t = info->trip0 + tb;
  const int64_t pr = find(tri_off, npairs, t);
  const int i2 = (int)(pr / ng), i3 = (int)(pr % ng);
  const dtc::Run run = dtc::run(i2, i3, grid, crow, cls, mode == MODAL_W_EXACT_3J);
  const int i1 = crow[run.k0 + (int)(t - tri_off[pr])];
  const int l1 = grid[i1], l2 = grid[i2], l3 = grid[i3];
  tri[3 * tb] = l1;
  tri[3 * tb + 1] = l2;
  tri[3 * tb + 2] = l3;
  z[tb] = direct_weight(l1, l2, l3, i1, i2, i3, dw, w_l, l_min, ctab, mode);
}

// A operand: q~_p(l, x) of the class-ordered grid rows, row k nbp + p
struct OpQRows {
  const double *qt;  // [n_x][nbp][L]
  const int *grid, *crow;
  int L, l_min, nbp;
  __device__ bool empty() const { return false; }
  __device__ double val(int64_t r, int64_t k) const {
    const int l = grid[crow[r / nbp]];
    return qt[(k * nbp + r % nbp) * L + (l - l_min)];
  }
};

// double-FP32 value of a_u b_v + a_v b_u (high part and unnormalised low part)
__device__ __forceinline__ void dtc_u_value(f2 au, f2 bv, f2 av, f2 bu, float &h, float &l) {
  const float p1 = __fmul_rn(au.h, bv.h);
  float e1 = fmaf(au.h, bv.h, -p1);
  e1 = fmaf(au.h, bv.l, e1);
  e1 = fmaf(au.l, bv.h, e1);
  const float p2 = __fmul_rn(av.h, bu.h);
  float e2 = fmaf(av.h, bu.h, -p2);
  e2 = fmaf(av.h, bu.l, e2);
  e2 = fmaf(av.l, bu.h, e2);
  h = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(h, p1);
  const float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(h, bb)), __fsub_rn(p2, bb));
  l = __fadd_rn(t, __fadd_rn(e1, e2));
}

// U rows of the batch's pairs: block (slot, K chunk).  The pair's q~ rows
// (W_x folded into those of l2) are staged as double-FP32 for xs points at
// a time; pass 0 finds each row's maximum |U| over the chunk (one warp per
// row, lanes over x), pass 1 recomputes U and writes the five slices with
// that row's exponent.  Rows P2 .. urows - 1 (padding of the column tiles)
// are zero.
__host__ __device__ inline size_t dtc_u_smem(int nbp, int xs, int urows, int P2) {
  return (size_t)2 * nbp * xs * sizeof(f2) + (size_t)urows * sizeof(float) + (size_t)P2 * sizeof(int);
}
__global__ void __launch_bounds__(256) k_dtc_make_u(const DtcBatch *__restrict__ info, const int *__restrict__ pairs_nz,
                                                    int ng, const int *__restrict__ grid, int l_min, int L, int nbp,
                                                    int n_x, const double *__restrict__ qt,
                                                    const double *__restrict__ xw, int P2, int urows, int Kpad, int xs,
                                                    int64_t rowsU, __nv_bfloat16 *__restrict__ Us,
                                                    int *__restrict__ eU, int *__restrict__ emaxU,
                                                    int *__restrict__ err) {
  const int slot = blockIdx.x;
  if (slot >= info->nslots) return;
  extern __shared__ __align__(16) unsigned char du_sm[];
  f2 *As = reinterpret_cast<f2 *>(du_sm);  // [nbp][xs]: W_x q~_p(l2, x)
  f2 *Bs = As + (size_t)nbp * xs;          // [nbp][xs]: q~_p(l3, x)
  float *rmax = reinterpret_cast<float *>(Bs + (size_t)nbp * xs);
  int *uvt = reinterpret_cast<int *>(rmax + urows);
  const int pair = pairs_nz[info->slot0 + slot];
  const int c2 = grid[pair / ng] - l_min, c3 = grid[pair % ng] - l_min;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ch = blockIdx.y;
  for (int i = threadIdx.x; i < urows; i += blockDim.x) rmax[i] = 0.f;
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    int u, v;
    pair_decode(i, u, v);
    uvt[i] = u | v << 8;
  }
  const int k0 = ch * OZ_KC, k1 = min(n_x, k0 + OZ_KC), kend = min(Kpad, k0 + OZ_KC);
  const int64_t rowbase = (int64_t)slot * urows;
  const int64_t sstride = rowsU * (int64_t)Kpad;
  for (int pass = 0; pass < 2; ++pass) {
    for (int xb = k0; xb < kend; xb += xs) {
      const int nx = min(xs, kend - xb);
      __syncthreads();
      for (int e = threadIdx.x; e < nbp * nx; e += blockDim.x) {
        const int p = e / nx, xl = e - p * nx, x = xb + xl;
        double a = 0.0, b = 0.0;
        if (x < k1) {
          const int64_t o = ((int64_t)x * nbp + p) * L;
          a = xw[x] * qt[o + c2];
          b = qt[o + c3];
        }
        As[p * xs + xl] = df_from_d_fast(a);
        Bs[p * xs + xl] = df_from_d_fast(b);
      }
      __syncthreads();
      for (int uv = warp; uv < urows; uv += nw) {
        __nv_bfloat16 *dst = Us + (rowbase + uv) * Kpad + xb;
        if (uv >= P2) {
          if (pass == 1)
            for (int xl = lane; xl < nx; xl += 32)
#pragma unroll
              for (int sl = 0; sl < OZ_SLICES; ++sl) dst[sl * sstride + xl] = __float2bfloat16_rn(0.f);
          continue;
        }
        const int u = uvt[uv] & 0xff, v = uvt[uv] >> 8;
        const f2 *au = As + u * xs, *av = As + v * xs, *bu = Bs + u * xs, *bv = Bs + v * xs;
        if (pass == 0) {
          float m = 0.f;
          for (int xl = lane; xl < nx; xl += 32) {
            float h, l;
            dtc_u_value(au[xl], bv[xl], av[xl], bu[xl], h, l);
            m = fmaxf(m, fabsf(h));
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0) rmax[uv] = fmaxf(rmax[uv], m);
        } else {
          const int e = exp_bound_f(rmax[uv]);
          for (int xl = lane; xl < nx; xl += 32) {
            float h, l;
            dtc_u_value(au[xl], bv[xl], av[xl], bu[xl], h, l);
            __nv_bfloat16 o[OZ_SLICES];
            split_f2(h, l, e, o);
#pragma unroll
            for (int sl = 0; sl < OZ_SLICES; ++sl) dst[sl * sstride + xl] = o[sl];
          }
        }
      }
    }
    if (pass == 0) {
      __syncthreads();
      for (int uv = threadIdx.x; uv < urows; uv += blockDim.x) {
        float m = rmax[uv];
        if (!(m < 1e37f)) {
          atomicOr(err, ERR_RANGE);
          m = 0.f;
          rmax[uv] = 0.f;
        }
        const int e = uv < P2 ? exp_bound_f(m) : -100000;
        eU[(int64_t)ch * rowsU + rowbase + uv] = e;
        if (e > -99999) atomicMax(emaxU, e);
      }
    }
  }
}

// work items of the batch's grouped GEMM: tile j, column tile h
__global__ void k_dtc_items(const DtcBatch *__restrict__ info, const int64_t *__restrict__ tile_off,
                            const int64_t *__restrict__ tri_off, const int64_t *__restrict__ slot_of, int64_t npairs,
                            int ng, const int *__restrict__ grid, const int *__restrict__ crow,
                            const int *__restrict__ cls, int mode, int cpt, int nbp, int nct, int wu, int urows,
                            int4 *__restrict__ items) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const DtcBatch b = *info;
  if (j >= b.nt) return;
  for (int h = 0; h < nct; ++h) {
    const dtc::Item it = dtc::item(b, j, h, tile_off, tri_off, slot_of, npairs, ng, grid, crow, cls,
                                   mode == MODAL_W_EXACT_3J, cpt, nbp, wu, urows);
    items[j * nct + h] = make_int4(it.a_row0, it.b_row0, it.tri0, it.packed);
  }
}

// X[tb][m] of the batch's triples from their Z blocks (one triple per block)
__global__ void __launch_bounds__(256) k_dtc_x(const DtcBatch *__restrict__ info, const double *__restrict__ Z,
                                               int nbp, int P2, const int *__restrict__ prim, int n_prim,
                                               double *__restrict__ Xb) {
  const int64_t tb = blockIdx.x;
  if (tb >= info->n_tri) return;
  extern __shared__ __align__(16) double dx_sm[];  // [nbp][P2]
  const int nz = nbp * P2;
  const double *zb = Z + tb * nz;
  if ((nz & 1) == 0) {  // the block starts on a 16-byte boundary: 16-byte loads, four in flight per thread
    const double2 *z2 = reinterpret_cast<const double2 *>(zb);
    double2 *s2 = reinterpret_cast<double2 *>(dx_sm);
    const int n2 = nz / 2;
    int i = threadIdx.x;
    for (; i + 3 * (int)blockDim.x < n2; i += 4 * blockDim.x) {
      const double2 v0 = z2[i], v1 = z2[i + blockDim.x], v2 = z2[i + 2 * blockDim.x], v3 = z2[i + 3 * blockDim.x];
      s2[i] = v0;
      s2[i + blockDim.x] = v1;
      s2[i + 2 * blockDim.x] = v2;
      s2[i + 3 * blockDim.x] = v3;
    }
    for (; i < n2; i += blockDim.x) s2[i] = z2[i];
  } else {
    for (int i = threadIdx.x; i < nz; i += blockDim.x) dx_sm[i] = zb[i];
  }
  __syncthreads();
  for (int m = threadIdx.x; m < n_prim; m += blockDim.x) {
    const int p = prim[3 * m], r = prim[3 * m + 1], s = prim[3 * m + 2];
    double v;
    if ((unsigned)p >= (unsigned)nbp || (unsigned)r >= (unsigned)nbp || (unsigned)s >= (unsigned)nbp)
      v = __longlong_as_double(0x7ff8000000000000LL);
    else
      v = dx_sm[p * P2 + pair_index(r, s)] + dx_sm[r * P2 + pair_index(p, s)] + dx_sm[s * P2 + pair_index(p, r)];
    Xb[tb * n_prim + m] = v;
  }
}

// acc += c x in double-FP32 (c, x double-FP32; acc unnormalised)
__device__ __forceinline__ void dtc_df_fma(f2 &acc, f2 c, f2 x) {
  const float p = __fmul_rn(c.h, x.h);
  const float e = fmaf(c.h, x.l, fmaf(c.l, x.h, fmaf(c.h, x.h, -p)));
  const float t = __fadd_rn(acc.h, p);
  const float bb = __fsub_rn(t, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
  acc.h = t;
}

// W[(a, m)][s] = sum over the batch's triples of pair slot s of z q_a(l1) X[tb][m]:
// block (slot, DTC_WTH modes m); the weights z q_a(l1) of DTC_WCH triples at
// a time in shared memory, the nb_late sums of each m in registers, the X
// values of four triples loaded ahead of their use.
// NB = nb_late rounded up to a multiple of 4 (weights of the extra rows are 0).
constexpr int DTC_WCH = 64, DTC_WTH = 256;
template <int NB>
__device__ __forceinline__ void dtc_w_step(f2 (&acc)[NB], const f2 *c, double xd) {
  const f2 x = df_from_d_fast(xd);
  const float4 *c4 = reinterpret_cast<const float4 *>(c);  // two weights per 16-byte load
#pragma unroll
  for (int a = 0; a < NB; a += 2) {
    const float4 v = c4[a / 2];
    dtc_df_fma(acc[a], f2{v.x, v.y}, x);
    dtc_df_fma(acc[a + 1], f2{v.z, v.w}, x);
  }
}
template <int NB>
__global__ void __launch_bounds__(DTC_WTH, 2) k_dtc_w(const DtcBatch *__restrict__ info,
                                                   const int *__restrict__ pairs_nz,
                                                   const int64_t *__restrict__ tri_off,
                                                   const int64_t *__restrict__ tri_cnt, const int *__restrict__ tri,
                                                   const double *__restrict__ z, const double *__restrict__ q, int L,
                                                   int l_min, int nbl, const double *__restrict__ X, int n_prim,
                                                   double *__restrict__ W, int NPK, int *__restrict__ err) {
  const int s = blockIdx.x;
  if (s >= info->nslots) return;
  __shared__ __align__(16) f2 cs[DTC_WCH][DTC_MAXNB];
  const int pair = pairs_nz[info->slot0 + s];
  const int64_t b0 = info->trip0, b1 = b0 + info->n_tri;
  const int64_t g0 = max(tri_off[pair], b0), g1 = min(tri_off[pair] + tri_cnt[pair], b1);
  const int m = blockIdx.y * DTC_WTH + threadIdx.x;
  const int mc = min(m, n_prim - 1);  // threads past n_prim load a valid address and store nothing
  f2 acc[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) acc[a] = f2{0.f, 0.f};
  for (int64_t c0 = g0; c0 < g1; c0 += DTC_WCH) {
    const int nc = (int)min((int64_t)DTC_WCH, g1 - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < nc * NB; e += blockDim.x) {
      const int j = e / NB, a = e - j * NB;
      const int64_t tb = c0 + j - b0;
      cs[j][a] = a < nbl ? df_from_d_fast(z[tb] * q[(int64_t)a * L + (tri[3 * tb] - l_min)]) : f2{0.f, 0.f};
    }
    __syncthreads();
    const double *xr = X + (c0 - b0) * n_prim + mc;
    int j = 0;
    for (; j + 4 <= nc; j += 4) {
      const double x0 = __ldg(xr + (int64_t)j * n_prim), x1 = __ldg(xr + (int64_t)(j + 1) * n_prim);
      const double x2 = __ldg(xr + (int64_t)(j + 2) * n_prim), x3 = __ldg(xr + (int64_t)(j + 3) * n_prim);
      dtc_w_step<NB>(acc, cs[j], x0);
      dtc_w_step<NB>(acc, cs[j + 1], x1);
      dtc_w_step<NB>(acc, cs[j + 2], x2);
      dtc_w_step<NB>(acc, cs[j + 3], x3);
    }
    for (; j < nc; ++j) dtc_w_step<NB>(acc, cs[j], __ldg(xr + (int64_t)j * n_prim));
  }
  if (m < n_prim) {
    bool bad = false;
#pragma unroll
    for (int a = 0; a < NB; ++a)
      if (a < nbl) {
        bad = bad || !(fabsf(acc[a].h) < 1e37f);
        W[((int64_t)a * n_prim + m) * NPK + s] = (double)acc[a].h + (double)acc[a].l;
      }
    if (bad) atomicOr(err, ERR_RANGE);
  }
}

using DtcWKernel = void (*)(const DtcBatch *, const int *, const int64_t *, const int64_t *, const int *,
                            const double *, const double *, int, int, int, const double *, int, double *, int, int *);
static DtcWKernel dtc_w_kernel(int nbl) {
  switch ((nbl + 3) / 4) {
    case 1: return k_dtc_w<4>;
    case 2: return k_dtc_w<8>;
    case 3: return k_dtc_w<12>;
    case 4: return k_dtc_w<16>;
    case 5: return k_dtc_w<20>;
    case 6: return k_dtc_w<24>;
    case 7: return k_dtc_w<28>;
    default: return k_dtc_w<32>;
  }
}

// Operands of the Gu GEMM: rows {b, c} of S over the batch's pair slots, and
// the rows (a, m) of W; zero beyond the batch's slots.
struct OpSPairs {
  const DtcBatch *info;
  const int *pairs_nz, *grid;
  const double *q;
  int ng, L, l_min;
  __device__ bool empty() const { return info->nslots <= 0; }
  __device__ double val(int64_t r, int64_t k) const {
    if (k >= info->nslots) return 0.0;
    const int pair = pairs_nz[info->slot0 + k];
    int b, c;
    pair_decode((int)r, b, c);
    const int k2 = grid[pair / ng] - l_min, k3 = grid[pair % ng] - l_min;
    const double *qb = q + (int64_t)b * L, *qc = q + (int64_t)c * L;
    return qb[k2] * qc[k3] + qc[k2] * qb[k3];
  }
};
struct OpWRows {
  const DtcBatch *info;
  const double *W;
  int NPK;
  __device__ bool empty() const { return info->nslots <= 0; }
  __device__ double val(int64_t r, int64_t k) const { return k < info->nslots ? W[r * NPK + k] : 0.0; }
};

// Gamma'[n][m] = Gu[{b,c}][(a,m)] + Gu[{a,c}][(b,m)] + Gu[{a,b}][(c,m)] for late mode n = (a, b, c)
__global__ void k_dtc_gather(const double *__restrict__ Gu, int nbl, int n_prim, const int *__restrict__ late,
                             int n_late, double *__restrict__ gamma) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_late * n_prim) return;
  const int n = (int)(idx / n_prim), m = (int)(idx % n_prim);
  const int a = late[3 * n], b = late[3 * n + 1], c = late[3 * n + 2];
  double v;
  if ((unsigned)a >= (unsigned)nbl || (unsigned)b >= (unsigned)nbl || (unsigned)c >= (unsigned)nbl) {
    v = __longlong_as_double(0x7ff8000000000000LL);
  } else {
    const int64_t rw = (int64_t)nbl * n_prim;
    v = Gu[pair_index(b, c) * rw + (int64_t)a * n_prim + m] + Gu[pair_index(a, c) * rw + (int64_t)b * n_prim + m] +
        Gu[pair_index(a, b) * rw + (int64_t)c * n_prim + m];
  }
  gamma[idx] = v;
}

// The grouped GEMM: one CTA per SM, items taken in a fixed stride.
static int grouped_gemm(const __nv_bfloat16 *As, const int *eA, const int *emaxA, int64_t rowsA,
                        const __nv_bfloat16 *Bs, const int *eB, const int *emaxB, int64_t rowsB, int Kpad, int wtile,
                        const int4 *items, const int *item_count, int max_items, double *Z, int nbp, int P2,
                        int *err, long long wait_cycles, int num_sms, cudaStream_t st, Profiler *prof) {
  CUtensorMap ta;
  BMaps tb;
  if (int r = make_slices_map(&ta, As, rowsA, Kpad, OZ_BM)) return r;
  if (int r = make_bmaps(&tb, Bs, rowsB, Kpad, 1u << (wtile / 16 - 1))) return r;
  OzParams P{};
  P.rowsA = rowsA;
  P.rowsB = rowsB;
  P.Kpad = Kpad;
  P.nchunks = (int)cdiv64(Kpad, OZ_KC);
  P.eA = eA;
  P.eB = eB;
  P.emaxA = emaxA;
  P.emaxB = emaxB;
  P.out = Z;
  P.err = err;
  P.wait_cycles = wait_cycles;
  P.nbp = nbp;
  P.items = items;
  P.item_count = item_count;
  P.P2 = P2;
  P.wtile = wtile;
  fill_mma_plans(P.plan);
  cudaError_t e = cudaFuncSetAttribute(k_ozaki_gemm<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  if (e == cudaSuccess) {
    ProfScope ps(prof, "dtc_gemm", st);
    const int grid = max(1, min(max_items, num_sms));
    k_ozaki_gemm<3><<<grid, OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_tc_err, sizeof g_tc_err, "direct grouped GEMM: %s", cudaGetErrorString(e));
    return MODAL_ECUDA;
  }
  return MODAL_OK;
}

// Shapes and scratch of the form.
struct DtcShape {
  int ng, nbp, nbl, n_x, L, n_late, n_prim, P2, P2l, cpt, nct, wu, urows, Kx, nchx, xs, cmax;
  int64_t npairs, Tcap, rowsA, rowsU, rowsW, nbatch;
  size_t scan_b, u_smem;
};
static DtcShape dtc_shape(const modal_problem *p, int ng) {
  DtcShape d{};
  d.ng = ng;
  d.nbp = p->nb_prim;
  d.nbl = p->nb_late;
  d.n_x = p->n_x;
  d.L = p->l_max - p->l_min + 1;
  d.n_late = p->n_late;
  d.n_prim = p->n_prim;
  d.P2 = d.nbp * (d.nbp + 1) / 2;
  d.P2l = d.nbl * (d.nbl + 1) / 2;
  d.cpt = OZ_BM / d.nbp;
  d.nct = (int)cdiv64(d.P2, OZ_BN);
  d.wu = g_tile_width(d.P2);
  d.urows = d.nct * d.wu;
  d.Kx = (int)pad32(d.n_x);
  d.nchx = (int)cdiv64(d.Kx, OZ_KC);
  d.xs = (int)std::min<int64_t>(OZ_KC, (160 * 1024) / (2 * (int64_t)d.nbp * (int64_t)sizeof(f2)));
  d.cmax = 3 * p->l_max / 2 + 2;
  d.npairs = (int64_t)ng * ng;
  d.Tcap = (int64_t)DTC_NT * d.cpt;
  d.rowsA = (int64_t)ng * d.nbp;
  d.rowsU = (int64_t)DTC_NP * d.urows;
  d.rowsW = (int64_t)d.nbl * d.n_prim;
  // batches: each ends at DTC_NT tiles, at DTC_NP pairs, or at the end
  const int64_t pairs_sorted = (int64_t)ng * (ng + 1) / 2;
  const int64_t tiles_bound = pairs_sorted + (int64_t)ng * (ng + 1) * (ng + 2) / 6 / d.cpt;
  d.nbatch = cdiv64(tiles_bound, DTC_NT) + cdiv64(pairs_sorted, DTC_NP);
  d.scan_b = scan_tmp_bytes(d.npairs);
  d.u_smem = dtc_u_smem(d.nbp, d.xs, d.urows, d.P2);
  return d;
}

struct DtcScratch {
  int *words;  // [0] status, exponent maxima: [3] q~ rows, [4] U, [5] S, [6] W
  double *ctab, *Z, *z, *Xb, *W, *Gu;
  int *crow, *cls, *pairs_nz, *tri;
  int64_t *tri_cnt, *tile_cnt, *nz_cnt, *tri_off, *tile_off, *slot_of, *tot;
  DtcBatch *info;
  int4 *items;
  void *scan_tmp;
  __nv_bfloat16 *As, *Us, *Ss, *Ws;
  int *eA, *eU, *eS, *eW;
  char *end;
};
static DtcScratch dtc_scratch(void *base, const DtcShape &d) {
  DtcScratch r{};
  char *w = (char *)base;
  r.words = (int *)w;
  w += 1024;
  auto take = [&](size_t bytes) {
    char *p = w;
    w += up256(bytes);
    return (void *)p;
  };
  r.ctab = (double *)take(sizeof(double) * (d.cmax + 1));
  r.crow = (int *)take(sizeof(int) * d.ng);
  r.cls = (int *)take(sizeof(int) * 2);
  r.tri_cnt = (int64_t *)take(sizeof(int64_t) * d.npairs);
  r.tile_cnt = (int64_t *)take(sizeof(int64_t) * d.npairs);
  r.nz_cnt = (int64_t *)take(sizeof(int64_t) * d.npairs);
  r.tri_off = (int64_t *)take(sizeof(int64_t) * d.npairs);
  r.tile_off = (int64_t *)take(sizeof(int64_t) * d.npairs);
  r.slot_of = (int64_t *)take(sizeof(int64_t) * d.npairs);
  r.pairs_nz = (int *)take(sizeof(int) * d.npairs);
  r.tot = (int64_t *)take(sizeof(int64_t) * 4);
  r.info = (DtcBatch *)take(sizeof(DtcBatch));
  r.scan_tmp = take(d.scan_b);
  r.As = (__nv_bfloat16 *)take((size_t)OZ_SLICES * d.rowsA * d.Kx * 2);
  r.eA = (int *)take(sizeof(int) * (size_t)d.nchx * d.rowsA);
  r.Us = (__nv_bfloat16 *)take((size_t)OZ_SLICES * d.rowsU * d.Kx * 2);
  r.eU = (int *)take(sizeof(int) * (size_t)d.nchx * d.rowsU);
  r.items = (int4 *)take(sizeof(int4) * (size_t)DTC_NT * d.nct);
  r.Z = (double *)take(sizeof(double) * (size_t)d.Tcap * d.nbp * d.P2);
  r.tri = (int *)take(sizeof(int) * 3 * (size_t)d.Tcap);
  r.z = (double *)take(sizeof(double) * (size_t)d.Tcap);
  r.Xb = (double *)take(sizeof(double) * (size_t)d.Tcap * d.n_prim);
  r.W = (double *)take(sizeof(double) * (size_t)d.rowsW * DTC_NP);
  r.Ss = (__nv_bfloat16 *)take((size_t)OZ_SLICES * d.P2l * DTC_NP * 2);
  r.eS = (int *)take(sizeof(int) * (size_t)d.P2l);
  r.Ws = (__nv_bfloat16 *)take((size_t)OZ_SLICES * d.rowsW * DTC_NP * 2);
  r.eW = (int *)take(sizeof(int) * (size_t)d.rowsW);
  r.Gu = (double *)take(sizeof(double) * (size_t)d.P2l * d.rowsW);
  r.end = w;
  return r;
}

static_assert(DTC_NP % OZ_BK == 0 && DTC_NP <= OZ_KC, "the pair slots of a batch are one exact K chunk");
bool tc_direct_supported(int nb_late, int nb_prim) {
  return nb_late >= 1 && nb_late <= DTC_MAXNB && nb_prim >= 1 && nb_prim <= DTC_MAXNB;
}

size_t tc_direct_scratch_bytes(const modal_problem *p, int ng) {
  const DtcShape d = dtc_shape(p, ng);
  return (size_t)(dtc_scratch(nullptr, d).end - (char *)nullptr) + 256;
}

#define DTC_CK(call, what)                                                         \
  do {                                                                             \
    const cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                       \
      snprintf(g_tc_err, sizeof g_tc_err, "%s: %s", what, cudaGetErrorString(e_)); \
      return MODAL_ECUDA;                                                          \
    }                                                                              \
  } while (0)

int tc_project_direct(const modal_problem *p, const int *grid, const double *dw, int ng, int mode, double *gamma,
                      void *scratch, int num_sms, long long wc, cudaStream_t st, Profiler *prof) {
  if (!tc_direct_supported(p->nb_late, p->nb_prim)) {
    snprintf(g_tc_err, sizeof g_tc_err, "the tensor-core direct form takes bases of at most %d functions",
             DTC_MAXNB);
    return MODAL_EUNSUPPORTED;
  }
  const DtcShape d = dtc_shape(p, ng);
  const DtcScratch s = dtc_scratch(scratch, d);
  int *words = s.words;
  DTC_CK(cudaMemsetAsync(words, 0, sizeof(int), st), "status reset");
  DTC_CK(launch_zero(s.Gu, (size_t)d.P2l * d.rowsW, st), "zero");
  {
    ProfScope ps(prof, "dtc_setup", st);
    DTC_CK(launch_threej_table(d.cmax, s.ctab, st), "3j table");
    k_dtc_classes<<<1, 32, 0, st>>>(ng, grid, mode, s.crow, s.cls);
    k_dtc_count<<<(unsigned)cdiv64(d.npairs, 256), 256, 0, st>>>(ng, grid, s.crow, s.cls, mode, d.cpt, s.tri_cnt,
                                                                  s.tile_cnt, s.nz_cnt);
    DTC_CK(cudaGetLastError(), "count");
    DTC_CK(scan_exclusive_i64(s.scan_tmp, d.scan_b, s.tri_cnt, s.tri_off, d.npairs, st), "scan");
    DTC_CK(scan_exclusive_i64(s.scan_tmp, d.scan_b, s.tile_cnt, s.tile_off, d.npairs, st), "scan");
    DTC_CK(scan_exclusive_i64(s.scan_tmp, d.scan_b, s.nz_cnt, s.slot_of, d.npairs, st), "scan");
    k_dtc_totals<<<1, 32, 0, st>>>(d.npairs, s.tri_cnt, s.tri_off, s.tile_cnt, s.tile_off, s.nz_cnt, s.slot_of,
                                   s.tot);
    k_dtc_compact<<<(unsigned)cdiv64(d.npairs, 256), 256, 0, st>>>(d.npairs, s.nz_cnt, s.slot_of, s.pairs_nz);
    DTC_CK(cudaGetLastError(), "totals");
  }
  // the A operand: q~ rows of the grid in class order, once per call
  k_reset_emax<<<1, 32, 0, st>>>(words + 3, 2);
  if (int r = split_op(d.rowsA, (int64_t)d.n_x, d.Kx, OpQRows{p->qt, grid, s.crow, d.L, p->l_min, d.nbp}, s.As,
                       s.eA, words + 3, words, st, prof, "dtc_split_q"))
    return r;
  DTC_CK(cudaFuncSetAttribute(k_dtc_make_u, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.u_smem), "attr");
  const size_t x_smem = sizeof(double) * (size_t)d.nbp * d.P2;
  DTC_CK(cudaFuncSetAttribute(k_dtc_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x_smem), "attr");
  for (int64_t b = 0; b < d.nbatch; ++b) {
    {
      ProfScope ps(prof, "dtc_fill", st, 2);
      k_dtc_info<<<1, 32, 0, st>>>(d.nct, d.cpt, d.npairs, s.tile_off, s.tri_off, s.slot_of, s.pairs_nz, s.tot,
                                   s.info);
      k_dtc_fill<<<(unsigned)cdiv64(d.Tcap, 256), 256, 0, st>>>(s.info, s.tri_off, d.npairs, ng, grid, s.crow, s.cls,
                                                                 mode, dw, p->w_l, p->l_min, s.ctab, s.tri, s.z);
      DTC_CK(cudaGetLastError(), "fill");
    }
    {
      ProfScope ps(prof, "dtc_make_u", st, 2);
      k_reset_emax<<<1, 32, 0, st>>>(words + 4, 1);
      k_dtc_make_u<<<dim3(DTC_NP, d.nchx), 256, d.u_smem, st>>>(s.info, s.pairs_nz, ng, grid, p->l_min, d.L, d.nbp,
                                                                 d.n_x, p->qt, p->x_w, d.P2, d.urows, d.Kx, d.xs,
                                                                 d.rowsU, s.Us, s.eU, words + 4, words);
      DTC_CK(cudaGetLastError(), "make_u");
    }
    {
      ProfScope ps(prof, "dtc_items", st);
      k_dtc_items<<<(unsigned)cdiv64(DTC_NT, 128), 128, 0, st>>>(s.info, s.tile_off, s.tri_off, s.slot_of, d.npairs,
                                                                   ng, grid, s.crow, s.cls, mode, d.cpt, d.nbp, d.nct,
                                                                   d.wu, d.urows, s.items);
      DTC_CK(cudaGetLastError(), "items");
    }
    if (int r = grouped_gemm(s.As, s.eA, words + 3, d.rowsA, s.Us, s.eU, words + 4, d.rowsU, d.Kx, d.wu, s.items,
                             &s.info->n_items, DTC_NT * d.nct, s.Z, d.nbp, d.P2, words, wc, num_sms, st, prof))
      return r;
    {
      ProfScope ps(prof, "dtc_x", st);
      k_dtc_x<<<(unsigned)d.Tcap, 256, x_smem, st>>>(s.info, s.Z, d.nbp, d.P2, p->prim_modes, d.n_prim, s.Xb);
      DTC_CK(cudaGetLastError(), "X");
    }
    {
      ProfScope ps(prof, "dtc_w", st);
      dtc_w_kernel(d.nbl)<<<dim3(DTC_NP, (unsigned)cdiv64(d.n_prim, DTC_WTH)), DTC_WTH, 0, st>>>(
          s.info, s.pairs_nz, s.tri_off, s.tri_cnt, s.tri, s.z, p->q, d.L, p->l_min, d.nbl, s.Xb, d.n_prim, s.W,
          DTC_NP, words);
      DTC_CK(cudaGetLastError(), "W");
    }
    k_reset_emax<<<1, 32, 0, st>>>(words + 5, 2);
    if (int r = split_op((int64_t)d.P2l, (int64_t)DTC_NP, DTC_NP,
                         OpSPairs{s.info, s.pairs_nz, grid, p->q, ng, d.L, p->l_min}, s.Ss, s.eS, words + 5, words,
                         st, prof, "dtc_split_sw"))
      return r;
    if (int r = split_op(d.rowsW, (int64_t)DTC_NP, DTC_NP, OpWRows{s.info, s.W, DTC_NP}, s.Ws, s.eW, words + 6,
                         words, st, prof, "dtc_split_sw"))
      return r;
    if (int r = dense_gemm(s.Ss, s.eS, words + 5, d.P2l, s.Ws, s.eW, words + 6, d.rowsW, DTC_NP, s.Gu, d.rowsW, 1,
                           true, words, wc, st, prof, "dtc_gemm_gu", &s.info->nslots, 0))
      return r;
  }
  {
    ProfScope ps(prof, "dtc_gather", st);
    k_dtc_gather<<<(unsigned)cdiv64((int64_t)d.n_late * d.n_prim, 256), 256, 0, st>>>(s.Gu, d.nbl, d.n_prim,
                                                                                     p->late_modes, d.n_late, gamma);
    DTC_CK(cudaGetLastError(), "gather");
  }
  return MODAL_OK;
}
#undef DTC_CK

// status words of a triple-product scratch used without the l contraction
// of this form: mode 1 at the start of a call (error bits and all maxima),
// mode 0 before each chunk (the maxima)
cudaError_t tc_init_words(void *scratch, const SepShape &s, int nxl_max, int mode, cudaStream_t st) {
  const LScratch r = l_scratch(scratch, s, nxl_max);
  k_init_words<<<1, 32, 0, st>>>(r.words, mode);
  return cudaGetLastError();
}
__global__ void k_or_word(int *dst, const int *src) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst |= *src;
}
cudaError_t tc_or_status(int *dst, void *scratch, cudaStream_t st) {
  k_or_word<<<1, 32, 0, st>>>(dst, (const int *)scratch);
  return cudaGetLastError();
}

int *tc_error_word(void *scratch) { return (int *)scratch; }

void tc_release(int) {}

}  // namespace modal
