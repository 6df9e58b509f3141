// tc.cu -- tensor-core (tcgen05) form of the separable path with exponent-
// aligned BF16 splitting (Ozaki, Ogita, Oishi & Rump 2012).
//
// Both dense contractions of the separable path -- the l contraction of
// Eq. legendre and the slice reduction of the triple product of Eq. 2D --
// run as C = A B^T over K on 5th-generation tensor cores:
//
//  * every row of A and B is scaled by a power of two 2^e (per K chunk) so
//    that |x / 2^e| <= 1, then written as five BF16 slices of 7 bits each:
//    x / 2^e * 2^7 = q0 + q1 2^-7 + q2 2^-14 + ...,  |q0| <= 128, |qs| <= 64;
//  * the 15 slice products with s + t <= 4 are issued as tcgen05.mma into
//    three TMEM accumulators: level 0 (q0 q0'), level 1 (q0 q1' + q1 q0') and
//    levels 2-4.  With at most 1024 K terms per chunk the level-0 and level-1
//    partial sums are integers (in units of 1 and 2^-7) below 2^24, hence
//    exact in the FP32 accumulator whatever the summation order;
//  * at the end of each chunk the epilogue warps read the accumulators
//    (tcgen05.ld), apply the row and column scales and add the chunk into a
//    double-FP32 (hi, lo) running sum held in registers, offset by a global
//    exponent bias so that the FP32 range cannot overflow.  The result is
//    written (or added) in FP64.
//
// Operands are staged by TMA (cp.async.bulk.tensor, 64-byte swizzle) in a
// two-stage mbarrier pipeline; one thread issues the MMAs.  Every wait is
// bounded: on give-up the CTA raises an error word, drains its copies in
// flight, frees TMEM and returns.
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace modal {

static thread_local char g_tc_err[256] = "";
const char *tc_last_error() { return g_tc_err; }

constexpr int OZ_BETA = 7;        // bits per slice
constexpr int OZ_SLICES = 5;      // slices per operand
constexpr int OZ_MAXLEV = 4;      // products with s + t <= 4
constexpr int OZ_KC = 1024;       // K terms per exact chunk
constexpr int OZ_BM = 128;        // rows per tile (TMEM lanes)
constexpr int OZ_BN = 128;        // columns per tile
constexpr int OZ_BK = 32;         // K per stage: 64-byte rows, 64-byte swizzle
constexpr int OZ_STAGES = 2;
constexpr int OZ_ROWB = OZ_BK * 2;                       // bytes per smem row
constexpr int OZ_A_BYTES = OZ_SLICES * OZ_BM * OZ_ROWB;  // 40 KB
constexpr int OZ_B_BYTES = OZ_SLICES * OZ_BN * OZ_ROWB;  // 40 KB
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;       // TMA warp, MMA warp, epilogue
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long OZ_WAIT_CYCLES = 4000000000LL;       // ~2 s at 2 GHz
static_assert(OZ_KC % OZ_BK == 0, "chunk must hold whole stages");

// error word bits
constexpr int ERR_TIMEOUT = 1;

// ---------------------------------------------------------------------------
// Splitting helpers (FP64 input)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int exp_bound(double m) {  // smallest e with m <= 2^e
  if (!(m > 0.0)) return -100000;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// Write the five slices of x / 2^e as BF16 values q_s 2^(-7 s).
__device__ __forceinline__ void split5(double x, int e, __nv_bfloat16 *out, int64_t slice_stride) {
  if (e < -99999) {
#pragma unroll
    for (int s = 0; s < OZ_SLICES; ++s) out[s * slice_stride] = __float2bfloat16_rn(0.f);
    return;
  }
  double r = ldexp(x, OZ_BETA - e);
#pragma unroll
  for (int s = 0; s < OZ_SLICES; ++s) {
    double q = rint(r);
    r = (r - q) * (double)(1 << OZ_BETA);
    out[s * slice_stride] = __float2bfloat16_rn((float)ldexp(q, -OZ_BETA * s));
  }
}

// Rows of the l-contraction operands.  Row r of A is A[j][l] q_a(l) with
// r = (j, a); row r of B is q~_p(l, x0 + xl) with r = (xl, p).  One warp per
// (row, K chunk): pass 1 finds max |x|, pass 2 writes the slices.
template <bool IS_A>
__global__ void k_split_lrows(int64_t rows, int L, int Kpad, const double *__restrict__ Atab,
                              const double *__restrict__ q, const double *__restrict__ qt, int nbl, int nbp,
                              int x0, __nv_bfloat16 *__restrict__ out, int *__restrict__ ex,
                              int *__restrict__ emax) {
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
  double m = 0.0;
  for (int l = l0 + lane; l < l1; l += 32) m = fmax(m, fabs(val(l)));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = exp_bound(m);
  const int64_t sstride = rows * (int64_t)Kpad;
  const int lend = min(Kpad, l0 + OZ_KC);
  for (int l = l0 + lane; l < lend; l += 32) {
    double v = l < L ? val(l) : 0.0;
    split5(v, e, out + r * Kpad + l, sstride);
  }
  if (lane == 0) {
    ex[(int64_t)ch * rows + r] = e;
    if (e > -99999) atomicMax(emax, e);
  }
}

// words[0] = error bits (cleared once per call), words[1..] = exponent maxima
__global__ void k_init_words(int *w, int reset_err) {
  if (threadIdx.x == 0) {
    if (reset_err) w[0] = 0;
  } else if (threadIdx.x < 8) {
    w[threadIdx.x] = -100000;
  }
}

// ---------------------------------------------------------------------------
// The GEMM kernel.
// OUT_MODE 0: l contraction, store M[(xl*n_mu + j)*nbl + a)*nbp + p] from row
//             (j, a) and column (xl, p).
// OUT_MODE 1: triple product, add into the G block of b (rows (a,{u,v}),
//             columns (c,t), c >= b) -- tiles decoded from blockIdx.x.
// ---------------------------------------------------------------------------
struct OzParams {
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
  // OUT_MODE 1
  GLayout g;
  long long wait_cycles;
};

__device__ __forceinline__ void df_add(float &hi, float &lo, float bh, float bl) {
  float s = hi + bh;
  float bb = s - hi;
  float e = (hi - (s - bb)) + (bh - bb);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

template <int OUT_MODE>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams P) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(sm + OZ_STAGES * OZ_STAGE_BYTES);
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
  if (OUT_MODE == 0) {
    a_row0 = (int64_t)blockIdx.x * OZ_BM;
    b_row0 = (int64_t)blockIdx.y * OZ_BN;
    R = min((int64_t)OZ_BM, P.rowsA - a_row0);
    C = min((int64_t)OZ_BN, P.rowsB - b_row0);
  } else {
    int t = blockIdx.x, rt = 0, ct = 0;
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
    a_row0 = rowoff + (int64_t)rt * OZ_BM;
    b_row0 = (int64_t)bblk * P.g.nbp + (int64_t)ct * OZ_BN;
    R = min((int64_t)OZ_BM, P.g.rows(bblk) - (int64_t)rt * OZ_BM);
    C = min((int64_t)OZ_BN, P.g.cols(bblk) - (int64_t)ct * OZ_BN);
    out_base = P.g.offset(bblk) + (int64_t)rt * OZ_BM * P.g.cols(bblk) + (int64_t)ct * OZ_BN;
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
  const int ksteps = P.Kpad / OZ_BK;
  const int steps_per_chunk = OZ_KC / OZ_BK;

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      ptx::prefetch_tmap(&tmB);
      int issued = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % OZ_STAGES;
        const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
        if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) break;
        unsigned char *st = sm + s * OZ_STAGE_BYTES;
        ptx::mbar_arrive_expect_tx(&full[s], OZ_STAGE_BYTES);
        ptx::tma_load_3d(st, &tmA, &full[s], i * OZ_BK, (int)a_row0, 0);
        ptx::tma_load_3d(st + OZ_A_BYTES, &tmB, &full[s], i * OZ_BK, (int)b_row0, 0);
        ++issued;
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
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(OZ_BM, OZ_BN);
      const uint32_t sbase = ptx::smem_u32(sm);
      int chunk = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % OZ_STAGES;
        const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
        const bool chunk_start = (i % steps_per_chunk) == 0;
        if (chunk_start && chunk > 0) {
          // accumulators must have been drained by the epilogue
          if (!ptx::mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), abort_flag, P.wait_cycles)) break;
        }
        if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) break;
        ptx::tc_fence_after();
        const uint32_t a0 = sbase + s * OZ_STAGE_BYTES;
        const uint32_t b0 = a0 + OZ_A_BYTES;
        bool fresh[3] = {chunk_start, chunk_start, chunk_start};
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
          for (int sa = 0; sa < OZ_SLICES; ++sa) {
#pragma unroll
            for (int sb = 0; sb < OZ_SLICES; ++sb) {
              if (sa + sb > OZ_MAXLEV) continue;
              const int lev = sa + sb < 2 ? sa + sb : 2;
              const uint64_t ad = ptx::smem_desc(a0 + sa * OZ_BM * OZ_ROWB + kk * 32, 16, 8 * OZ_ROWB, ptx::SW_64B);
              const uint64_t bd = ptx::smem_desc(b0 + sb * OZ_BN * OZ_ROWB + kk * 32, 16, 8 * OZ_ROWB, ptx::SW_64B);
              ptx::mma_bf16(tmem + lev * OZ_BN, ad, bd, idesc, fresh[lev] ? 0u : 1u);
              fresh[lev] = false;
            }
          }
        }
        ptx::mma_commit(&empty[s]);  // stage s may be refilled once these MMAs retire
        const bool chunk_end = ((i + 1) % steps_per_chunk) == 0 || i + 1 == ksteps;
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
    const int ebias = (*P.emaxA) + (*P.emaxB) + 40;
    float hi[64], lo[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
    bool ok = true;
    for (int ch = 0; ch < P.nchunks; ++ch) {
      if (!ptx::mbar_wait(acc_full, (uint32_t)(ch & 1), abort_flag, P.wait_cycles)) { ok = false; break; }
      ptx::tc_fence_after();
      const int ea = (a_row0 + row < P.rowsA) ? P.eA[(int64_t)ch * P.rowsA + a_row0 + row] : -100000;
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < 4; ++cb) {
        float v0[16], v1[16], v2[16];
        const uint32_t cc = (uint32_t)(col0 + cb * 16);
        ptx::tmem_ld16(tl + cc, v0);
        ptx::tmem_ld16(tl + OZ_BN + cc, v1);
        ptx::tmem_ld16(tl + 2 * OZ_BN + cc, v2);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int c = cb * 16 + k;
          const int64_t bcol = b_row0 + col0 + c;
          const int eb = (bcol < P.rowsB) ? __ldg(P.eB + (int64_t)ch * P.rowsB + bcol) : -100000;
          if (ea < -99999 || eb < -99999) continue;
          // exact level-0 and level-1 sums, then the rest
          float s = v0[k] + v1[k];
          float bb = s - v0[k];
          float e = (v0[k] - (s - bb)) + (v1[k] - bb);
          e += v2[k];
          const int sh = ea + eb - 2 * OZ_BETA - ebias;
          df_add(hi[c], lo[c], ldexpf(s, sh), ldexpf(e, sh));
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(acc_empty);
    }
    if (ok && !*abort_flag && row < R) {
#pragma unroll 4
      for (int c = 0; c < 64; ++c) {
        const int col = col0 + c;
        if (col >= C) continue;
        const double v = ldexp((double)hi[c] + (double)lo[c], ebias);
        if (OUT_MODE == 0) {
          const int64_t rA = a_row0 + row, rB = b_row0 + col;
          const int j = (int)(rA / P.nbl), a = (int)(rA % P.nbl);
          const int xl = (int)(rB / P.nbp), p = (int)(rB % P.nbp);
          P.out[(((int64_t)xl * P.n_mu + j) * P.nbl + a) * P.nbp + p] = v;
        } else {
          double *d = P.out + out_base + (int64_t)row * P.g.cols(bblk) + col;
          *d += v;
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
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 3-D map over [slices][rows][Kpad] BF16, box (OZ_BK, box_rows, slices), 64-byte swizzle.
static int make_slices_map(CUtensorMap *m, const void *base, int64_t rows, int Kpad, int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    snprintf(g_tc_err, sizeof g_tc_err, "cuTensorMapEncodeTiled unavailable");
    return MODAL_EUNSUPPORTED;
  }
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)OZ_SLICES};
  cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)rows * Kpad * 2};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, (cuuint32_t)OZ_SLICES};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    snprintf(g_tc_err, sizeof g_tc_err, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MODAL_EINVAL;
  }
  return MODAL_OK;
}

static size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// scratch for one radial chunk: l-contraction slices + exponents, error word
size_t tc_scratch_bytes(const SepShape &s, int nxc) {
  const int Kpad = cdiv(s.L, OZ_BK) * OZ_BK;
  const int nch = cdiv(s.L, OZ_KC);
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl, rowsB = (int64_t)nxc * s.nbp;
  size_t b = 0;
  b += up256((size_t)OZ_SLICES * rowsA * Kpad * 2) + up256((size_t)OZ_SLICES * rowsB * Kpad * 2);
  b += up256((size_t)nch * rowsA * 4) + up256((size_t)nch * rowsB * 4);
  b += 256 * 4;
  b += tc_triple_scratch_bytes(s, nxc);
  return b + 1024;
}

int tc_contract_l(const SepShape &s, const double *A, const double *q, const double *qt, int x0, int nxc,
                  double *M, void *scratch, long long wait_cycles, cudaStream_t st, char **scratch_end,
                  bool reset_err) {
  const int Kpad = cdiv(s.L, OZ_BK) * OZ_BK;
  const int nch = cdiv(s.L, OZ_KC);
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl, rowsB = (int64_t)nxc * s.nbp;
  // status words first, at a fixed offset whatever the chunk size:
  // [0] error bits, [1] emaxA, [2] emaxB, [3] emax of the triple's B, [4] of Y
  char *w = (char *)scratch;
  int *words = (int *)w; w += 256 * 4;
  __nv_bfloat16 *As = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * rowsA * Kpad * 2);
  __nv_bfloat16 *Bs = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * rowsB * Kpad * 2);
  int *eA = (int *)w; w += up256((size_t)nch * rowsA * 4);
  int *eB = (int *)w; w += up256((size_t)nch * rowsB * 4);
  if (scratch_end) *scratch_end = w;
  cudaError_t e;
  k_init_words<<<1, 32, 0, st>>>(words, reset_err ? 1 : 0);
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  {
    const int64_t wa = rowsA * nch, wb = rowsB * nch;
    k_split_lrows<true><<<(unsigned)cdiv64(wa * 32, 256), 256, 0, st>>>(rowsA, s.L, Kpad, A, q, qt, s.nbl, s.nbp,
                                                                      x0, As, eA, words + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
    k_split_lrows<false><<<(unsigned)cdiv64(wb * 32, 256), 256, 0, st>>>(rowsB, s.L, Kpad, A, q, qt, s.nbl,
                                                                       s.nbp, x0, Bs, eB, words + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  }
  {
    CUtensorMap ta, tb;
    if (int r = make_slices_map(&ta, As, rowsA, Kpad, OZ_BM)) return r;
    if (int r = make_slices_map(&tb, Bs, rowsB, Kpad, OZ_BN)) return r;
    OzParams P{};
    P.rowsA = rowsA;
    P.rowsB = rowsB;
    P.Kpad = Kpad;
    P.nchunks = nch;
    P.eA = eA;
    P.eB = eB;
    P.emaxA = words + 1;
    P.emaxB = words + 2;
    P.out = M;
    P.err = words;
    P.n_mu = s.n_mu;
    P.nbl = s.nbl;
    P.nbp = s.nbp;
    P.wait_cycles = wait_cycles;
    if ((e = cudaFuncSetAttribute(k_ozaki_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
        cudaSuccess)
      goto cuda_fail;
    dim3 grid((unsigned)cdiv64(rowsA, OZ_BM), (unsigned)cdiv64(rowsB, OZ_BN));
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
struct f2 {
  float h, l;
};
__device__ __forceinline__ f2 df_from_d(double x) {
  float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
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

// Slices of a double-FP32 value y with |y| <= 2^e: q_s 2^(-7 s).
__device__ __forceinline__ void split5_df(f2 y, int e, __nv_bfloat16 (&out)[OZ_SLICES]) {
  if (e < -99999) {
#pragma unroll
    for (int s = 0; s < OZ_SLICES; ++s) out[s] = __float2bfloat16_rn(0.f);
    return;
  }
  float h = ldexpf(y.h, OZ_BETA - e), l = ldexpf(y.l, OZ_BETA - e);
#pragma unroll
  for (int s = 0; s < OZ_SLICES; ++s) {
    float q = rintf(h);
    f2 r = df_two_sum(h - q, l);  // h - q is exact (|h - q| <= 1/2)
    out[s] = __float2bfloat16_rn(ldexpf(q, -OZ_BETA * s));
    h = r.h * (float)(1 << OZ_BETA);
    l = r.l * (float)(1 << OZ_BETA);
  }
}

// Per chunk of OZ_KC slices and block of 64 columns: exact max |M| (B-operand
// exponent), max sqrt(w)|M| (Y bound), double-FP32 copy of M and of w, and the
// K-major BF16 slices of M.
constexpr int TP_COLS = 64;
__global__ void __launch_bounds__(256) k_tp_prep_cols(int64_t K, int Kpad, int nblp, int n_mu, int x0,
                                                      const double *__restrict__ M, const double *__restrict__ om,
                                                      const double *__restrict__ xw, f2 *__restrict__ Mdf,
                                                      f2 *__restrict__ wdf, double *__restrict__ mxW,
                                                      int *__restrict__ eB, __nv_bfloat16 *__restrict__ Bt,
                                                      int *__restrict__ emaxB) {
  __shared__ double red1[4][TP_COLS], red2[4][TP_COLS];
  __shared__ int esh[TP_COLS];
  __shared__ __nv_bfloat16 tile[OZ_SLICES][TP_COLS][32 + 8];
  const int ch = blockIdx.y;
  const int c0 = blockIdx.x * TP_COLS;
  const int tc = threadIdx.x % TP_COLS, tk = threadIdx.x / TP_COLS;  // 64 cols x 4 k-lanes
  const int col = c0 + tc;
  const int64_t k0 = (int64_t)ch * OZ_KC, k1 = min(K, k0 + OZ_KC);
  double m1 = 0.0, m2 = 0.0;
  if (col < nblp) {
    for (int64_t k = k0 + tk; k < k1; k += 4) {
      const double v = M[k * nblp + col];
      const double w = om[k % n_mu] * xw[x0 + k / n_mu];
      m1 = fmax(m1, fabs(v));
      m2 = fmax(m2, sqrt(w) * fabs(v));
      Mdf[k * nblp + col] = df_from_d(v);
      if (col == 0) wdf[k] = df_from_d(w);
    }
  }
  red1[tk][tc] = m1;
  red2[tk][tc] = m2;
  __syncthreads();
  if (tk == 0) {
    for (int i = 1; i < 4; ++i) {
      m1 = fmax(m1, red1[i][tc]);
      m2 = fmax(m2, red2[i][tc]);
    }
    const int e = exp_bound(m1);
    esh[tc] = e;
    if (col < nblp) {
      eB[(int64_t)ch * nblp + col] = e;
      mxW[(int64_t)ch * nblp + col] = m2 * (1.0 + 1e-12);  // room for the rounding of sqrt(w)
      if (e > -99999) atomicMax(emaxB, e);
    }
  }
  __syncthreads();
  const int e = esh[tc];
  const int64_t kpend = min((int64_t)Kpad, k0 + OZ_KC);
  for (int64_t kt = k0; kt < kpend; kt += 32) {
    // each thread splits 8 k of its column
    for (int i = 0; i < 8; ++i) {
      const int kk = tk * 8 + i;
      const int64_t k = kt + kk;
      const double v = (col < nblp && k < K) ? M[k * nblp + col] : 0.0;
      __nv_bfloat16 o[OZ_SLICES];
      split5_df(df_from_d(v), e, o);
#pragma unroll
      for (int s = 0; s < OZ_SLICES; ++s) tile[s][tc][kk] = o[s];
    }
    __syncthreads();
    // write: per (slice, column) one 64-byte row of 32 k
    for (int idx = threadIdx.x; idx < OZ_SLICES * TP_COLS * 4; idx += 256) {
      const int part = idx & 3, cc = (idx >> 2) % TP_COLS, s = idx / (4 * TP_COLS);
      if (c0 + cc < nblp && kt + part * 8 < Kpad) {
        const uint4 *src = reinterpret_cast<const uint4 *>(&tile[s][cc][part * 8]);
        uint4 *dst = reinterpret_cast<uint4 *>(Bt + ((int64_t)s * nblp + c0 + cc) * Kpad + kt + part * 8);
        *dst = *src;
      }
    }
    __syncthreads();
  }
}

// Y rows: global row r -> (b, a, uv) with rows ordered by b, then a, then uv.
__device__ __forceinline__ void y_row_decode(int64_t r, int P2, int &b, int &a, int &u, int &v) {
  // rows before block b: P2 * b (b + 1) / 2
  int bb = (int)((sqrt(8.0 * (double)(r / P2) + 1.0) - 1.0) * 0.5);
  while ((int64_t)P2 * bb * (bb + 1) / 2 > r) --bb;
  while ((int64_t)P2 * (bb + 1) * (bb + 2) / 2 <= r) ++bb;
  const int64_t loc = r - (int64_t)P2 * bb * (bb + 1) / 2;
  b = bb;
  a = (int)(loc / P2);
  pair_decode((int)(loc % P2), u, v);
}

constexpr int TY_ROWS = 64, TY_K = 64;
__global__ void __launch_bounds__(256) k_tp_make_y(int64_t rowsY, int64_t K, int Kpad, int nbp, int nblp, int P2,
                                                   const f2 *__restrict__ Mdf, const f2 *__restrict__ wdf,
                                                   const double *__restrict__ mxW, int *__restrict__ eY,
                                                   __nv_bfloat16 *__restrict__ Ysl, int *__restrict__ emaxY) {
  __shared__ __nv_bfloat16 tile[OZ_SLICES][TY_ROWS][TY_K + 8];
  const int64_t r0 = (int64_t)blockIdx.x * TY_ROWS;
  const int64_t kb = (int64_t)blockIdx.y * TY_K;
  const int ch = (int)(kb / OZ_KC);
  const int tr = threadIdx.x % TY_ROWS, tk = threadIdx.x / TY_ROWS;  // 64 rows x 4 k-lanes
  const int64_t r = r0 + tr;
  int b = 0, a = 0, u = 0, v = 0, e = -100000;
  if (r < rowsY) {
    y_row_decode(r, P2, b, a, u, v);
    const double *mw = mxW + (int64_t)ch * nblp;
    const double bound = mw[a * nbp + u] * mw[b * nbp + v] + mw[a * nbp + v] * mw[b * nbp + u];
    e = exp_bound(bound);
    if (tk == 0 && (kb % OZ_KC) == 0) {
      eY[(int64_t)ch * rowsY + r] = e;
      if (e > -99999) atomicMax(emaxY, e);
    }
  }
  for (int i = 0; i < TY_K / 4; ++i) {
    const int kk = tk * (TY_K / 4) + i;
    const int64_t k = kb + kk;
    __nv_bfloat16 o[OZ_SLICES];
    f2 y = {0.f, 0.f};
    if (r < rowsY && k < K) {
      const f2 *Mk = Mdf + k * nblp;
      const f2 s = df_addv(df_mul(Mk[a * nbp + u], Mk[b * nbp + v]), df_mul(Mk[a * nbp + v], Mk[b * nbp + u]));
      y = df_mul(wdf[k], s);
    }
    split5_df(y, e, o);
#pragma unroll
    for (int s = 0; s < OZ_SLICES; ++s) tile[s][tr][kk] = o[s];
  }
  __syncthreads();
  // write 64-row x 64-k tiles: per (slice, row) 128 bytes = 8 x 16 B
  for (int idx = threadIdx.x; idx < OZ_SLICES * TY_ROWS * 8; idx += 256) {
    const int part = idx & 7, rr = (idx >> 3) % TY_ROWS, s = idx / (8 * TY_ROWS);
    const int64_t kk = kb + part * 8;
    if (r0 + rr < rowsY && kk < Kpad) {
      const uint4 *src = reinterpret_cast<const uint4 *>(&tile[s][rr][part * 8]);
      uint4 *dst = reinterpret_cast<uint4 *>(Ysl + ((int64_t)s * rowsY + r0 + rr) * Kpad + kk);
      *dst = *src;
    }
  }
}

static int64_t y_rows(const SepShape &s) {
  const int64_t P2 = (int64_t)s.nbp * (s.nbp + 1) / 2;
  return P2 * s.nbl * (s.nbl + 1) / 2;
}

size_t tc_triple_scratch_bytes(const SepShape &s, int nxc) {
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int64_t nblp = (int64_t)s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  const int64_t rowsY = y_rows(s);
  size_t b = 0;
  b += up256((size_t)K * nblp * 8) + up256((size_t)K * 8);            // Mdf, wdf
  b += up256((size_t)nch * nblp * 8) + up256((size_t)nch * nblp * 4);  // mxW, eB
  b += up256((size_t)OZ_SLICES * nblp * Kpad * 2);                     // Bt
  b += up256((size_t)nch * rowsY * 4);                                 // eY
  b += up256((size_t)OZ_SLICES * rowsY * Kpad * 2);                    // Y slices
  return b;
}

int tc_separable_chunk(const SepShape &s, const double *A, const double *q, const double *qt, const double *om,
                       const double *xw, int x0, int nxc, double *M, double *G, bool accumulate, void *scratch,
                       int num_sms, long long wait_cycles, cudaStream_t st) {
  (void)num_sms;
  char *w = nullptr;
  if (int r = tc_contract_l(s, A, q, qt, x0, nxc, M, scratch, wait_cycles, st, &w, !accumulate)) return r;
  int *words = (int *)scratch;  // status words written by tc_contract_l
  cudaError_t e;
  const int64_t K = (int64_t)nxc * s.n_mu;
  const int Kpad = (int)(cdiv64(K, 64) * 64);
  const int nblp = s.nbl * s.nbp;
  const int nch = (int)cdiv64(K, OZ_KC);
  const int64_t rowsY = y_rows(s);
  const int P2 = s.nbp * (s.nbp + 1) / 2;
  f2 *Mdf = (f2 *)w; w += up256((size_t)K * nblp * 8);
  f2 *wdf = (f2 *)w; w += up256((size_t)K * 8);
  double *mxW = (double *)w; w += up256((size_t)nch * nblp * 8);
  int *eB = (int *)w; w += up256((size_t)nch * nblp * 4);
  __nv_bfloat16 *Bt = (__nv_bfloat16 *)w; w += up256((size_t)OZ_SLICES * nblp * Kpad * 2);
  int *eY = (int *)w; w += up256((size_t)nch * rowsY * 4);
  __nv_bfloat16 *Ysl = (__nv_bfloat16 *)w;
  if (!accumulate) {
    GLayout g = make_glayout(s.nbl, s.nbp);
    if ((e = launch_zero(G, (size_t)g.size(), st)) != cudaSuccess) goto cuda_fail;
  }
  k_tp_prep_cols<<<dim3((unsigned)cdiv(nblp, TP_COLS), (unsigned)nch), 256, 0, st>>>(
      K, Kpad, nblp, s.n_mu, x0, M, om, xw, Mdf, wdf, mxW, eB, Bt, words + 3);
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  k_tp_make_y<<<dim3((unsigned)cdiv64(rowsY, TY_ROWS), (unsigned)(Kpad / TY_K)), 256, 0, st>>>(
      rowsY, K, Kpad, s.nbp, nblp, P2, Mdf, wdf, mxW, eY, Ysl, words + 4);
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  {
    CUtensorMap ta, tb;
    if (int r = make_slices_map(&ta, Ysl, rowsY, Kpad, OZ_BM)) return r;
    if (int r = make_slices_map(&tb, Bt, nblp, Kpad, OZ_BN)) return r;
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
    P.g = make_glayout(s.nbl, s.nbp);
    P.wait_cycles = wait_cycles;
    int64_t tiles = 0;
    for (int b = 0; b < s.nbl; ++b) tiles += cdiv64(P.g.rows(b), OZ_BM) * cdiv64(P.g.cols(b), OZ_BN);
    if ((e = cudaFuncSetAttribute(k_ozaki_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM)) !=
        cudaSuccess)
      goto cuda_fail;
    k_ozaki_gemm<1><<<(unsigned)tiles, OZ_THREADS, OZ_SMEM, st>>>(ta, tb, P);
    if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  }
  return MODAL_OK;
cuda_fail:
  snprintf(g_tc_err, sizeof g_tc_err, "triple product: %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

int *tc_error_word(void *scratch, const SepShape &, int) { return (int *)scratch; }

void tc_release(int) {}

}  // namespace modal
