// tc_f32acc.cu -- the l contraction of Eq. legendre on tcgen05 tensor cores
// with plain FP32 accumulation in TMEM, in the two comparison forms of the
// mixed-precision path:
//
//  * TF32 (MODAL_PREC_TF32): operands rounded to TF32 (cvt.rna), one
//    kind::tf32 product per 8-deep K step;
//  * BF16x3 (MODAL_PREC_BF16X3): each operand x written as hi = bf16(x) and
//    lo = bf16(x - hi), three kind::f16 products hi hi' + hi lo' + lo hi'
//    per 16-deep K step (the lo lo' term, ~2^-16 of the others, is dropped).
//
// Both accumulate the whole K = L sum in one FP32 TMEM accumulator (no exact
// chunking: these forms trade the Ozaki form's 1e-9 for fewer products) and
// write M in FP32 (for the FP32 triple product with compensated chunk sums)
// or FP64 (modal_contract_l).  Rows of A are (j, a): A[j][l] q_a(l); rows of
// B are (x, p): q~_p(l, x); M[x][j][a][p] = sum_l A B.
//
// Operands are K-major, staged by TMA into a four-stage mbarrier ring (128-byte
// swizzle for TF32, 64-byte for BF16); one thread issues the MMAs, four warps
// drain the 128 x 128 accumulator.  Every wait is bounded; on give-up the CTA
// raises the error word, waits for its copies in flight, frees TMEM and returns.
#include <cuda_bf16.h>

#include <cstdio>

#include "common.cuh"
#include "kernels.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace modal {

static thread_local char g_fa_err[256] = "";
const char *fa_last_error() { return g_fa_err; }

namespace {
constexpr int FA_BM = 128, FA_BN = 128;
constexpr int FA_BK = 32;                      // K elements per stage
constexpr int FA_STAGES = 4;
constexpr int FA_TILE_BYTES = 16384;           // one operand tile per stage, both kinds
constexpr int FA_STAGE_BYTES = 2 * FA_TILE_BYTES;
constexpr int FA_THREADS = 192;                // TMA warp, MMA warp, four drain warps
constexpr int FA_SMEM = FA_STAGES * FA_STAGE_BYTES + 1024 + 256;
constexpr int FA_ERR_TIMEOUT = 1, FA_ERR_RANGE = 2;
static_assert(FA_BM * FA_BK * 4 == FA_TILE_BYTES && 2 * FA_BM * FA_BK * 2 == FA_TILE_BYTES, "tile bytes");

// instruction descriptors: FP32 accumulator, K-major A and B
constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
}  // namespace

struct FaParams {
  int64_t rowsA, rowsB;
  int Kpad;
  int n_mu, nbl, nbp;
  void *out;
  int out_f64;
  int *err;
  long long wait_cycles;
};

// Operand rows in the form's layout: TF32 [rows][Kpad] FP32; BF16x3
// [2][rows][Kpad] BF16 (hi plane, then lo plane); zero for l >= L.
template <int KIND, bool IS_A>
__global__ void k_fa_split(int64_t rows, int L, int Kpad, const double *__restrict__ Atab,
                           const double *__restrict__ q, const double *__restrict__ qt, int nbl, int nbp, int x0,
                           void *__restrict__ out, int *__restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * Kpad) return;
  const int64_t r = i / Kpad;
  const int l = (int)(i % Kpad);
  double v = 0.0;
  if (l < L) {
    if (IS_A) {
      const int j = (int)(r / nbl), a = (int)(r % nbl);
      v = Atab[(int64_t)j * L + l] * q[(int64_t)a * L + l];
    } else {
      const int xl = (int)(r / nbp), p = (int)(r % nbp);
      v = qt[((int64_t)(x0 + xl) * nbp + p) * L + l];
    }
  }
  float f = __double2float_rn(v);
  if (!isfinite(f)) {
    atomicOr(err, FA_ERR_RANGE);
    f = 0.f;
  }
  if (KIND == TC_FORM_TF32) {
    reinterpret_cast<float *>(out)[i] = round_tf32(f);
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
    reinterpret_cast<__nv_bfloat16 *>(out)[i] = hi;
    reinterpret_cast<__nv_bfloat16 *>(out)[rows * Kpad + i] = lo;
  }
}

template <int KIND>
__global__ void __launch_bounds__(FA_THREADS, 1)
    k_fa_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, FaParams P) {
  extern __shared__ unsigned char smraw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(sm + FA_STAGES * FA_STAGE_BYTES);
  uint64_t *empty = full + FA_STAGES;
  uint64_t *acc_full = empty + FA_STAGES;
  uint64_t *mma_done = acc_full + 1;
  uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t a_row0 = (int64_t)blockIdx.y * FA_BM, b_row0 = (int64_t)blockIdx.x * FA_BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < FA_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(mma_done, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, FA_BN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksteps = P.Kpad / FA_BK;

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      ptx::prefetch_tmap(&tmB);
      int issued = 0;
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % FA_STAGES;
        const uint32_t ph = (uint32_t)((i / FA_STAGES) & 1);
        if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag, P.wait_cycles)) break;
        unsigned char *st = sm + s * FA_STAGE_BYTES;
        ptx::mbar_arrive_expect_tx(&full[s], FA_STAGE_BYTES);
        if (KIND == TC_FORM_TF32) {
          ptx::tma_load_2d(st, &tmA, &full[s], i * FA_BK, (int)a_row0);
          ptx::tma_load_2d(st + FA_TILE_BYTES, &tmB, &full[s], i * FA_BK, (int)b_row0);
        } else {
          ptx::tma_load_3d(st, &tmA, &full[s], i * FA_BK, (int)a_row0, 0);
          ptx::tma_load_3d(st + FA_TILE_BYTES, &tmB, &full[s], i * FA_BK, (int)b_row0, 0);
        }
        ++issued;
      }
      if (*abort_flag) {  // the copies in flight land before shared memory is released
        for (int i = (issued > FA_STAGES ? issued - FA_STAGES : 0); i < issued; ++i) {
          volatile int dummy = 0;
          ptx::mbar_wait(&full[i % FA_STAGES], (uint32_t)((i / FA_STAGES) & 1), &dummy, TC_DEFAULT_WAIT_CYCLES);
        }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0) {
      const uint32_t sbase = ptx::smem_u32(sm);
      for (int i = 0; i < ksteps; ++i) {
        const int s = i % FA_STAGES;
        const uint32_t ph = (uint32_t)((i / FA_STAGES) & 1);
        if (!ptx::mbar_wait(&full[s], ph, abort_flag, P.wait_cycles)) break;
        ptx::tc_fence_after();
        const uint32_t a0 = sbase + s * FA_STAGE_BYTES, b0 = a0 + FA_TILE_BYTES;
        if (KIND == TC_FORM_TF32) {
          // rows of 128 bytes (32 FP32), 8-row groups 1 KB apart; K = 8 per MMA
          constexpr uint32_t idesc = idesc_tf32(FA_BM, FA_BN);
          const uint64_t ad0 = ptx::smem_desc(a0, 16, 1024, ptx::SW_128B);
          const uint64_t bd0 = ptx::smem_desc(b0, 16, 1024, ptx::SW_128B);
#pragma unroll
          for (int kk = 0; kk < FA_BK / 8; ++kk)
            mma_tf32(tmem, ad0 + (uint64_t)((kk * 32) >> 4), bd0 + (uint64_t)((kk * 32) >> 4), idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        } else {
          // two planes (hi, lo) of 128 rows x 64 bytes; K = 16 per MMA
          constexpr uint32_t idesc = ptx::idesc_bf16_f32(FA_BM, FA_BN);
          constexpr uint32_t plane = FA_BM * 64;
          const uint64_t ad0 = ptx::smem_desc(a0, 16, 512, ptx::SW_64B);
          const uint64_t bd0 = ptx::smem_desc(b0, 16, 512, ptx::SW_64B);
#pragma unroll
          for (int kk = 0; kk < FA_BK / 16; ++kk) {
            const uint64_t k16 = (uint64_t)((kk * 32) >> 4);
            ptx::mma_bf16(tmem, ad0 + k16, bd0 + k16, idesc, (i > 0 || kk > 0) ? 1u : 0u);   // hi hi'
            ptx::mma_bf16(tmem, ad0 + k16, bd0 + k16 + (plane >> 4), idesc, 1u);              // hi lo'
            ptx::mma_bf16(tmem, ad0 + k16 + (plane >> 4), bd0 + k16, idesc, 1u);              // lo hi'
          }
        }
        ptx::mma_commit(&empty[s]);
      }
      ptx::mma_commit(acc_full);
      ptx::mma_commit(mma_done);
      volatile int dummy = 0;
      ptx::mbar_wait(mma_done, 0, &dummy, TC_DEFAULT_WAIT_CYCLES);
    }
  } else {
    // ================= drain: row (j, a) of this thread, 128 columns (x, p) =================
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const bool got = ptx::mbar_wait(acc_full, 0, abort_flag, P.wait_cycles);
    if (__all_sync(0xffffffffu, got) && !*abort_flag) {
      ptx::tc_fence_after();
      const int64_t rA = a_row0 + row;
      const int64_t mx = (int64_t)P.n_mu * P.nbl * P.nbp;
      const int64_t mrow = rA * P.nbp;  // (j nbl + a) nbp
      const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int cb = 0; cb < FA_BN / 16; ++cb) {
        float v[16];
        ptx::tmem_ld16(tl + (uint32_t)(cb * 16), v);
        ptx::tmem_ld_wait();
        if (rA < P.rowsA) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int64_t rB = b_row0 + cb * 16 + c;
            if (rB < P.rowsB) {
              const int64_t xl = rB / P.nbp, pp = rB % P.nbp;
              const int64_t idx = xl * mx + mrow + pp;
              if (P.out_f64) reinterpret_cast<double *>(P.out)[idx] = (double)v[c];
              else reinterpret_cast<float *>(P.out)[idx] = v[c];
            }
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.err, FA_ERR_TIMEOUT);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, FA_BN);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeFn fa_encode() {
  static const EncodeFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeFn)p;
    return (EncodeFn) nullptr;
  }();
  return fn;
}

// TF32: 2-D map over [rows][Kpad] FP32, box (32, 128), 128-byte swizzle.
// BF16x3: 3-D map over [2][rows][Kpad] BF16, box (32, 128, 2), 64-byte swizzle.
static int fa_make_map(int kind, CUtensorMap *m, const void *base, int64_t rows, int Kpad) {
  EncodeFn enc = fa_encode();
  if (!enc) {
    snprintf(g_fa_err, sizeof g_fa_err, "cuTensorMapEncodeTiled unavailable");
    return MODAL_EUNSUPPORTED;
  }
  CUresult r;
  if (kind == TC_FORM_TF32) {
    cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kpad * 4};
    cuuint32_t box[2] = {(cuuint32_t)FA_BK, (cuuint32_t)FA_BM};
    cuuint32_t es[2] = {1, 1};
    r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, 2};
    cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)rows * Kpad * 2};
    cuuint32_t box[3] = {(cuuint32_t)FA_BK, (cuuint32_t)FA_BM, 2};
    cuuint32_t es[3] = {1, 1, 1};
    r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) {
    snprintf(g_fa_err, sizeof g_fa_err, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MODAL_EINVAL;
  }
  return MODAL_OK;
}

static size_t fa_up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch: [status words 256 B][A operand][B operand of nxc_max radial points]
struct FaScratch {
  int *words;
  void *A, *B;
  char *end;
};
static FaScratch fa_scratch(void *base, const SepShape &s, int nxc_max) {
  const int Kpad = cdiv(s.L, FA_BK) * FA_BK;
  const size_t per = 4;  // bytes per element: one FP32, or two BF16 planes
  FaScratch r;
  char *w = (char *)base;
  r.words = (int *)w; w += 256;
  r.A = w; w += fa_up256(per * (size_t)s.n_mu * s.nbl * Kpad);
  r.B = w; w += fa_up256(per * (size_t)nxc_max * s.nbp * Kpad);
  r.end = w;
  return r;
}

size_t fa_scratch_bytes(const SepShape &s, int nxc_max) {
  FaScratch r = fa_scratch(nullptr, s, nxc_max);
  return (size_t)(r.end - (char *)nullptr) + 256;
}

int *fa_error_word(void *scratch) { return (int *)scratch; }

int fa_prepare_l(int kind, const SepShape &s, const double *A, const double *q, void *scratch, int nxc_max,
                 cudaStream_t st, Profiler *prof, bool reset_status) {
  FaScratch r = fa_scratch(scratch, s, nxc_max);
  const int Kpad = cdiv(s.L, FA_BK) * FA_BK;
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl;
  cudaError_t e;
  {
    ProfScope ps(prof, "fa_split_lA", st);
    if (reset_status && (e = cudaMemsetAsync(r.words, 0, 256, st)) != cudaSuccess) goto fail;
    const unsigned blocks = (unsigned)cdiv64(rowsA * Kpad, 256);
    if (kind == TC_FORM_TF32)
      k_fa_split<TC_FORM_TF32, true><<<blocks, 256, 0, st>>>(rowsA, s.L, Kpad, A, q, nullptr, s.nbl, s.nbp, 0,
                                                             r.A, r.words);
    else
      k_fa_split<TC_FORM_BF16X3, true><<<blocks, 256, 0, st>>>(rowsA, s.L, Kpad, A, q, nullptr, s.nbl, s.nbp, 0,
                                                               r.A, r.words);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  }
  return MODAL_OK;
fail:
  snprintf(g_fa_err, sizeof g_fa_err, "l-contraction operand split: %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

int fa_contract_l(int kind, const SepShape &s, const double *qt, int x0, int nxc, int nxc_max, void *M,
                  bool out_f64, void *scratch, long long wait_cycles, cudaStream_t st, Profiler *prof) {
  FaScratch r = fa_scratch(scratch, s, nxc_max);
  const int Kpad = cdiv(s.L, FA_BK) * FA_BK;
  const int64_t rowsA = (int64_t)s.n_mu * s.nbl, rowsB = (int64_t)nxc * s.nbp;
  cudaError_t e;
  {
    ProfScope ps(prof, "fa_split_lB", st);
    const unsigned blocks = (unsigned)cdiv64(rowsB * Kpad, 256);
    if (kind == TC_FORM_TF32)
      k_fa_split<TC_FORM_TF32, false><<<blocks, 256, 0, st>>>(rowsB, s.L, Kpad, nullptr, nullptr, qt, s.nbl, s.nbp,
                                                              x0, r.B, r.words);
    else
      k_fa_split<TC_FORM_BF16X3, false><<<blocks, 256, 0, st>>>(rowsB, s.L, Kpad, nullptr, nullptr, qt, s.nbl,
                                                                s.nbp, x0, r.B, r.words);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  }
  {
    CUtensorMap ta, tb;
    if (int rr = fa_make_map(kind, &ta, r.A, rowsA, Kpad)) return rr;
    if (int rr = fa_make_map(kind, &tb, r.B, rowsB, Kpad)) return rr;
    FaParams P{};
    P.rowsA = rowsA;
    P.rowsB = rowsB;
    P.Kpad = Kpad;
    P.n_mu = s.n_mu;
    P.nbl = s.nbl;
    P.nbp = s.nbp;
    P.out = M;
    P.out_f64 = out_f64 ? 1 : 0;
    P.err = r.words;
    P.wait_cycles = wait_cycles;
    auto kern = kind == TC_FORM_TF32 ? k_fa_gemm<TC_FORM_TF32> : k_fa_gemm<TC_FORM_BF16X3>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, FA_SMEM)) != cudaSuccess)
      goto fail;
    dim3 grid((unsigned)cdiv64(rowsB, FA_BN), (unsigned)cdiv64(rowsA, FA_BM));
    ProfScope ps(prof, kind == TC_FORM_TF32 ? "fa_gemm_l_tf32" : "fa_gemm_l_bf16x3", st);
    kern<<<grid, FA_THREADS, FA_SMEM, st>>>(ta, tb, P);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  }
  return MODAL_OK;
fail:
  snprintf(g_fa_err, sizeof g_fa_err, "l contraction (FP32 accumulation): %s", cudaGetErrorString(e));
  return MODAL_ECUDA;
}

}  // namespace modal
