// tc.cuh -- tcgen05 (5th-generation tensor core) form of the separable path.
#pragma once
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace modal {
// triple-product variants: the Y operand through HBM, or formed in shared memory
constexpr int TC_TRIPLE_MATERIALISED = 0;
constexpr int TC_TRIPLE_FUSED = 1;
constexpr int TC_TRIPLE_FUSED2 = 2;
constexpr int TC_TRIPLE_PAIR = 3;   // Y through HBM, GEMM on CTA pairs (2-SM MMA)
constexpr int TC_TRIPLE_QUEUE = 4;  // Y through HBM, persistent GEMM over a work queue
// whether the second fused form can serve a basis (its M~ tile per stage)
bool tc_fused2_fits(int nbl, int nbp);
// scratch for l-contraction chunks of nxl radial points and triple-product
// chunks of nxc points (nxc <= nxl)
size_t tc_scratch_bytes(const SepShape &s, int nxl, int nxc, int variant);
size_t tc_triple_scratch_bytes(const SepShape &s, int nxc, int variant);
// default bound of every device-side wait of the tensor-core kernels (SM clocks)
constexpr long long TC_DEFAULT_WAIT_CYCLES = 4000000000LL;
// Split the x-independent A operand of the l contraction (once per call).
int tc_prepare_l(const SepShape &s, const double *A, const double *q, void *scratch, int nxc_max, cudaStream_t st,
                 Profiler *prof = nullptr, bool reset_status = true);
// l contraction of one radial chunk on the tensor cores: M (FP64) [xl][j][a][p].
int tc_contract_l(const SepShape &s, const double *qt, int x0, int nxc, int nxc_max, double *M, void *scratch,
                  long long wait_cycles, cudaStream_t st, Profiler *prof = nullptr);
// Triple product of one radial chunk [x0, x0 + nxc) whose M (FP64,
// [xl][j][a][p]) starts at M: G (+)= sum over its slices.
// Tile shape of the queue form (TC_TRIPLE_QUEUE): column tiles of at most
// wmax and K ranges split to give every SM two items (split) or not.
// tune = 0: wmax 128, split; else bits 0-3 = wmax / 16, bit 4 = no split.
inline int tune_wmax(int tune) { return tune ? 16 * (tune & 15) : 128; }
inline bool tune_split(int tune) { return !(tune & 16); }
int tc_triple_chunk(const SepShape &s, const double *M, const double *om, const double *xw, int x0, int nxc,
                    int nxl_max, double *G, bool accumulate, void *scratch, long long wait_cycles, int num_sms,
                    int variant, int split_k, cudaStream_t st, Profiler *prof = nullptr, bool absM = false,
                    int tune = 0);
// The triple product of one radial chunk in two phases (operands incl. the Y
// slices; the persistent queue GEMM on at most grid_sms SMs) with two
// alternating scratch sets, so that the phases of neighbouring chunks can
// run on two streams at once.  Scratch: tc_ovl_scratch_bytes.
size_t tc_ovl_scratch_bytes(const SepShape &s, int nxl, int nxc);
// part 0: operands and the Y rows of the first-form G blocks (GLayout),
// part 1: the Y rows of the others, part < 0: all
int tc_triple_prep(const SepShape &s, const double *M, const double *om, const double *xw, int x0, int nxc,
                   int nxl_max, int nxc_max, void *scratch, int set, int part, cudaStream_t st,
                   Profiler *prof = nullptr);
// single: one CTA per tile or K range of a tile (K splits by the modelled
// makespan on grid_sms SMs); otherwise the persistent queue on grid_sms SMs
// part (single form only): the tiles of the first-form blocks (0), of the
// others (1), or all (< 0)
int tc_triple_gemm(const SepShape &s, int nxc, int nxl_max, int nxc_max, double *G, bool accumulate,
                   void *scratch, int set, long long wait_cycles, int grid_sms, int tune, bool single,
                   int split_k, int part, cudaStream_t st, Profiler *prof = nullptr);
// The adjoint of the separable form on the tensor cores (exact slicing):
// dL/dM by one GEMM over the Y rows per radial chunk, then dL/dq~ and dL/dq
// by two more; nxc radial points per chunk (tc_backward_nxc: by memory and
// the dL/dM GEMM's CTA waves on num_sms SMs).  The status
// word is tc_error_word(scratch).
size_t tc_backward_scratch_bytes(const SepShape &s, int nxc);
int tc_backward_nxc(const SepShape &s, int num_sms);
int tc_backward(const SepShape &s, int nxc, const modal_problem *p, const double *gbar, double *dqt, double *dq,
                void *scratch, long long wait_cycles, cudaStream_t st, Profiler *prof = nullptr);
// C[m][n] += A B^T over one batch of T terms of the direct form (only the
// t < *count - t0 valid ones; a batch past the end does no work), on the
// exact-slicing GEMM.  Status word: tc_error_word(scratch).
size_t tc_gemm_batch_scratch_bytes(int m, int n, int T);
int tc_gemm_batch(int m, int n, int T, const double *A, const double *B, const int64_t *count, int64_t t0, double *C,
                  int64_t ldc, void *scratch, bool reset_status, long long wait_cycles, cudaStream_t st,
                  Profiler *prof = nullptr);
// The direct form (Eq. 3D) with its radial integrals and its Gamma' update on
// the tensor cores (exact-slicing GEMMs; pairs (l2, l3) grouped, see tc.cu):
// gamma overwritten; status word tc_error_word(scratch).  Bases of at most 32
// functions on either side (tc_direct_supported).
bool tc_direct_supported(int nb_late, int nb_prim);
size_t tc_direct_scratch_bytes(const modal_problem *p, int ng);
int tc_project_direct(const modal_problem *p, const int *grid, const double *dw, int ng, int mode, double *gamma,
                      void *scratch, int num_sms, long long wait_cycles, cudaStream_t st, Profiler *prof = nullptr);
// Layout of G that the triple product of a variant fills (the gather reads it)
GLayout tc_triple_glayout(const SepShape &s, int variant);
// status words of a triple-product scratch driven without this form's l
// contraction (mode 1: call start, 0: per chunk), and the OR of its error
// bits into another status word
cudaError_t tc_init_words(void *scratch, const SepShape &s, int nxl_max, int mode, cudaStream_t st);
cudaError_t tc_or_status(int *dst, void *scratch, cudaStream_t st);
// device status word of the tensor-core scratch (bit 0: a bounded wait gave up,
// bit 1: a value outside the FP32 exponent range of the split operands)
int *tc_error_word(void *scratch);
const char *tc_last_error();
void tc_release(int device);

// The l contraction with plain FP32 accumulation (tc_f32acc.cu): TF32
// operands (one kind::tf32 product) or BF16 hi/lo pairs (three products).
constexpr int TC_FORM_TF32 = 0;
constexpr int TC_FORM_BF16X3 = 1;
size_t fa_scratch_bytes(const SepShape &s, int nxc_max);
int fa_prepare_l(int kind, const SepShape &s, const double *A, const double *q, void *scratch, int nxc_max,
                 cudaStream_t st, Profiler *prof = nullptr, bool reset_status = true);
// M [xl][j][a][p] of radial points [x0, x0 + nxc), FP32 or FP64
int fa_contract_l(int kind, const SepShape &s, const double *qt, int x0, int nxc, int nxc_max, void *M,
                  bool out_f64, void *scratch, long long wait_cycles, cudaStream_t st, Profiler *prof = nullptr);
int *fa_error_word(void *scratch);
const char *fa_last_error();
}  // namespace modal
