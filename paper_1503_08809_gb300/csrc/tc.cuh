// tc.cuh -- tcgen05 (5th-generation tensor core) form of the separable path.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace modal {
size_t tc_scratch_bytes(const SepShape &s, int nxc);
size_t tc_triple_scratch_bytes(const SepShape &s, int nxc);
// l contraction of one radial chunk on the tensor cores: M (FP64) [xl][j][a][p].
int tc_contract_l(const SepShape &s, const double *A, const double *q, const double *qt, int x0, int nxc,
                  double *M, void *scratch, long long wait_cycles, cudaStream_t st, char **scratch_end,
                  bool reset_err);
// default bound of every device-side wait of the tensor-core kernels (SM clocks)
constexpr long long TC_DEFAULT_WAIT_CYCLES = 4000000000LL;
// One radial chunk: M (FP64 scratch for the chunk) and G (+)= triple product.
int tc_separable_chunk(const SepShape &s, const double *A, const double *q, const double *qt,
                       const double *om, const double *xw, int x0, int nxc, double *M, double *G,
                       bool accumulate, void *scratch, int num_sms, long long wait_cycles, cudaStream_t st);
// device error word of the tensor-core scratch (bit 0: a bounded wait gave up)
int *tc_error_word(void *scratch, const SepShape &s, int nxc);
const char *tc_last_error();
void tc_release(int device);
}  // namespace modal
