// tc.cuh -- tcgen05 (5th-generation tensor core) form of the separable path.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace modal {
size_t tc_scratch_bytes(const SepShape &s, int nxc);
// One radial chunk: M (FP32 scratch for the chunk) and G (+)= triple product.
int tc_separable_chunk(const SepShape &s, const double *A, const double *q, const double *qt,
                       const double *om, const double *xw, int x0, int nxc, float *M, double *G,
                       bool accumulate, void *scratch, int num_sms, cudaStream_t st);
const char *tc_last_error();
void tc_release(int device);
}  // namespace modal
