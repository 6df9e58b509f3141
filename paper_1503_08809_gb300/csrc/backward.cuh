// backward.cuh -- adjoint of the separable path (row a9).
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace modal {
size_t backward_scratch_bytes(const SepShape &s, int nxc, int prec);
int run_backward(const SepShape &s, int nxc, int prec, const modal_problem *p, const double *gbar,
                 double *dqt, double *dq, void *scratch, int num_sms, cudaStream_t st);
const char *backward_last_error();
}  // namespace modal
