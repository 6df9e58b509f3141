// direct.cuh -- kernels of the direct path (k_direct.cu), driven from modal_abi.cu.
#pragma once
#include "common.cuh"

namespace modal {

__global__ void k_transpose(const double *__restrict__ in, int64_t rows, int64_t cols,
                            double *__restrict__ out);
__global__ void k_direct_count(int ng, const int *__restrict__ grid, int mode,
                               int64_t *__restrict__ counts);
__global__ void k_direct_total(const int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
                               int64_t npairs, int64_t *__restrict__ ntri);
__global__ void k_direct_fill_batch(int ng, const int *__restrict__ grid, const double *__restrict__ dw,
                                    const double *__restrict__ w_l, int l_min, const double *__restrict__ ctab,
                                    int mode, const int64_t *__restrict__ offsets, const int64_t *__restrict__ ntri,
                                    int64_t t0, int T, int *__restrict__ tri, double *__restrict__ z);
__global__ void k_direct_X(int nbp, int n_x, int l_min, const double *__restrict__ qtT,
                           const double *__restrict__ xw, const int *__restrict__ tri, int64_t t0, int T,
                           int xc, const int *__restrict__ prim, int n_prim, double *__restrict__ Xb,
                           const int64_t *__restrict__ ntri, int64_t tglob0);
__global__ void k_direct_Y(int nbl, int L, int l_min, const double *__restrict__ q,
                           const int *__restrict__ tri, const double *__restrict__ z, int64_t t0, int T,
                           const int64_t *__restrict__ ntri, int64_t tglob0, const int *__restrict__ late,
                           int n_late, double *__restrict__ Yb);

// CUB scan (exclusive prefix sum of int64) with caller scratch
cudaError_t scan_exclusive_i64(void *tmp, size_t tmp_bytes, const int64_t *in, int64_t *out,
                               int64_t n, cudaStream_t st);
size_t scan_tmp_bytes(int64_t n);

}  // namespace modal
