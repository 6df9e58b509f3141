// direct.cuh -- kernels of the direct path (k_direct.cu), driven from modal_abi.cu.
#pragma once
#include "common.cuh"

namespace modal {

// 1/2 x the Gosper form of h^2 (Section 2.1), divided by prod(2l+1)/(4 pi)
__device__ __forceinline__ double gosper_3j2(int l1, int l2, int l3) {
  double L = (double)(l1 + l2 + l3);
  double L1 = L - 2.0 * l1, L2 = L - 2.0 * l2, L3 = L - 2.0 * l3;
  double v = (2.0 / MODAL_PI) * (L + 1.0 / 3.0) /
             ((L + 1.0) * (L1 + 1.0 / 3.0) * (L2 + 1.0 / 3.0) * (L3 + 1.0 / 3.0));
  return v * sqrt((L1 + 1.0 / 6.0) * (L2 + 1.0 / 6.0) * (L3 + 1.0 / 6.0) / (L + 1.0 / 6.0));
}

// Weight of the sorted triple l1 <= l2 <= l3 (grid points i1, i2, i3) in
// Eq. 3D: z = mult * dw1 dw2 dw3 * w_l1 w_l2 w_l3 * H / (144 pi), H the exact
// 3j^2 from the ratio table ctab[n] = prod_{k<=n} (1 - 1/(2k)) (exact mode)
// or 1/2 x the Gosper form; mult = distinct orderings (6, 3 or 1).
__device__ __forceinline__ double direct_weight(int l1, int l2, int l3, int i1, int i2, int i3,
                                                const double *__restrict__ dw, const double *__restrict__ w_l,
                                                int l_min, const double *__restrict__ ctab, int mode) {
  double H;
  if (mode == MODAL_W_EXACT_3J) {
    const int g = (l1 + l2 + l3) / 2;
    H = ctab[g - l1] * ctab[g - l2] * ctab[g - l3] / ((2.0 * g + 1.0) * ctab[g]);
  } else {
    H = 0.5 * gosper_3j2(l1, l2, l3);
  }
  const int mult = (l1 == l2 && l2 == l3) ? 1 : ((l1 == l2 || l2 == l3) ? 3 : 6);
  const double d = (dw ? dw[i1] * dw[i2] * dw[i3] : 1.0) * w_l[l1 - l_min] * w_l[l2 - l_min] * w_l[l3 - l_min];
  return (double)mult * d * H / (144.0 * MODAL_PI);
}

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
