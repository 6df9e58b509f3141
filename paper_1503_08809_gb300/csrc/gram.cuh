// gram.cuh -- launchers of k_gram.cu: the Gram matrix's symmetrisation and
// the FP64 Cholesky solve behind the full Gamma (Appendix A).
#pragma once
#include "common.cuh"

namespace modal {

// G <- (G + G^T) / 2 for an [n][n] row-major matrix
cudaError_t launch_symmetrise(double *G, int n, cudaStream_t st);

// p[0 .. n) <- v
cudaError_t launch_fill(double *p, int64_t n, double v, cudaStream_t st);

// Scratch of gram_solve: the factor (n x n) and a status word.
size_t gram_solve_scratch_bytes(int n);

// Number of kernel launches of gram_solve (for the profiler).
int gram_solve_launches(int n, int m);

// X = G^{-1} R by G = L L^T (blocked Cholesky, FP64) and the solves
// L Y = R, L^T X = Y.  G: [n][n] row-major, only i >= j read.  R, X: [n][m]
// row-major; X may be R.  If a pivot is not positive (or not a number) the
// device word *info (int) becomes 1 + its index, the later steps do nothing
// and X is filled with NaN; otherwise *info = 0.  `info` may be the status
// word inside the scratch (gram_solve_info).
cudaError_t gram_solve(int n, int m, const double *G, const double *R, double *X, void *scratch,
                       int *info, cudaStream_t st);
int *gram_solve_info(void *scratch, int n);

}  // namespace modal
