// kernels.cuh -- launcher declarations shared by the translation units.
#pragma once
#include "common.cuh"

namespace modal {

// k_basis.cu
cudaError_t launch_gl_nodes(int n, double *mu, double *om, cudaStream_t st);
cudaError_t launch_legendre_table(int n_mu, const double *mu, int l_min, int l_max,
                                  const double *w_l, double *A, cudaStream_t st);
cudaError_t launch_x_weights(int kind, int n, const double *x, double *w, cudaStream_t st);
cudaError_t launch_threej_table(int nmax, double *c, cudaStream_t st);

// k_simt.cu : CUDA-core contraction / triple product / symmetrise
struct SepShape {
  int l_min, l_max, L, nbl, nbp, n_x, n_mu;
};
// M chunk for x in [x0, x0+nxc): M[xl][j][a][p] (T = double or float)
template <typename T>
cudaError_t launch_contract_l(const SepShape &s, const double *A, const double *q, const double *qt,
                              int x0, int nxc, T *M, cudaStream_t st);
// G (+)= sum over the chunk's slices (see GLayout); Gpart = [ksplit][Gsize] scratch
int triple_launches(const SepShape &s, int nxc, int ksplit, bool accumulate);
template <typename T>
cudaError_t launch_triple(const SepShape &s, const T *M, const double *om, const double *xw, int x0,
                          int nxc, int ksplit, double *G, double *Gpart, bool accumulate,
                          int num_sms, cudaStream_t st, bool absM = false);
int triple_ksplit(const SepShape &s, int nxc, int num_sms);
// layout: the G layout the triple product filled (NULL: make_glayout's)
cudaError_t launch_gather(const SepShape &s, const double *G, const int *late, const int *prim,
                          int n_late, int n_prim, double scale, double *gamma, cudaStream_t st,
                          const GLayout *layout = nullptr);
cudaError_t launch_zero(double *p, size_t n, cudaStream_t st);

// generic K-major FP64 GEMM: C[m][n] (+)= sum_k A[m*lda + k] B[n*ldb + k]; with
// kdev, only the first min(k, *kdev - koff) terms (read on the device; none:
// C unchanged when accumulating, zero otherwise)
cudaError_t launch_gemm_nt_f64(int m, int n, int k, const double *A, int64_t lda, const double *B,
                               int64_t ldb, double *C, int64_t ldc, bool accumulate, cudaStream_t st,
                               const int64_t *kdev = nullptr, int64_t koff = 0);

}  // namespace modal
