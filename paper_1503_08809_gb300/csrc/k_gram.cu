// k_gram.cu -- the late basis's Gram matrix and the full Gamma (Appendix A:
// Gamma_nm = sum_r <Q_n, Q_r>^{-1} <Q_r, Q~_m>).
//
// The Gram matrix comes out of the separable kernels (the projection with
// q~ -> q); this file holds what is new: its symmetrisation, a blocked
// Cholesky factorisation G = L L^T in FP64 and the two triangular solves
// L Y = Gamma', L^T Gamma = Y.  All steps are stream-ordered launches with no
// host synchronisation.  A pivot that is not above n 2^-52 times the
// matrix's own diagonal entry (G not positive definite, or numerically
// singular as with a mode listed twice, whose pivot is rounding noise of
// ~1e-16 relative; a regular Gram matrix's smallest is ~1e-2) or that is not
// a number is recorded in a device word as 1 + its index (the first failure
// wins); every later kernel reads the word and does nothing, and the last one
// fills the result with NaN.
//
// Sizes are small next to the projection (n_late <= a few thousand), so the
// kernels are plain CUDA-core FP64 tiles: the factorisation's trailing
// update and the solves' updates are one strided tiled kernel (64 x 64 output
// tiles, 4 x 4 per thread); each diagonal block (64 x 64) is factored and
// inverted in shared memory, and the panel and the solves apply the inverse.
#include <cmath>
#include <mutex>

#include "gram.cuh"

namespace modal {

constexpr int GB = 64;  // block size of the factorisation and the solves
// dynamic shared memory of the diagonal-block kernels: two GB x GB blocks
// with rows padded to GB + 1 (distinct banks for threads on distinct rows)
constexpr int DIAG_SMEM = 2 * GB * (GB + 1) * (int)sizeof(double);

__global__ void k_symmetrise(double *G, int n) {
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  if (i >= n || j >= i) return;  // each pair (i > j) by one thread
  const double v = 0.5 * (G[(int64_t)i * n + j] + G[(int64_t)j * n + i]);
  G[(int64_t)i * n + j] = v;
  G[(int64_t)j * n + i] = v;
}

cudaError_t launch_symmetrise(double *G, int n, cudaStream_t st) {
  if (n < 2) return cudaSuccess;
  k_symmetrise<<<dim3(cdiv(n, 16), cdiv(n, 16)), dim3(16, 16), 0, st>>>(G, n);
  return cudaGetLastError();
}

__global__ void k_fill(double *p, int64_t n, double v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cudaError_t launch_fill(double *p, int64_t n, double v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

// Cholesky of the diagonal block at (k0, k0) of size nb <= GB, in place
// (lower triangle), right-looking inside shared memory, followed by the
// inverse of that factor, V = L_kk^{-1} (lower), written to Dinv (GB x GB,
// zero outside the nb x nb lower triangle): the panel and both solves then
// apply V as small parallel products instead of running a 64-step
// dependent substitution per row or column (FP64 latency dominates those on
// this part).  G: the input matrix (its diagonal scales the pivot test), n:
// its order.
__global__ void __launch_bounds__(256) k_potrf_inv_diag(double *L, const double *G, int64_t ld, int n, int k0,
                                                        int nb, double *Dinv, int *info) {
  extern __shared__ double diag_sm[];
  double(*s)[GB + 1] = reinterpret_cast<double(*)[GB + 1]>(diag_sm);
  double(*v)[GB + 1] = reinterpret_cast<double(*)[GB + 1]>(diag_sm + GB * (GB + 1));
  __shared__ double gdiag[GB];  // the input's diagonal (scale of the pivot test)
  __shared__ double rdiag[GB];  // 1 / pivot
  __shared__ double piv_s;      // the current pivot
  __shared__ int bad;
  if (*info) return;  // an earlier block failed
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    s[r][c] = c <= r ? L[(int64_t)(k0 + r) * ld + k0 + c] : 0.0;
  }
  if (tid < nb) gdiag[tid] = G[(int64_t)(k0 + tid) * ld + k0 + tid];
  __syncthreads();
  const double tol = (double)n * 0x1p-52;
  // Thread 0 alone takes the square root and the reciprocal of each pivot
  // (FP64 sequences that cost the whole warp's issue slots on this part), as
  // soon as the pivot is final: step j's trailing update gives it the
  // diagonal entry j + 1 first.  The others read the result after a barrier.
  auto pivot = [&](int j) {
    const double d = s[j][j], g = gdiag[j];
    if (g > 0.0 && d > tol * g) {  // false also for NaN
      const double p = sqrt(d);
      piv_s = p;
      rdiag[j] = 1.0 / p;
    } else {
      bad = j + 1;
    }
  };
  if (tid == 0) {
    bad = 0;
    pivot(0);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (bad) break;  // the same value for every thread
    const double r = rdiag[j], p = piv_s;
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) s[i][j] *= r;
    __syncthreads();  // column j scaled; every thread has read the pivot
    if (tid == 0) s[j][j] = p;
    for (int i = j + 1 + (tid >> 4); i < nb; i += 16) {
      for (int l = j + 1 + (tid & 15); l <= i; l += 16) s[i][l] -= s[i][j] * s[l][j];
      if (tid == 0 && i == j + 1) pivot(j + 1);  // entry (j+1, j+1) is final now
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicCAS(info, 0, k0 + bad);
    return;
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    if (c <= r) L[(int64_t)(k0 + r) * ld + k0 + c] = s[r][c];
  }
  // V[i][c] = (delta_ic - sum_{c <= l < i} L[i][l] V[l][c]) / L[i][i], row by
  // row; four lanes of one warp share a column and split the sum
  const int c = tid >> 2, q = tid & 3;
  for (int i = 0; i < GB; ++i) {  // every lane runs every step (shuffles)
    double part = 0.0;
    if (c < nb && i < nb)
      for (int l = c + q; l < i; l += 4) part += s[i][l] * v[l][c];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    if (q == 0 && c < nb && i < nb) v[i][c] = i < c ? 0.0 : ((i == c ? 1.0 : 0.0) - part) * rdiag[i];
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < GB * GB; e += blockDim.x) {
    const int r = e / GB, cc = e % GB;
    Dinv[e] = (r < nb && cc <= r) ? v[r][cc] : 0.0;
  }
}

// Panel below the diagonal block: L21 = A21 L11^{-T} = A21 V^T, GB rows per
// CTA (each row's entries from its own copy in shared memory, so the result
// overwrites A21 in place).
__global__ void __launch_bounds__(256) k_panel_apply(double *L, int64_t ld, int k0, int nb, int n,
                                                    const double *__restrict__ Dinv, const int *info) {
  extern __shared__ double diag_sm[];
  double(*A)[GB + 1] = reinterpret_cast<double(*)[GB + 1]>(diag_sm);
  double(*V)[GB + 1] = reinterpret_cast<double(*)[GB + 1]>(diag_sm + GB * (GB + 1));
  if (*info) return;
  const int tid = threadIdx.x;
  const int row0 = k0 + nb + blockIdx.x * GB;
  const int rows = min(GB, n - row0);
  for (int e = tid; e < GB * GB; e += blockDim.x) {
    const int r = e / GB, c = e % GB;
    A[r][c] = (r < rows && c < nb) ? L[(int64_t)(row0 + r) * ld + k0 + c] : 0.0;
    V[r][c] = Dinv[e];
  }
  __syncthreads();
  const int r = tid >> 2, jq = tid & 3;
  if (r >= rows) return;
#pragma unroll 4
  for (int t = 0; t < GB / 4; ++t) {
    const int j = jq + 4 * t;
    if (j >= nb) break;
    double acc = 0.0;
    for (int l = 0; l <= j; ++l) acc += A[r][l] * V[j][l];
    L[(int64_t)(row0 + r) * ld + k0 + j] = acc;
  }
}

// C[i][j] -= sum_k A(i, k) B(k, j) with A(i, k) = A[i a_si + k a_sk] and
// B(k, j) = B[k b_sk + j b_sj]; 64 x 64 tiles of C, 4 x 4 per thread.  With
// `lower` the grid runs over the tiles (ti >= tj) of a square C only.
__global__ void __launch_bounds__(256) k_gemm_sub(int m, int n, int K, const double *__restrict__ A,
                                                  int64_t a_si, int64_t a_sk, const double *__restrict__ B,
                                                  int64_t b_sk, int64_t b_sj, double *C, int64_t ldc,
                                                  int lower, const int *info) {
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, TX = BN / TN, TY = BM / TM;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  if (*info) return;
  int ti, tj;
  if (lower) {
    const int t = blockIdx.x;
    ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    tj = t - ti * (ti + 1) / 2;
  } else {
    ti = blockIdx.x;
    tj = blockIdx.y;
  }
  const int m0 = ti * BM, n0 = tj * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int kk = e % BK, r = e / BK;
      As[kk][r] = (m0 + r < m && k0 + kk < K) ? A[(int64_t)(m0 + r) * a_si + (int64_t)(k0 + kk) * a_sk] : 0.0;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      const int c = e % BN, kk = e / BN;
      Bs[kk][c] = (n0 + c < n && k0 + kk < K) ? B[(int64_t)(k0 + kk) * b_sk + (int64_t)(n0 + c) * b_sj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * TY];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + ty + i * TY;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + tx + j * TX;
      if (c < n) C[(int64_t)r * ldc + c] -= acc[i][j];
    }
  }
}

// The diagonal block's inverse applied to rows k0 .. k0 + nb of X, on all m
// right-hand columns, in place: forward (Y_k = V X_k, from L_kk Y_k = X_k)
// or backward (X_k = V^T Y_k, from L_kk^T X_k = Y_k).  GB columns per CTA;
// a thread computes one row of 16 interleaved columns.
template <bool BACKWARD>
__global__ void __launch_bounds__(256) k_tri_apply(const double *__restrict__ Dinv, double *X, int m, int k0,
                                                  int nb, const int *info) {
  extern __shared__ double diag_sm[];
  double(*Xs)[GB + 1] = reinterpret_cast<double(*)[GB + 1]>(diag_sm);
  double(*V)[GB + 1] = reinterpret_cast<double(*)[GB + 1]>(diag_sm + GB * (GB + 1));
  if (*info) return;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * GB;
  const int cols = min(GB, m - c0);
  for (int e = tid; e < GB * GB; e += blockDim.x) {
    const int r = e / GB, c = e % GB;
    Xs[r][c] = (r < nb && c < cols) ? X[(int64_t)(k0 + r) * m + c0 + c] : 0.0;
    V[r][c] = Dinv[e];
  }
  __syncthreads();
  const int i = tid >> 2, cq = tid & 3;
  if (i >= nb) return;
#pragma unroll 4
  for (int t = 0; t < GB / 4; ++t) {
    const int c = cq + 4 * t;
    if (c >= cols) break;
    double acc = 0.0;
    if (!BACKWARD)
      for (int l = 0; l <= i; ++l) acc += V[i][l] * Xs[l][c];
    else
      for (int l = i; l < nb; ++l) acc += V[l][i] * Xs[l][c];
    X[(int64_t)(k0 + i) * m + c0 + c] = acc;
  }
}

__global__ void k_nan_if_failed(double *X, int64_t n, const int *info) {
  if (!*info) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) X[i] = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
}

__global__ void k_copy_word(const int *src, int *dst) { *dst = *src; }

static size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// scratch: the factor L (n x n), the inverses of its diagonal blocks
// (GB x GB each), the status word
static size_t dinv_offset(int n) { return up256((size_t)n * n * sizeof(double)); }
static size_t info_offset(int n) { return dinv_offset(n) + up256((size_t)cdiv(n, GB) * GB * GB * sizeof(double)); }

size_t gram_solve_scratch_bytes(int n) { return info_offset(n) + 256; }

int *gram_solve_info(void *scratch, int n) { return (int *)((char *)scratch + info_offset(n)); }

int gram_solve_launches(int n, int m) {
  if (n == 0) return 0;
  const int nblk = cdiv(n, GB);
  int k = nblk + 2 * (nblk - 1);              // factor: diagonal block, panel, trailing update
  if (m > 0) k += 2 * (2 * nblk - 1) + 1;     // both solves, NaN fill
  return k + 1;                               // status copy
}

static cudaError_t diag_attributes() {
  static cudaError_t err = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    err = cudaFuncSetAttribute(k_potrf_inv_diag, a, DIAG_SMEM);
    if (err == cudaSuccess) err = cudaFuncSetAttribute(k_panel_apply, a, DIAG_SMEM);
    if (err == cudaSuccess) err = cudaFuncSetAttribute(k_tri_apply<false>, a, DIAG_SMEM);
    if (err == cudaSuccess) err = cudaFuncSetAttribute(k_tri_apply<true>, a, DIAG_SMEM);
  });
  return err;
}

cudaError_t gram_solve(int n, int m, const double *G, const double *R, double *X, void *scratch, int *info,
                       cudaStream_t st) {
  double *L = (double *)scratch;
  double *Dinv = (double *)((char *)scratch + dinv_offset(n));
  int *word = gram_solve_info(scratch, n);
  cudaError_t e;
  if ((e = diag_attributes()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(word, 0, sizeof(int), st)) != cudaSuccess) return e;
  if (n == 0) return info && info != word ? cudaMemsetAsync(info, 0, sizeof(int), st) : cudaSuccess;
  if ((e = cudaMemcpyAsync(L, G, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if (m > 0 && X != R &&
      (e = cudaMemcpyAsync(X, R, (size_t)n * m * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  // factorisation, one block column at a time
  for (int k0 = 0; k0 < n; k0 += GB) {
    const int nb = min(GB, n - k0);
    double *Vk = Dinv + (int64_t)(k0 / GB) * GB * GB;
    k_potrf_inv_diag<<<1, 256, DIAG_SMEM, st>>>(L, G, n, n, k0, nb, Vk, word);
    const int rest = n - k0 - nb;
    if (rest > 0) {
      k_panel_apply<<<cdiv(rest, GB), 256, DIAG_SMEM, st>>>(L, n, k0, nb, n, Vk, word);
      const int T = cdiv(rest, 64);
      const double *P = L + (int64_t)(k0 + nb) * n + k0;  // L21 [rest][nb]
      k_gemm_sub<<<T * (T + 1) / 2, 256, 0, st>>>(rest, rest, nb, P, n, 1, P, 1, n,
                                                 L + (int64_t)(k0 + nb) * n + k0 + nb, n, 1, word);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (m > 0) {
    // L Y = R (in X), top block down
    for (int k0 = 0; k0 < n; k0 += GB) {
      const int nb = min(GB, n - k0);
      k_tri_apply<false><<<cdiv(m, GB), 256, DIAG_SMEM, st>>>(Dinv + (int64_t)(k0 / GB) * GB * GB, X, m, k0,
                                                               nb, word);
      const int rest = n - k0 - nb;
      if (rest > 0)
        k_gemm_sub<<<dim3(cdiv(rest, 64), cdiv(m, 64)), 256, 0, st>>>(
            rest, m, nb, L + (int64_t)(k0 + nb) * n + k0, n, 1, X + (int64_t)k0 * m, m, 1,
            X + (int64_t)(k0 + nb) * m, m, 0, word);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // L^T X = Y, bottom block up
    for (int k0 = (n - 1) / GB * GB; k0 >= 0; k0 -= GB) {
      const int nb = min(GB, n - k0);
      k_tri_apply<true><<<cdiv(m, GB), 256, DIAG_SMEM, st>>>(Dinv + (int64_t)(k0 / GB) * GB * GB, X, m, k0,
                                                              nb, word);
      if (k0 > 0)  // rows above: X_top -= (L block row k)^T X_k
        k_gemm_sub<<<dim3(cdiv(k0, 64), cdiv(m, 64)), 256, 0, st>>>(
            k0, m, nb, L + (int64_t)k0 * n, 1, n, X + (int64_t)k0 * m, m, 1, X, m, 0, word);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t total = (int64_t)n * m;
    k_nan_if_failed<<<(unsigned)cdiv64(total, 256), 256, 0, st>>>(X, total, word);
  }
  if (info && info != word) k_copy_word<<<1, 1, 0, st>>>(word, info);
  return cudaGetLastError();
}

}  // namespace modal
