// k_simt.cu -- CUDA-core (FP64 / FP32) forms of rows a5-a7 of the separable
// path: the l contraction (Eq. legendre), the triple product with the
// slice reduction (Eq. 2D), and the symmetrise/gather into Gamma'.
// Register-tiled SIMT GEMM loops with shared-memory staging; the FP32 form
// sums short chunks in FP32 and accumulates the chunk sums in FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace modal {

template <typename T>
struct SimtCfg;
template <>
struct SimtCfg<double> {  // 64x64 tile, 4x4 per thread
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct SimtCfg<float> {  // 128x64 tile, 8x4 per thread (FP64 chunk accumulators too)
  static constexpr int BM = 128, BN = 64, BK = 16, TM = 8, TN = 4;
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void simt_fma_tile(const T (*As)[BM + 1], const T (*Bs)[BN + 1],
                                              T (&acc)[TM][TN], int tx, int ty) {
  constexpr int TX = BN / TN, TY = BM / TM;
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    T a[TM], b[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * TY];
#pragma unroll
    for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// Running sum of the FP32 chunk sums: a double-FP32 (hi, lo) pair updated
// with Knuth's TwoSum -- FP32 operations only (GB300's FP64 rate is 1/64 of
// its FP32 rate), ~48 significant bits.  For FP64 tiles it is unused.
template <typename T, int TM, int TN>
struct ChunkAcc;
template <int TM, int TN>
struct ChunkAcc<float, TM, TN> {
  float hi[TM][TN], lo[TM][TN];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) { hi[i][j] = 0.f; lo[i][j] = 0.f; }
  }
  __device__ __forceinline__ void promote(float (&acc)[TM][TN]) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        float a = hi[i][j], b = acc[i][j];
        float s = a + b, bb = s - a;
        float e = (a - (s - bb)) + (b - bb);
        e += lo[i][j];
        hi[i][j] = s + e;
        lo[i][j] = e - (hi[i][j] - s);
        acc[i][j] = 0.f;
      }
  }
  __device__ __forceinline__ double value(const float (&acc)[TM][TN], int i, int j) const {
    return (double)hi[i][j] + (double)lo[i][j] + (double)acc[i][j];
  }
};
template <int TM, int TN>
struct ChunkAcc<double, TM, TN> {
  __device__ __forceinline__ void zero() {}
  __device__ __forceinline__ void promote(double (&)[TM][TN]) {}
  __device__ __forceinline__ double value(const double (&acc)[TM][TN], int i, int j) const { return acc[i][j]; }
};

// FP32 chunk length (in K steps of BK) before promotion into the running sum.
constexpr int PROMOTE_STEPS = 2;

// ---------------------------------------------------------------------------
// a5 (CUDA cores): M[xl][j][a][p] = sum_l A[j][l] q_a(l) q~_p(l, x0 + xl).
// GEMM rows (j, a), columns (xl, p), K = l; the A operand A[j][l] q_a(l) is
// formed while staging (the product table q_a q~_p over l is never materialised).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_contract_l(SepShape s, const double *__restrict__ A,
                                                    const double *__restrict__ q,
                                                    const double *__restrict__ qt, int x0, int nxc,
                                                    T *__restrict__ M) {
  using C = SimtCfg<T>;
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN;
  constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int L = s.L, nbl = s.nbl, nbp = s.nbp;
  const int64_t rows = (int64_t)s.n_mu * nbl, cols = (int64_t)nxc * nbp;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  T acc[TM][TN];
  ChunkAcc<T, TM, TN> run;
  run.zero();
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0;

  int step = 0;
  for (int k0 = 0; k0 < L; k0 += BK, ++step) {
    for (int e = tid; e < BM * BK; e += NT) {
      int kk = e % BK, r = e / BK;
      int64_t m = m0 + r;
      int l = k0 + kk;
      double v = 0.0;
      if (m < rows && l < L) {
        int j = (int)(m / nbl), a = (int)(m % nbl);
        v = A[(size_t)j * L + l] * q[(size_t)a * L + l];
      }
      As[kk][r] = (T)v;
    }
    for (int e = tid; e < BN * BK; e += NT) {
      int kk = e % BK, c = e / BK;
      int64_t n = n0 + c;
      int l = k0 + kk;
      double v = 0.0;
      if (n < cols && l < L) {
        int xl = (int)(n / nbp), p = (int)(n % nbp);
        v = qt[((size_t)(x0 + xl) * nbp + p) * L + l];
      }
      Bs[kk][c] = (T)v;
    }
    __syncthreads();
    simt_fma_tile<T, BM, BN, BK, TM, TN>(As, Bs, acc, tx, ty);
    __syncthreads();
    if ((step + 1) % PROMOTE_STEPS == 0) run.promote(acc);
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty + i * TY;
    if (m >= rows) continue;
    int j = (int)(m / nbl), a = (int)(m % nbl);
#pragma unroll
    for (int jj = 0; jj < TN; ++jj) {
      int64_t n = n0 + tx + jj * TX;
      if (n >= cols) continue;
      int xl = (int)(n / nbp), p = (int)(n % nbp);
      M[(((size_t)xl * s.n_mu + j) * nbl + a) * nbp + p] = (T)run.value(acc, i, jj);
    }
  }
}

template <typename T>
cudaError_t launch_contract_l(const SepShape &s, const double *A, const double *q, const double *qt,
                              int x0, int nxc, T *M, cudaStream_t st) {
  using C = SimtCfg<T>;
  int64_t rows = (int64_t)s.n_mu * s.nbl, cols = (int64_t)nxc * s.nbp;
  dim3 grid((unsigned)cdiv64(rows, C::BM), (unsigned)cdiv64(cols, C::BN));
  k_contract_l<T><<<grid, 256, 0, st>>>(s, A, q, qt, x0, nxc, M);
  return cudaGetLastError();
}
template cudaError_t launch_contract_l<double>(const SepShape &, const double *, const double *,
                                               const double *, int, int, double *, cudaStream_t);
template cudaError_t launch_contract_l<float>(const SepShape &, const double *, const double *,
                                              const double *, int, int, float *, cudaStream_t);

// ---------------------------------------------------------------------------
// a6 (CUDA cores): G[(a,b,{u,v}),(c,t)] (+)= sum_s Y_ab{u,v}(s) M_ct(s) over
// the chunk's slices s = (xl, j), Y = om_j W_x (M_au M_bv + M_av M_bu).
// One CTA per (b, row tile, column tile) and K split; tiles of the
// triangular block structure are decoded from blockIdx.x.
// ---------------------------------------------------------------------------
template <int BM, int BN>
__device__ __forceinline__ void decode_triple_tile(const GLayout &g, int t, int &b, int &rt, int &ct) {
  for (b = 0; b < g.nbl; ++b) {
    int nrt = (int)cdiv64(g.rows(b), BM), nct = (int)cdiv64(g.cols(b), BN);
    if (t < nrt * nct) {
      rt = t / nct;
      ct = t % nct;
      return;
    }
    t -= nrt * nct;
  }
  b = -1;
}

template <int BM, int BN>
static int64_t triple_tiles(const GLayout &g) {
  int64_t n = 0;
  for (int b = 0; b < g.nbl; ++b) n += cdiv64(g.rows(b), BM) * cdiv64(g.cols(b), BN);
  return n;
}

template <typename T>
__global__ void __launch_bounds__(256) k_triple(SepShape s, GLayout g, const T *__restrict__ M,
                                                const double *__restrict__ om,
                                                const double *__restrict__ xw, int x0, int64_t S,
                                                int64_t k_per_split, double *__restrict__ out,
                                                int64_t out_stride, int absM) {
  using C = SimtCfg<T>;
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, TM = C::TM, TN = C::TN;
  constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
  constexpr int AIT = BM * BK / NT, BIT = BN * BK / NT;
  static_assert(NT % BK == 0, "loader mapping");
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  int b, rt, ct;
  decode_triple_tile<BM, BN>(g, blockIdx.x, b, rt, ct);
  if (b < 0) return;
  const int nbp = s.nbp, nblp = s.nbl * s.nbp, n_mu = s.n_mu;
  const int64_t R = g.rows(b), Cn = g.cols(b);
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int kk_ld = tid % BK, r_ld = tid / BK;

  // loader row/column descriptors (fixed over the K loop)
  int ro1[AIT], ro2[AIT], ro3[AIT], ro4[AIT];  // offsets a*nbp+u, b*nbp+v, a*nbp+v, b*nbp+u
  bool rok[AIT];
#pragma unroll
  for (int it = 0; it < AIT; ++it) {
    int64_t row = (int64_t)rt * BM + r_ld + it * (NT / BK);
    rok[it] = row < R;
    int a = 0, uv = 0, u = 0, v = 0;
    if (rok[it]) {
      a = (int)(row / g.P2);
      uv = (int)(row % g.P2);
      pair_decode(uv, u, v);
    }
    ro1[it] = a * nbp + u;
    ro2[it] = b * nbp + v;
    ro3[it] = a * nbp + v;
    ro4[it] = b * nbp + u;
  }
  int co[BIT];
  bool cok[BIT];
#pragma unroll
  for (int it = 0; it < BIT; ++it) {
    int64_t col = (int64_t)ct * BN + r_ld + it * (NT / BK);
    cok[it] = col < Cn;
    int c = b + (int)(col / nbp), t = (int)(col % nbp);
    co[it] = cok[it] ? c * nbp + t : 0;
  }

  T acc[TM][TN];
  ChunkAcc<T, TM, TN> run;
  run.zero();
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0;

  const int64_t kbeg = (int64_t)blockIdx.y * k_per_split;
  const int64_t kend = min(S, kbeg + k_per_split);
  int step = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK, ++step) {
    const int64_t k = k0 + kk_ld;
    const bool kok = k < kend;
    const T *Mk = M + (kok ? k : 0) * nblp;
    T w = 0;
    if (kok) {
      int xl = (int)(k / n_mu), j = (int)(k % n_mu);
      w = (T)(om[j] * xw[x0 + xl]);
      if (absM && w < 0) w = -w;
    }
    // absM: the error-scale projection (every M and weight by its magnitude)
    auto ld = [&](int i) -> T {
      const T m = Mk[i];
      return (absM && m < 0) ? -m : m;
    };
#pragma unroll
    for (int it = 0; it < AIT; ++it) {
      T v = 0;
      if (kok && rok[it]) v = w * (ld(ro1[it]) * ld(ro2[it]) + ld(ro3[it]) * ld(ro4[it]));
      As[kk_ld][r_ld + it * (NT / BK)] = v;
    }
#pragma unroll
    for (int it = 0; it < BIT; ++it) {
      T v = 0;
      if (kok && cok[it]) v = ld(co[it]);
      Bs[kk_ld][r_ld + it * (NT / BK)] = v;
    }
    __syncthreads();
    simt_fma_tile<T, BM, BN, BK, TM, TN>(As, Bs, acc, tx, ty);
    __syncthreads();
    if ((step + 1) % PROMOTE_STEPS == 0) run.promote(acc);
  }
  double *o = out + (int64_t)blockIdx.y * out_stride + g.offset(b);
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t row = (int64_t)rt * BM + ty + i * TY;
    if (row >= R) continue;
#pragma unroll
    for (int jj = 0; jj < TN; ++jj) {
      int64_t col = (int64_t)ct * BN + tx + jj * TX;
      if (col >= Cn) continue;
      o[row * Cn + col] = run.value(acc, i, jj);
    }
  }
}

__global__ void k_reduce_parts(int64_t n, int nparts, const double *__restrict__ part, int64_t stride,
                               double *__restrict__ G, int accumulate) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = accumulate ? G[i] : 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * stride + i];
  G[i] = s;
}

int triple_ksplit(const SepShape &s, int nxc, int num_sms) {
  GLayout g = make_glayout(s.nbl, s.nbp);
  int64_t tiles = triple_tiles<SimtCfg<double>::BM, SimtCfg<double>::BN>(g);
  int64_t S = (int64_t)nxc * s.n_mu;
  int64_t want = cdiv64(2LL * num_sms, tiles);
  int64_t maxk = cdiv64(S, 256);  // at least 256 slices per split
  int64_t ks = want < maxk ? want : maxk;
  if (ks < 1) ks = 1;
  if (ks > 64) ks = 64;
  return (int)ks;
}

// kernels launch_triple launches: the tile kernel, plus the reduction of the
// K-split partial tables unless one split writes G directly
int triple_launches(const SepShape &s, int nxc, int ksplit, bool accumulate) {
  using C = SimtCfg<double>;
  const int64_t S = (int64_t)nxc * s.n_mu;
  const int64_t kps = cdiv64(cdiv64(S, ksplit), C::BK) * C::BK;
  const int nks = (int)cdiv64(S, kps);
  return (nks == 1 && !accumulate) ? 1 : 2;
}

template <typename T>
cudaError_t launch_triple(const SepShape &s, const T *M, const double *om, const double *xw, int x0,
                          int nxc, int ksplit, double *G, double *Gpart, bool accumulate,
                          int num_sms, cudaStream_t st, bool absM) {
  (void)num_sms;
  using C = SimtCfg<T>;
  GLayout g = make_glayout(s.nbl, s.nbp);
  int64_t tiles = triple_tiles<C::BM, C::BN>(g);
  int64_t S = (int64_t)nxc * s.n_mu;
  int64_t kps = cdiv64(cdiv64(S, ksplit), C::BK) * C::BK;
  int nks = (int)cdiv64(S, kps);
  dim3 grid((unsigned)tiles, (unsigned)nks);
  const bool direct = (nks == 1 && !accumulate);
  double *out = direct ? G : Gpart;
  k_triple<T><<<grid, 256, 0, st>>>(s, g, M, om, xw, x0, S, kps, out, g.size(), absM ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || direct) return e;
  int64_t n = g.size();
  k_reduce_parts<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(n, nks, Gpart, n, G, accumulate ? 1 : 0);
  return cudaGetLastError();
}
template cudaError_t launch_triple<double>(const SepShape &, const double *, const double *,
                                           const double *, int, int, int, double *, double *, bool,
                                           int, cudaStream_t, bool);
template cudaError_t launch_triple<float>(const SepShape &, const float *, const double *,
                                          const double *, int, int, int, double *, double *, bool,
                                          int, cudaStream_t, bool);

// ---------------------------------------------------------------------------
// a7: Gamma'[n][n'] = scale * (G[ab{pr}, c s] + G[ab{ps}, c r] + G[ab{rs}, c p])
// with (a,b,c) the sorted late triple, scale = 1/(48 pi) (Eq. 2D); in blocks
// of the second form (GLayout) the same three index calls give the
// expansion along the row of a.  Mode indices outside the basis give NaN (no
// out-of-range read).
// ---------------------------------------------------------------------------
__global__ void k_gather(GLayout g, const double *__restrict__ G, const int *__restrict__ late,
                         const int *__restrict__ prim, int n_late, int n_prim, double scale,
                         double *__restrict__ gamma) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_late * n_prim) return;
  int n = (int)(idx / n_prim), m = (int)(idx % n_prim);
  int a = late[3 * n], b = late[3 * n + 1], c = late[3 * n + 2];
  int p = prim[3 * m], r = prim[3 * m + 1], t = prim[3 * m + 2];
  if ((unsigned)a >= (unsigned)g.nbl || (unsigned)b >= (unsigned)g.nbl || (unsigned)c >= (unsigned)g.nbl ||
      (unsigned)p >= (unsigned)g.nbp || (unsigned)r >= (unsigned)g.nbp || (unsigned)t >= (unsigned)g.nbp) {
    gamma[idx] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  // sort the late triple
  if (a > b) { int z = a; a = b; b = z; }
  if (b > c) { int z = b; b = c; c = z; }
  if (a > b) { int z = a; a = b; b = z; }
  const int64_t i1 = g.index(a, b, pair_index(p, r), c, t), i2 = g.index(a, b, pair_index(p, t), c, r),
                i3 = g.index(a, b, pair_index(r, t), c, p);
  if (i1 < 0 || i2 < 0 || i3 < 0) {  // only in MODAL_DEBUG builds (checked index helpers)
    gamma[idx] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  gamma[idx] = scale * (G[i1] + G[i2] + G[i3]);
}

cudaError_t launch_gather(const SepShape &s, const double *G, const int *late, const int *prim,
                          int n_late, int n_prim, double scale, double *gamma, cudaStream_t st,
                          const GLayout *layout) {
  const GLayout g = layout ? *layout : make_glayout(s.nbl, s.nbp);
  int64_t n = (int64_t)n_late * n_prim;
  if (n == 0) return cudaSuccess;
  k_gather<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(g, G, late, prim, n_late, n_prim, scale, gamma);
  return cudaGetLastError();
}

__global__ void k_zero(double *p, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}
cudaError_t launch_zero(double *p, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_zero<<<(unsigned)cdiv64((int64_t)n, 256), 256, 0, st>>>(p, (int64_t)n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Generic FP64 GEMM with both operands K-major: C[m][n] (+)= sum_k A[m][k] B[n][k].
// Used by the direct path (Gamma += Y^T diag(z) X over a batch of triples,
// the reduction of Section 3.2.4 that the paper hands to DGEMM).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gemm_nt_f64(int m, int n, int K, const double *__restrict__ A,
                                                     int64_t lda, const double *__restrict__ B,
                                                     int64_t ldb, double *__restrict__ C, int64_t ldc,
                                                     int accumulate, const int64_t *__restrict__ kdev,
                                                     int64_t koff) {
  using Cf = SimtCfg<double>;
  if (kdev) {  // K read on the device: at most *kdev - koff terms
    const int64_t kd = *kdev - koff;
    if (kd < K) K = kd < 0 ? 0 : (int)kd;
    if (K == 0 && accumulate) return;
  }
  constexpr int BM = Cf::BM, BN = Cf::BN, BK = Cf::BK, TM = Cf::TM, TN = Cf::TN;
  constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      int kk = e % BK, r = e / BK;
      As[kk][r] = (m0 + r < m && k0 + kk < K) ? A[(int64_t)(m0 + r) * lda + k0 + kk] : 0.0;
    }
    for (int e = tid; e < BN * BK; e += NT) {
      int kk = e % BK, c = e / BK;
      Bs[kk][c] = (n0 + c < n && k0 + kk < K) ? B[(int64_t)(n0 + c) * ldb + k0 + kk] : 0.0;
    }
    __syncthreads();
    simt_fma_tile<double, BM, BN, BK, TM, TN>(As, Bs, acc, tx, ty);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int r = m0 + ty + i * TY;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int c = n0 + tx + j * TX;
      if (c >= n) continue;
      double *d = C + (int64_t)r * ldc + c;
      *d = accumulate ? *d + acc[i][j] : acc[i][j];
    }
  }
}

cudaError_t launch_gemm_nt_f64(int m, int n, int k, const double *A, int64_t lda, const double *B,
                               int64_t ldb, double *C, int64_t ldc, bool accumulate, cudaStream_t st,
                               const int64_t *kdev, int64_t koff) {
  if (m == 0 || n == 0) return cudaSuccess;
  dim3 grid(cdiv(m, 64), cdiv(n, 64));
  k_gemm_nt_f64<<<grid, 256, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, accumulate ? 1 : 0, kdev, koff);
  return cudaGetLastError();
}

}  // namespace modal
