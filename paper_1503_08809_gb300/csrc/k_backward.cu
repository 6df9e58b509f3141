// k_backward.cu -- row a9: adjoint of the separable projection (not in the
// paper; it follows from Eq. 2D and Eq. legendre).
//
// Forward, per slice s = (x, mu_j) with w_s = om_j W_x:
//   G[(a,b,{u,v}),(c,t)] = sum_s Y_ab{u,v}(s) M_ct(s),
//   Y_ab{u,v}(s) = w_s (M_au M_bv + M_av M_bu),
//   Gamma'[n][n'] = 1/(48 pi) (G[ab{pr},cs] + G[ab{ps},cr] + G[ab{rs},cp]).
// Backward, given gbar = dL/dGamma':
//   Gbar  = scatter of gbar / (48 pi) onto the three G entries of each (n, n'),
//   dM_ct(s) += sum_rows Gbar[row,(c,t)] Y_row(s)                 (M as right operand)
//   dY_row(s) = sum_cols Gbar[row,col] M_col(s)                    (M inside Y)
//   dM_au += w dY M_bv,  dM_bv += w dY M_au,  dM_av += w dY M_bu,  dM_bu += w dY M_av,
//   dq~_p(l,x) = sum_{j,a} dM_ap(x,j) A[j][l] q_a(l),   A[j][l] = w_l P_l(mu_j),
//   dq_a(l)    = sum_{x,j,p} dM_ap(x,j) A[j][l] q~_p(l,x).
// M is recomputed per radial chunk (never stored for the whole problem).
#include <cstdio>

#include "backward.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace modal {

static thread_local char g_bw_err[256] = "";
const char *backward_last_error() { return g_bw_err; }

// ---- 1. scatter dL/dGamma' onto the G layout ------------------------------
__global__ void k_scatter_gbar(GLayout g, const double *__restrict__ gbar, const int *__restrict__ late,
                               const int *__restrict__ prim, int n_late, int n_prim, double scale,
                               double *__restrict__ Gbar) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_late * n_prim) return;
  int n = (int)(idx / n_prim), m = (int)(idx % n_prim);
  int a = late[3 * n], b = late[3 * n + 1], c = late[3 * n + 2];
  int p = prim[3 * m], r = prim[3 * m + 1], t = prim[3 * m + 2];
  if ((unsigned)a >= (unsigned)g.nbl || (unsigned)b >= (unsigned)g.nbl || (unsigned)c >= (unsigned)g.nbl ||
      (unsigned)p >= (unsigned)g.nbp || (unsigned)r >= (unsigned)g.nbp || (unsigned)t >= (unsigned)g.nbp)
    return;
  if (a > b) { int z = a; a = b; b = z; }
  if (b > c) { int z = b; b = c; c = z; }
  if (a > b) { int z = a; a = b; b = z; }
  double v = scale * gbar[idx];
  const int64_t i1 = g.index(a, b, pair_index(p, r), c, t), i2 = g.index(a, b, pair_index(p, t), c, r),
                i3 = g.index(a, b, pair_index(r, t), c, p);
  if (i1 < 0 || i2 < 0 || i3 < 0) return;  // only in MODAL_DEBUG builds (checked index helpers)
  atomicAdd(Gbar + i1, v);
  atomicAdd(Gbar + i2, v);
  atomicAdd(Gbar + i3, v);
}

// ---- 2. dL/dM for a chunk of KS slices per CTA ------------------------------
// Shared memory: Ms[KS][nblp], dMs[KS][nblp] (both of type T), and per tile
// Gt[RT][CT+1], Yt[RT][KS], dYt[RT][KS].  Loops: row tiles of every block b,
// column tiles inside; dY accumulates over the column tiles of a row tile and
// is then folded into dMs with the product rule.
constexpr int BW_RT = 64, BW_CT = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_dM(SepShape s, GLayout g, const T *__restrict__ M,
                                            const double *__restrict__ Gbar, const double *__restrict__ om,
                                            const double *__restrict__ xw, int x0, int64_t S, int KS,
                                            T *__restrict__ dM) {
  extern __shared__ unsigned char smraw[];
  const int nbp = s.nbp, nblp = s.nbl * s.nbp, n_mu = s.n_mu;
  T *Ms = reinterpret_cast<T *>(smraw);
  T *dMs = Ms + (size_t)KS * nblp;
  T *Gt = dMs + (size_t)KS * nblp;            // [RT][CT+1]
  T *Yt = Gt + BW_RT * (BW_CT + 1);           // [RT][KS]
  T *dYt = Yt + BW_RT * KS;                   // [RT][KS]
  T *wk = dYt + BW_RT * KS;                   // [KS]
  const int tid = threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.x * KS;
  const int nk = (int)min((int64_t)KS, S - k0);
  for (int e = tid; e < KS * nblp; e += blockDim.x) {
    int kk = e / nblp;
    Ms[e] = kk < nk ? M[(k0 + kk) * nblp + (e % nblp)] : (T)0;
    dMs[e] = 0;
  }
  for (int kk = tid; kk < KS; kk += blockDim.x) {
    T w = 0;
    if (kk < nk) {
      int64_t k = k0 + kk;
      w = (T)(om[k % n_mu] * xw[x0 + k / n_mu]);
    }
    wk[kk] = w;
  }
  __syncthreads();
  for (int b = 0; b < g.nbl; ++b) {
    const int64_t R = g.rows(b), C = g.cols(b);
    const double *Gb = Gbar + g.offset(b);
    for (int64_t r0 = 0; r0 < R; r0 += BW_RT) {
      const int nr = (int)min((int64_t)BW_RT, R - r0);
      // Y tile for these rows
      for (int e = tid; e < BW_RT * KS; e += blockDim.x) {
        int rr = e % BW_RT, kk = e / BW_RT;  // Yt, dYt are [KS][RT]
        T v = 0, dz = 0;
        if (rr < nr) {
          int64_t row = r0 + rr;
          int a = (int)(row / g.P2), uv = (int)(row % g.P2), u, vv;
          pair_decode(uv, u, vv);
          const T *Mk = Ms + (size_t)kk * nblp;
          v = wk[kk] * (Mk[a * nbp + u] * Mk[b * nbp + vv] + Mk[a * nbp + vv] * Mk[b * nbp + u]);
        }
        Yt[e] = v;
        dYt[e] = dz;
      }
      for (int64_t c0 = 0; c0 < C; c0 += BW_CT) {
        const int nc = (int)min((int64_t)BW_CT, C - c0);
        __syncthreads();
        for (int e = tid; e < BW_RT * BW_CT; e += blockDim.x) {
          int rr = e / BW_CT, cc = e % BW_CT;
          Gt[rr * (BW_CT + 1) + cc] = (rr < nr && cc < nc) ? (T)Gb[(r0 + rr) * C + c0 + cc] : (T)0;
        }
        __syncthreads();
        // right-operand role: dMs[k][b*nbp + c0 + cc] += sum_rr Gt[rr][cc] Yt[rr][k]
        for (int e = tid; e < BW_CT * KS; e += blockDim.x) {
          int cc = e % BW_CT, kk = e / BW_CT;
          if (cc >= nc) continue;
          T acc = 0;
          const T *yk = Yt + kk * BW_RT;
          for (int rr = 0; rr < nr; ++rr) acc = fma(Gt[rr * (BW_CT + 1) + cc], yk[rr], acc);
          dMs[(size_t)kk * nblp + b * nbp + c0 + cc] += acc;
        }
        // inside-Y role: dYt[rr][k] += sum_cc Gt[rr][cc] M_k[b*nbp + c0 + cc]
        for (int e = tid; e < BW_RT * KS; e += blockDim.x) {
          int rr = e % BW_RT, kk = e / BW_RT;
          if (rr >= nr) continue;
          const T *Mk = Ms + (size_t)kk * nblp + b * nbp + c0;
          T acc = 0;
          for (int cc = 0; cc < nc; ++cc) acc = fma(Gt[rr * (BW_CT + 1) + cc], Mk[cc], acc);
          dYt[e] += acc;
        }
      }
      __syncthreads();
      // product rule: fold dY into dM (shared-memory atomics: rows share entries)
      for (int e = tid; e < BW_RT * KS; e += blockDim.x) {
        int rr = e % BW_RT, kk = e / BW_RT;
        if (rr >= nr) continue;
        int64_t row = r0 + rr;
        int a = (int)(row / g.P2), uv = (int)(row % g.P2), u, vv;
        pair_decode(uv, u, vv);
        T d = wk[kk] * dYt[e];
        const T *Mk = Ms + (size_t)kk * nblp;
        T *dk = dMs + (size_t)kk * nblp;
        atomicAdd(dk + a * nbp + u, d * Mk[b * nbp + vv]);
        atomicAdd(dk + b * nbp + vv, d * Mk[a * nbp + u]);
        atomicAdd(dk + a * nbp + vv, d * Mk[b * nbp + u]);
        atomicAdd(dk + b * nbp + u, d * Mk[a * nbp + vv]);
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < nk * nblp; e += blockDim.x) dM[k0 * nblp + e] = dMs[e];
}

// ---- 3. Generic SIMT GEMM with functor loaders (backward contractions) ----
template <typename T>
struct BwCfg {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

// dq~: rows m = (xl, p), cols n = l, k = (j, a)
template <typename T>
struct DqtOps {
  const T *dM;
  const double *A, *q;
  int L, n_mu, nbl, nbp;
  __device__ double a(int64_t m, int64_t k) const {
    int xl = (int)(m / nbp), p = (int)(m % nbp);
    int j = (int)(k / nbl), aa = (int)(k % nbl);
    return (double)dM[(((int64_t)xl * n_mu + j) * nbl + aa) * nbp + p];
  }
  __device__ double b(int64_t n, int64_t k) const {
    int j = (int)(k / nbl), aa = (int)(k % nbl);
    return A[(int64_t)j * L + n] * q[(int64_t)aa * L + n];
  }
};
// dq: rows m = a, cols n = l, k = (xl, j, p)
template <typename T>
struct DqOps {
  const T *dM;
  const double *A, *qt;
  int L, n_mu, nbl, nbp, x0;
  __device__ double a(int64_t m, int64_t k) const {
    int64_t xj = k / nbp;
    int p = (int)(k % nbp);
    return (double)dM[(xj * nbl + m) * nbp + p];
  }
  __device__ double b(int64_t n, int64_t k) const {
    int64_t xj = k / nbp;
    int p = (int)(k % nbp);
    int xl = (int)(xj / n_mu), j = (int)(xj % n_mu);
    return A[(int64_t)j * L + n] * qt[((int64_t)(x0 + xl) * nbp + p) * L + n];
  }
};

// C[m][n] = sum_k a(m,k) b(n,k) over this CTA's K range; out(m, n, v) stores.
// T-typed products with an FP64 accumulator every BK*2 terms (FP32 form).
template <typename T, class Ops, bool ATOMIC>
__global__ void __launch_bounds__(256) k_gemm_ops(int64_t Mr, int64_t Nc, int64_t K, int64_t kps, Ops ops,
                                                  double *__restrict__ out, int64_t ldo) {
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, TX = BN / TN, TY = BM / TM, NT = 256;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int64_t kb = (int64_t)blockIdx.z * kps, ke = min(K, kb + kps);
  T acc[TM][TN];
  float hi[TM][TN], lo[TM][TN];  // double-FP32 running sum of FP32 chunk sums (FP32 form)
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) { acc[i][j] = 0; hi[i][j] = 0.f; lo[i][j] = 0.f; }
  int step = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += BK, ++step) {
    for (int e = tid; e < BM * BK; e += NT) {
      int kk = e % BK, r = e / BK;
      int64_t m = m0 + r, k = k0 + kk;
      As[kk][r] = (m < Mr && k < ke) ? (T)ops.a(m, k) : (T)0;
    }
    for (int e = tid; e < BN * BK; e += NT) {
      int kk = e % BK, c = e / BK;
      int64_t n = n0 + c, k = k0 + kk;
      Bs[kk][c] = (n < Nc && k < ke) ? (T)ops.b(n, k) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + i * TY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (sizeof(T) == 4 && (step & 1)) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          float a = hi[i][j], b = (float)acc[i][j];
          float s = a + b, bb = s - a;
          float e = (a - (s - bb)) + (b - bb) + lo[i][j];
          hi[i][j] = s + e;
          lo[i][j] = e - (hi[i][j] - s);
          acc[i][j] = 0;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty + i * TY;
    if (m >= Mr) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx + j * TX;
      if (n >= Nc) continue;
      double v = (double)hi[i][j] + (double)lo[i][j] + (double)acc[i][j];
      if (ATOMIC) atomicAdd(out + m * ldo + n, v);
      else out[m * ldo + n] = v;
    }
  }
}

// ---- host driver -----------------------------------------------------------
static int bw_ks(const SepShape &s, size_t elem) {
  const size_t budget = 200 * 1024;
  const size_t tiles = elem * (BW_RT * (BW_CT + 1));
  size_t per_k = elem * (2 * (size_t)s.nbl * s.nbp + 2 * BW_RT + 1);
  if (budget <= tiles + per_k) return 1;
  int ks = (int)((budget - tiles) / per_k);
  return ks > 32 ? 32 : (ks < 1 ? 1 : ks);
}
static size_t bw_smem(const SepShape &s, size_t elem, int ks) {
  return elem * (2 * (size_t)ks * s.nbl * s.nbp + BW_RT * (BW_CT + 1) + 2 * (size_t)BW_RT * ks + ks);
}

size_t backward_scratch_bytes(const SepShape &s, int nxc, int prec) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t elem = prec == MODAL_PREC_FP64 ? 8 : 4;
  GLayout g = make_glayout(s.nbl, s.nbp);
  size_t b = 2 * up(8 * (size_t)s.n_mu) + up(8 * (size_t)s.n_mu * s.L) + up(8 * (size_t)g.size());
  b += 2 * up(elem * (size_t)nxc * s.n_mu * s.nbl * s.nbp);  // M and dM chunks
  return b + 1024;
}

template <typename T>
static cudaError_t bw_chunk(const SepShape &s, const modal_problem *p, const double *A, const double *om,
                            const double *Gbar, int x0, int nxc, T *M, T *dM, double *dqt, double *dq,
                            int num_sms, cudaStream_t st) {
  cudaError_t e = launch_contract_l<T>(s, A, p->q, p->qt, x0, nxc, M, st);
  if (e != cudaSuccess) return e;
  GLayout g = make_glayout(s.nbl, s.nbp);
  const int64_t S = (int64_t)nxc * s.n_mu;
  const int KS = bw_ks(s, sizeof(T));
  const size_t smem = bw_smem(s, sizeof(T), KS);
  e = cudaFuncSetAttribute(k_dM<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dM<T><<<(unsigned)cdiv64(S, KS), 256, smem, st>>>(s, g, M, Gbar, om, p->x_w, x0, S, KS, dM);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // dq~ rows (xl, p) of this chunk: a plain store into dqt[x0 + xl]
  {
    DqtOps<T> ops{dM, A, p->q, s.L, s.n_mu, s.nbl, s.nbp};
    int64_t Mr = (int64_t)nxc * s.nbp, Nc = s.L, K = (int64_t)s.n_mu * s.nbl;
    dim3 grid((unsigned)cdiv64(Mr, 64), (unsigned)cdiv64(Nc, 64), 1);
    k_gemm_ops<T, DqtOps<T>, false><<<grid, 256, 0, st>>>(Mr, Nc, K, K, ops,
                                                          dqt + (int64_t)x0 * s.nbp * s.L, s.L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (dq) {
    DqOps<T> ops{dM, A, p->qt, s.L, s.n_mu, s.nbl, s.nbp, x0};
    int64_t Mr = s.nbl, Nc = s.L, K = (int64_t)nxc * s.n_mu * s.nbp;
    int64_t tiles = cdiv64(Mr, 64) * cdiv64(Nc, 64);
    int64_t want = cdiv64(4LL * num_sms, tiles);
    int64_t kps = cdiv64(cdiv64(K, want), 4096) * 4096;
    int64_t nks = cdiv64(K, kps);
    dim3 grid((unsigned)cdiv64(Mr, 64), (unsigned)cdiv64(Nc, 64), (unsigned)nks);
    k_gemm_ops<T, DqOps<T>, true><<<grid, 256, 0, st>>>(Mr, Nc, K, kps, ops, dq, s.L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int run_backward(const SepShape &s, int nxc, int prec, const modal_problem *p, const double *gbar, double *dqt,
                 double *dq, void *scratch, int num_sms, cudaStream_t st) {
  auto fail = [](cudaError_t e, const char *what) {
    snprintf(g_bw_err, sizeof g_bw_err, "%s: %s", what, cudaGetErrorString(e));
    return MODAL_ECUDA;
  };
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const bool f64 = prec == MODAL_PREC_FP64;
  const size_t elem = f64 ? 8 : 4;
  GLayout g = make_glayout(s.nbl, s.nbp);
  char *w = (char *)scratch;
  double *mu = (double *)w; w += up(8 * (size_t)s.n_mu);
  double *om = (double *)w; w += up(8 * (size_t)s.n_mu);
  double *A = (double *)w; w += up(8 * (size_t)s.n_mu * s.L);
  double *Gbar = (double *)w; w += up(8 * (size_t)g.size());
  void *M = w; w += up(elem * (size_t)nxc * s.n_mu * s.nbl * s.nbp);
  void *dM = w;
  cudaError_t e;
  if ((e = launch_zero(dqt, (size_t)s.n_x * s.nbp * s.L, st)) != cudaSuccess) return fail(e, "zero dqt");
  if (dq && (e = launch_zero(dq, (size_t)s.nbl * s.L, st)) != cudaSuccess) return fail(e, "zero dq");
  if (s.n_x == 0 || (int64_t)p->n_late * p->n_prim == 0) return MODAL_OK;
  if ((e = launch_gl_nodes(s.n_mu, mu, om, st)) != cudaSuccess) return fail(e, "gl nodes");
  if ((e = launch_legendre_table(s.n_mu, mu, s.l_min, s.l_max, p->w_l, A, st)) != cudaSuccess)
    return fail(e, "legendre table");
  if ((e = launch_zero(Gbar, (size_t)g.size(), st)) != cudaSuccess) return fail(e, "zero Gbar");
  {
    int64_t n = (int64_t)p->n_late * p->n_prim;
    k_scatter_gbar<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(g, gbar, p->late_modes, p->prim_modes, p->n_late,
                                                              p->n_prim, 1.0 / (48.0 * MODAL_PI), Gbar);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "scatter");
  }
  for (int x0 = 0; x0 < s.n_x; x0 += nxc) {
    int nc = (s.n_x - x0) < nxc ? (s.n_x - x0) : nxc;
    if (f64)
      e = bw_chunk<double>(s, p, A, om, Gbar, x0, nc, (double *)M, (double *)dM, dqt, dq, num_sms, st);
    else
      e = bw_chunk<float>(s, p, A, om, Gbar, x0, nc, (float *)M, (float *)dM, dqt, dq, num_sms, st);
    if (e != cudaSuccess) return fail(e, "adjoint chunk");
  }
  return MODAL_OK;
}

}  // namespace modal
