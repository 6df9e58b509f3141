// k_basis.cu -- rows a1-a3 of the separable path: Gauss-Legendre nodes,
// the weighted Legendre table and the radial weights.
#include "common.cuh"
#include "kernels.cuh"

namespace modal {

// ---------------------------------------------------------------------------
// a1: Gauss-Legendre nodes/weights (Section 2.2).  One warp per root pair
// (+-mu).  The three-term recurrence
//   (k+1) P_{k+1} = (2k+1) mu P_k - k P_{k-1},   i.e.
//   [P_{k+1}, P_k]^T = M_k [P_k, P_{k-1}]^T,  M_k = [[a_k mu, -b_k], [1, 0]],
// with a_k = (2k+1)/(k+1), b_k = k/(k+1), is evaluated as the ordered product
// of the M_k: each lane multiplies the matrices of its segment of k, and a
// shuffle tree multiplies the 32 segment products in order, so the latency
// of one evaluation is ~n/32 steps instead of n.  Newton in FP64 from the
// usual cosine guess, then one evaluation of P_n, P_{n-1} in double-double
// at the FP64 root x0 gives the last correction d = P_n / P_n' (node
// x0 - d) and P_n'(x0); the derivative at the node follows from the Legendre
// equation, P_n'' = (2 x P_n' - n(n+1) P_n)/(1 - x^2), as P_n'(x0) - d P_n''.
// The weight 2 / ((1 - x^2) P_n'(x)^2) is formed from these in double-double
// and rounded once.  The a_k, b_k are tabulated per block in shared memory in
// double-double.  Output ascending.
// ---------------------------------------------------------------------------
constexpr int GL_WARPS = 4;  // roots per block

struct M2 {
  double a, b, c, d;  // [[a, b], [c, d]]
};
struct M2dd {
  dd a, b, c, d;
};
__device__ __forceinline__ M2 m2_mul(const M2 &x, const M2 &y) {  // x y
  return {fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c), fma(x.c, y.b, x.d * y.d)};
}
__device__ __forceinline__ M2dd m2dd_mul(const M2dd &x, const M2dd &y) {
  return {dd_add(dd_mul(x.a, y.a), dd_mul(x.b, y.c)), dd_add(dd_mul(x.a, y.b), dd_mul(x.b, y.d)),
          dd_add(dd_mul(x.c, y.a), dd_mul(x.d, y.c)), dd_add(dd_mul(x.c, y.b), dd_mul(x.d, y.d))};
}
__device__ __forceinline__ double shfl_up_d(double v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
__device__ __forceinline__ dd shfl_up_dd(dd v, int off) { return {shfl_up_d(v.hi, off), shfl_up_d(v.lo, off)}; }

// k range of this lane's segment of 1 .. n-1
__device__ __forceinline__ void gl_segment(int n, int lane, int &k0, int &k1) {
  const int len = (n - 1 + 31) / 32;
  k0 = 1 + lane * len;
  k1 = min(n, k0 + len);
}

// [P_n, P_{n-1}] at x (FP64): lane 31 returns them
__device__ __forceinline__ void leg_pair_warp_d(int n, double x, const dd *ca, const dd *cb, int lane, double &pn,
                                                double &pm) {
  int k0, k1;
  gl_segment(n, lane, k0, k1);
  M2 t = {1.0, 0.0, 0.0, 1.0};
  for (int k = k0; k < k1; ++k) {  // t = M_k t
    const double ax = ca[k].hi * x, bk = cb[k].hi;
    t = {fma(ax, t.a, -bk * t.c), fma(ax, t.b, -bk * t.d), t.a, t.b};
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {  // ordered product: higher k on the left
    M2 lo = {shfl_up_d(t.a, off), shfl_up_d(t.b, off), shfl_up_d(t.c, off), shfl_up_d(t.d, off)};
    if (lane >= off && ((lane + 1) & (2 * off - 1)) == 0) t = m2_mul(t, lo);
  }
  pn = fma(t.a, x, t.b);  // applied to [P_1, P_0] = [x, 1]
  pm = fma(t.c, x, t.d);
}

__device__ __forceinline__ void leg_pair_warp_dd(int n, double x, const dd *ca, const dd *cb, int lane, dd &pn,
                                                 dd &pm) {
  int k0, k1;
  gl_segment(n, lane, k0, k1);
  const dd one = {1.0, 0.0}, zero = {0.0, 0.0};
  M2dd t = {one, zero, zero, one};
  for (int k = k0; k < k1; ++k) {
    const dd ax = dd_mul_d(ca[k], x);
    t = {dd_sub(dd_mul(ax, t.a), dd_mul(cb[k], t.c)), dd_sub(dd_mul(ax, t.b), dd_mul(cb[k], t.d)), t.a, t.b};
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    M2dd lo = {shfl_up_dd(t.a, off), shfl_up_dd(t.b, off), shfl_up_dd(t.c, off), shfl_up_dd(t.d, off)};
    if (lane >= off && ((lane + 1) & (2 * off - 1)) == 0) t = m2dd_mul(t, lo);
  }
  pn = dd_add(dd_mul_d(t.a, x), t.b);
  pm = dd_add(dd_mul_d(t.c, x), t.d);
}

__global__ void __launch_bounds__(32 * GL_WARPS) k_gl_nodes(int n, double *__restrict__ mu, double *__restrict__ om) {
  extern __shared__ dd coef[];
  dd *ca = coef, *cb = coef + n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    ca[k] = dd_div_d({2.0 * k + 1.0, 0.0}, (double)(k + 1));
    cb[k] = dd_div_d({(double)k, 0.0}, (double)(k + 1));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * GL_WARPS + (threadIdx.x >> 5);  // root pair of this warp
  const int half = (n + 1) / 2;
  if (i >= half) return;  // warp-uniform
  if (n == 1) {
    if (lane == 0) {
      mu[0] = 0.0;
      om[0] = 2.0;
    }
    return;
  }
  const double nn = (double)n;
  double x = (1.0 - (nn - 1.0) / (8.0 * nn * nn * nn)) * cos(MODAL_PI * (4.0 * i + 3.0) / (4.0 * nn + 2.0));
  for (int it = 0; it < 12; ++it) {
    double pn, pm;
    leg_pair_warp_d(n, x, ca, cb, lane, pn, pm);
    double dx = 0.0;
    if (lane == 31) {
      const double dp = nn * (x * pn - pm) / (x * x - 1.0);
      dx = pn / dp;
    }
    dx = __shfl_sync(0xffffffffu, dx, 31);
    x -= dx;
    if (fabs(dx) <= 1e-15 * fabs(x)) break;  // warp-uniform
  }
  if ((n & 1) && i == n / 2) x = 0.0;  // exact centre node of an odd rule
  dd pn, pm;
  leg_pair_warp_dd(n, x, ca, cb, lane, pn, pm);
  if (lane != 31) return;
  const dd one = {1.0, 0.0};
  const dd X0 = {x, 0.0};
  const dd x2m1 = dd_sub(dd_mul_d(X0, x), one);                             // x0^2 - 1 (exact-ish)
  const dd dp0 = dd_div(dd_mul_d(dd_sub(dd_mul_d(pn, x), pm), nn), x2m1);  // P_n'(x0)
  const double d = (pn.hi + pn.lo) / (dp0.hi + dp0.lo);                    // Newton step
  const double ddp = (2.0 * x * (dp0.hi + dp0.lo) - nn * (nn + 1.0) * (pn.hi + pn.lo)) / (1.0 - x * x);
  const dd X = dd_sub(X0, {d, 0.0});                                        // node
  const dd dpx = dd_sub(dp0, {d * ddp, 0.0});                               // P_n'(node)
  const dd omx = dd_sub(one, dd_mul(X, X));
  const dd w = dd_div({2.0, 0.0}, dd_mul(omx, dd_mul(dpx, dpx)));
  const double xv = X.hi + X.lo, wv = w.hi + w.lo;
  if ((n & 1) && i == n / 2) {
    mu[i] = 0.0;
    om[i] = wv;
    return;
  }
  mu[n - 1 - i] = xv;
  om[n - 1 - i] = wv;
  mu[i] = -xv;
  om[i] = wv;
}

// ---------------------------------------------------------------------------
// a2: A[j][l - l_min] = w_l P_l(mu_j) (the `factor` array of the Modal2D
// listing).  A block of 128 threads owns 128 nodes; each thread runs the
// FP64 recurrence for its node, 32 l at a time into shared memory, and the
// block writes the 128 x 32 tile with coalesced row segments.
// ---------------------------------------------------------------------------
constexpr int LEG_NODES = 128;
constexpr int LEG_LT = 32;

__global__ void __launch_bounds__(LEG_NODES) k_legendre_table(int n_mu, const double *__restrict__ mu,
                                                            int l_min, int l_max,
                                                            const double *__restrict__ w_l,
                                                            double *__restrict__ A) {
  __shared__ double tile[LEG_NODES][LEG_LT + 1];
  const int L = l_max - l_min + 1;
  const int j0 = blockIdx.x * LEG_NODES;
  const int j = j0 + threadIdx.x;
  __shared__ double rinv[LEG_LT];  // 1 / (l + 1) for the degrees l of the window
  double x = (j < n_mu) ? mu[j] : 0.0;
  double p0 = 1.0, p1 = x;  // P_{l}, P_{l+1} with l = next degree to emit
  int lnext = 0;            // degree held in p0
  while (lnext < l_min) {   // up to the first degree (l_min is small)
    const double p2 = ((2.0 * lnext + 3.0) * x * p1 - (double)(lnext + 1) * p0) / (double)(lnext + 2);
    p0 = p1;
    p1 = p2;
    ++lnext;
  }
  for (int lb = l_min; lb <= l_max; lb += LEG_LT) {
    // the divisions of the window's steps, one per thread and off the
    // recurrence's dependency chain (an FP64 division is a long sequence on
    // this part's FP64 pipe)
    if (threadIdx.x < LEG_LT) rinv[threadIdx.x] = 1.0 / (double)(lb + threadIdx.x + 1);
    __syncthreads();
    for (int c = 0; c < LEG_LT; ++c) {
      const int l = lb + c;
      if (l > lnext) {  // one step: P_l from P_{l-1}, P_{l-2} (divisor l + 1 = (l - 1) + 2)
        const double p2 = ((2.0 * lnext + 3.0) * x * p1 - (double)(lnext + 1) * p0) * rinv[c];
        p0 = p1;
        p1 = p2;
        ++lnext;
      }
      double v = 0.0;
      if (l <= l_max) v = (w_l ? w_l[l - l_min] : 1.0) * p0;
      tile[threadIdx.x][c] = v;
    }
    __syncthreads();
    // coalesced write: warp w writes rows w, w+4, ...; lane = column
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < LEG_NODES; r += LEG_NODES / 32) {
      int jj = j0 + r, l = lb + lane;
      if (jj < n_mu && l <= l_max) A[(size_t)jj * L + (l - l_min)] = tile[r][lane];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// a3: radial weights including x^2 (Section 3.2.4).
// kind 0: trapezium; kind 1: Hermite cubic with forward-difference slopes,
// integrated exactly per interval:
//   int_k = dr_k/2 (y_k + y_{k+1}) + dr_k^2/12 (D_k - D_{k+1}), D_k = dy_k/dr_k,
// with D at the last node equal to the last interval's.  The weight of node
// m collects the coefficient of y_m from every interval touching it.
// ---------------------------------------------------------------------------
__global__ void k_x_weights(int kind, int n, const double *__restrict__ x, double *__restrict__ w) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s = 0.0;
  if (n >= 2) {
    // trapezium part
    if (m > 0) s += 0.5 * (x[m] - x[m - 1]);
    if (m < n - 1) s += 0.5 * (x[m + 1] - x[m]);
    if (kind == 1) {
      // slope D_k = (y_{k+1} - y_k) / h_k depends on y_k (-1/h_k) and y_{k+1} (+1/h_k).
      // interval k adds h_k^2/12 (D_k - D_{k+1}); for k = n-2, D_{k+1} := D_k.
      for (int k = max(0, m - 2); k <= min(n - 2, m); ++k) {
        double hk = x[k + 1] - x[k];
        double c = hk * hk / 12.0;
        double dDk = (m == k + 1 ? 1.0 / hk : 0.0) - (m == k ? 1.0 / hk : 0.0);
        double dDk1;
        if (k + 2 <= n - 1) {
          double h1 = x[k + 2] - x[k + 1];
          dDk1 = (m == k + 2 ? 1.0 / h1 : 0.0) - (m == k + 1 ? 1.0 / h1 : 0.0);
        } else {
          dDk1 = dDk;
        }
        s += c * (dDk - dDk1);
      }
    }
  }
  w[m] = s * x[m] * x[m];
}

// Ratio table c_n = prod_{k=1..n} (1 - 1/(2k)), n = 0..nmax, each entry in
// double-double then rounded: (l1 l2 l3;000)^2 = c_{g-l1} c_{g-l2} c_{g-l3} /
// ((2g+1) c_g) with 2g = l1 + l2 + l3 (the factorial form, Section 2.1).
// One CTA: the factors go in blocks of TJ_B; the products of the blocks, their
// running products, then each entry as its block's running product times the
// factors of its own block up to n (at most TJ_B double-double steps per
// thread and phase instead of n).
constexpr int TJ_B = 32, TJ_MAXBLK = 1024;
__device__ __forceinline__ dd tj_factors(dd p, int k0, int k1) {  // p prod_{k0 <= k <= k1} (2k - 1)/(2k)
  for (int k = k0; k <= k1; ++k) p = dd_div_d(dd_mul_d(p, 2.0 * k - 1.0), 2.0 * k);
  return p;
}
__global__ void __launch_bounds__(1024) k_threej_table(int nmax, double *__restrict__ c) {
  __shared__ dd run[TJ_MAXBLK];  // run[b] = product of the factors 1 .. b TJ_B
  const int nblk = nmax / TJ_B + 1;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    run[b] = b == 0 ? dd{1.0, 0.0} : tj_factors(dd{1.0, 0.0}, (b - 1) * TJ_B + 1, b * TJ_B);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int b = 1; b < nblk; ++b) run[b] = dd_mul(run[b - 1], run[b]);
  __syncthreads();
  for (int n = threadIdx.x; n <= nmax; n += blockDim.x) {
    const int b = n / TJ_B;
    const dd p = tj_factors(run[b], b * TJ_B + 1, n);
    c[n] = p.hi + p.lo;
  }
}

// ---- launchers -------------------------------------------------------------
cudaError_t launch_gl_nodes(int n, double *mu, double *om, cudaStream_t st) {
  int half = (n + 1) / 2;
  size_t smem = 2 * sizeof(dd) * (size_t)n;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;  // n > 6400: not supported
  cudaError_t e = cudaFuncSetAttribute(k_gl_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gl_nodes<<<cdiv(half, GL_WARPS), 32 * GL_WARPS, smem, st>>>(n, mu, om);
  return cudaGetLastError();
}
cudaError_t launch_legendre_table(int n_mu, const double *mu, int l_min, int l_max,
                                  const double *w_l, double *A, cudaStream_t st) {
  k_legendre_table<<<cdiv(n_mu, LEG_NODES), LEG_NODES, 0, st>>>(n_mu, mu, l_min, l_max, w_l, A);
  return cudaGetLastError();
}
cudaError_t launch_x_weights(int kind, int n, const double *x, double *w, cudaStream_t st) {
  k_x_weights<<<cdiv(n, 128), 128, 0, st>>>(kind, n, x, w);
  return cudaGetLastError();
}
cudaError_t launch_threej_table(int nmax, double *c, cudaStream_t st) {
  if (nmax / TJ_B + 1 > TJ_MAXBLK) return cudaErrorInvalidValue;  // l_max beyond ~21800
  k_threej_table<<<1, 1024, 0, st>>>(nmax, c);
  return cudaGetLastError();
}

}  // namespace modal
