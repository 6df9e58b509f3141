// k_direct.cu -- row a8: the direct (non-separable) projection of Eq. 3D on
// a multipole grid.  Triples l1 <= l2 <= l3 (the Modal3D listing's loop
// bounds) are enumerated on the device into one flat list (the flattened
// triangular iteration space of Section 3.2.1), then processed in batches:
//   X[n'][t] = sum_x W_x sum_perm q~ q~ q~   (radial integral per triple)
//   Y[n][t]  = z_t sum_perm q q q            (late side times the weight)
//   Gamma   += Y X^T                         (the DGEMM reduction of Section 3.2.4)
#include <cub/device/device_scan.cuh>

#include "common.cuh"
#include "direct.cuh"
#include "kernels.cuh"

namespace modal {

// qt[x][p][l] -> qtT[l][x][p]: one slab of all (x, p) per multipole.
__global__ void k_transpose(const double *__restrict__ in, int64_t rows, int64_t cols,
                            double *__restrict__ out) {
  __shared__ double t[32][33];
  int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][i];
  }
}

// Count valid l3 for each grid pair (i1 <= i2): l3 = grid[i3], i3 >= i2,
// l3 <= l1 + l2 (triangle; the grid is increasing), and even l1+l2+l3 in
// EXACT mode (the 3j symbol vanishes otherwise).
__global__ void k_direct_count(int ng, const int *__restrict__ grid, int mode,
                               int64_t *__restrict__ counts) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ng * ng) return;
  int i1 = (int)(idx / ng), i2 = (int)(idx % ng);
  int64_t c = 0;
  if (i2 >= i1) {
    int l1 = grid[i1], l2 = grid[i2];
    for (int i3 = i2; i3 < ng; ++i3) {
      int l3 = grid[i3];
      if (l3 > l1 + l2) break;
      if (mode == MODAL_W_EXACT_3J && ((l1 + l2 + l3) & 1)) continue;
      ++c;
    }
  }
  counts[idx] = c;
}

// Length of the flat triple list: the last pair's offset plus its count.
__global__ void k_direct_total(const int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
                               int64_t npairs, int64_t *__restrict__ ntri) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *ntri = npairs > 0 ? offsets[npairs - 1] + counts[npairs - 1] : 0;
}

// Triples t0 .. t0 + T - 1 of the flat list (grid pairs (i1 <= i2) in
// row-major order, then l3 ascending) with their weights
//   z = mult * dw1 dw2 dw3 * w_l1 w_l2 w_l3 * H / (144 pi),
// into batch-local arrays.  Thread tt finds its pair by a binary search of
// the scanned pair counts and its l3 by counting that pair's valid ones; the
// list's length is read on the device (threads past it write nothing).
__global__ void k_direct_fill_batch(int ng, const int *__restrict__ grid, const double *__restrict__ dw,
                                    const double *__restrict__ w_l, int l_min, const double *__restrict__ ctab,
                                    int mode, const int64_t *__restrict__ offsets, const int64_t *__restrict__ ntri,
                                    int64_t t0, int T, int *__restrict__ tri, double *__restrict__ z) {
  const int tt = blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= T) return;
  const int64_t t = t0 + tt;
  if (t >= *ntri) return;
  // the last pair whose offset is <= t (pairs with no triples share the next
  // pair's offset, so this one has t inside its range)
  int64_t lo = 0, hi = (int64_t)ng * ng;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= t) lo = mid + 1;
    else hi = mid;
  }
  const int64_t pr = lo - 1;
  const int i1 = (int)(pr / ng), i2 = (int)(pr % ng);
  int64_t k = t - offsets[pr];
  const int l1 = grid[i1], l2 = grid[i2];
  for (int i3 = i2; i3 < ng; ++i3) {
    const int l3 = grid[i3];
    if (l3 > l1 + l2) break;
    if (mode == MODAL_W_EXACT_3J && ((l1 + l2 + l3) & 1)) continue;
    if (k-- > 0) continue;
    tri[3 * tt] = l1;
    tri[3 * tt + 1] = l2;
    tri[3 * tt + 2] = l3;
    z[tt] = direct_weight(l1, l2, l3, i1, i2, i3, dw, w_l, l_min, ctab, mode);
    return;
  }
}

// X[n'][tt] for one triple per CTA.  Z[p][{u,v}] = sum_x q~_p(l1,x) U[x][{u,v}],
// U = W_x (q~_u(l2) q~_v(l3) + q~_v(l2) q~_u(l3)); then the symmetrised value
// X = Z[p][{r,s}] + Z[r][{p,s}] + Z[s][{p,r}] (the permanent expanded along l1).
__global__ void __launch_bounds__(256) k_direct_X(int nbp, int n_x, int l_min, const double *__restrict__ qtT,
                                                  const double *__restrict__ xw, const int *__restrict__ tri,
                                                  int64_t t0, int T, int xc, const int *__restrict__ prim,
                                                  int n_prim, double *__restrict__ Xb,
                                                  const int64_t *__restrict__ ntri, int64_t tglob0) {
  extern __shared__ double sm[];
  if (tglob0 + blockIdx.x >= *ntri) return;  // past the end of the triple list (whole block)
  const int P2 = nbp * (nbp + 1) / 2;
  const int NZ = nbp * P2;
  double *Z = sm;                      // [nbp][P2]
  double *U = Z + NZ;                  // [xc][P2]
  double *q1 = U + (int64_t)xc * P2;   // [xc][nbp]
  double *q2 = q1 + xc * nbp;
  double *q3 = q2 + xc * nbp;
  const int tt = blockIdx.x;
  const int64_t t = t0 + tt;
  const int l1 = tri[3 * t], l2 = tri[3 * t + 1], l3 = tri[3 * t + 2];
  const int64_t slab = (int64_t)n_x * nbp;
  const double *s1 = qtT + (int64_t)(l1 - l_min) * slab;
  const double *s2 = qtT + (int64_t)(l2 - l_min) * slab;
  const double *s3 = qtT + (int64_t)(l3 - l_min) * slab;
  for (int o = threadIdx.x; o < NZ; o += blockDim.x) Z[o] = 0.0;
  for (int x0 = 0; x0 < n_x; x0 += xc) {
    int nx = min(xc, n_x - x0);
    __syncthreads();
    for (int e = threadIdx.x; e < nx * nbp; e += blockDim.x) {
      int64_t gidx = (int64_t)x0 * nbp + e;
      q1[e] = s1[gidx];
      q2[e] = s2[gidx];
      q3[e] = s3[gidx];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nx * P2; e += blockDim.x) {
      int xl = e / P2, uv = e % P2, u, v;
      pair_decode(uv, u, v);
      const double *a2 = q2 + xl * nbp, *a3 = q3 + xl * nbp;
      U[e] = xw[x0 + xl] * (a2[u] * a3[v] + a2[v] * a3[u]);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < NZ; o += blockDim.x) {
      int p = o / P2, uv = o % P2;
      double s = Z[o];
      for (int xl = 0; xl < nx; ++xl) s = fma(q1[xl * nbp + p], U[xl * P2 + uv], s);
      Z[o] = s;
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < n_prim; m += blockDim.x) {
    int p = prim[3 * m], r = prim[3 * m + 1], s = prim[3 * m + 2];
    double v;
    if ((unsigned)p >= (unsigned)nbp || (unsigned)r >= (unsigned)nbp || (unsigned)s >= (unsigned)nbp)
      v = __longlong_as_double(0x7ff8000000000000LL);
    else
      v = Z[p * P2 + pair_index(r, s)] + Z[r * P2 + pair_index(p, s)] + Z[s * P2 + pair_index(p, r)];
    Xb[(int64_t)m * T + tt] = v;
  }
}

// Y[n][tt] = z_t sum over the 6 assignments of (a,b,c) to (l1,l2,l3).
__global__ void k_direct_Y(int nbl, int L, int l_min, const double *__restrict__ q,
                           const int *__restrict__ tri, const double *__restrict__ z, int64_t t0,
                           int T, const int64_t *__restrict__ ntri, int64_t tglob0, const int *__restrict__ late,
                           int n_late, double *__restrict__ Yb) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_late * T) return;
  const int64_t ntri_batch = *ntri - tglob0;  // triples of this batch (<= 0: none)
  if (ntri_batch <= 0) return;
  int n = (int)(idx / T), tt = (int)(idx % T);
  double v = 0.0;
  if (tt < ntri_batch) {
    int64_t t = t0 + tt;
    int k1 = tri[3 * t] - l_min, k2 = tri[3 * t + 1] - l_min, k3 = tri[3 * t + 2] - l_min;
    int a = late[3 * n], b = late[3 * n + 1], c = late[3 * n + 2];
    if ((unsigned)a >= (unsigned)nbl || (unsigned)b >= (unsigned)nbl || (unsigned)c >= (unsigned)nbl) {
      v = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      const double *qa = q + (int64_t)a * L, *qb = q + (int64_t)b * L, *qc = q + (int64_t)c * L;
      double s = qa[k1] * (qb[k2] * qc[k3] + qc[k2] * qb[k3]) + qb[k1] * (qa[k2] * qc[k3] + qc[k2] * qa[k3]) +
                 qc[k1] * (qa[k2] * qb[k3] + qb[k2] * qa[k3]);
      v = z[t] * s;
    }
  }
  Yb[idx] = v;
}

// ---- scan helpers --------------------------------------------------------
size_t scan_tmp_bytes(int64_t n) {
  size_t b = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, b, (const int64_t *)nullptr, (int64_t *)nullptr, n);
  return b;
}
cudaError_t scan_exclusive_i64(void *tmp, size_t tmp_bytes, const int64_t *in, int64_t *out,
                               int64_t n, cudaStream_t st) {
  return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, in, out, n, st);
}

}  // namespace modal
