/*
 * modal_oracle.c -- plain, slow, obviously-correct CPU oracle for the Modal
 * Gamma' projection of Briggs et al., "Separable projection integrals for
 * higher-order correlators of the cosmic microwave sky" (arXiv 1503.08809).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library under paper_1503_08809_gb300/) never calls it, and the two
 * share no code, headers, tables or constants.
 *
 * Everything is double precision; the Gauss-Legendre nodes and the 3j
 * product form use long double because Section 2.2 warns that ordinary
 * library nodes are not accurate enough for the separable form.
 *
 * Conventions shared with the callers (plain data, not arithmetic):
 *   l runs over the dense range l_min..l_max, L = l_max - l_min + 1;
 *   q  [nbl][L]       late-time 1D basis q_a(l)                    (Eq. 3D)
 *   qt [nx][nbp][L]   projected primordial basis q~_p(l, x)        (Eq. 3D)
 *   wl [L]            (2l+1)/(v_l sqrt(C_l))                       (Eq. legendre)
 *   xw [nx]           radial quadrature weights including x^2      (Eq. 3D, r^2 dr)
 *   late [nlate][3], prim [nprim][3]: index triples of the modes n -> (i,j,k)
 *                     (Appendix A, the n -> ijk map)
 *   gamma [nlate][nprim]  row n = late mode, column n' = primordial mode.
 *
 * parity status: every function here is pinned by tests/test_oracle_pins.py
 * (closed forms, exact rationals, brute force, identities).  oracle_direct in
 * SMOOTH (Gosper) weight mode is pinned to its formula (a literal cube sum on
 * a small grid); its agreement with the dense sum on sparse grids is an
 * approximation, measured but not pinned.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Wigner 3j symbol (l1 l2 l3; 0 0 0)^2.                                     */
/* Section 2.1 (after Eq. weight-function): zero unless the l_i form a       */
/* triangle and l1+l2+l3 is even; otherwise it has an exact factorial        */
/* expression.  With L = l1+l2+l3 = 2g that expression is                    */
/*   (2g-2l1)!(2g-2l2)!(2g-2l3)!/(2g+1)! * [g!/((g-l1)!(g-l2)!(g-l3)!)]^2.    */
/* Writing (2n)!/(n!)^2 = 4^n c_n with c_n = prod_{k=1..n} (1 - 1/(2k)), the   */
/* powers of four cancel and                                                  */
/*   3j^2 = c_{g-l1} c_{g-l2} c_{g-l3} / ((2g+1) c_g),                        */
/* a product of factors in (0,1] that cannot overflow.                        */
/* ------------------------------------------------------------------------ */
static ld c_half_binom(int n) {
  ld c = 1.0L;
  for (int k = 1; k <= n; ++k) c *= 1.0L - 1.0L / (2.0L * (ld)k);
  return c;
}

double oracle_threej000_sq(int l1, int l2, int l3) {
  if (l1 < 0 || l2 < 0 || l3 < 0) return 0.0;
  int L = l1 + l2 + l3;
  if (L & 1) return 0.0;                                   /* parity condition */
  if (l3 > l1 + l2 || l1 > l2 + l3 || l2 > l1 + l3) return 0.0; /* triangle */
  int g = L / 2;
  ld v = c_half_binom(g - l1) * c_half_binom(g - l2) * c_half_binom(g - l3);
  v /= (ld)(2 * g + 1) * c_half_binom(g);
  return (double)v;
}

/* Same value from a precomputed table c[n], n <= nmax (used by the direct
 * sum so that each triple costs O(1)). */
static double threej_tab(const ld *c, int l1, int l2, int l3) {
  int L = l1 + l2 + l3;
  if (L & 1) return 0.0;
  if (l3 > l1 + l2 || l1 > l2 + l3 || l2 > l1 + l3) return 0.0;
  int g = L / 2;
  return (double)(c[g - l1] * c[g - l2] * c[g - l3] / ((ld)(2 * g + 1) * c[g]));
}

/* Gosper approximation of the same quantity (Section 2.1, the h^2 formula
 * after Eq. weight-function).  With L = l1+l2+l3, L_i = L - 2 l_i the paper
 * gives h^2 ~ (1/(2 pi^2)) prod(2l_i+1) (L+1/3)/((L+1) prod(L_i+1/3))
 *             * sqrt(prod(L_i+1/6)/(L+1/6)),
 * and h^2 = prod(2l_i+1)/(4 pi) * 3j^2 (Eq. weight-function), so
 * 3j^2 ~ (2/pi) (L+1/3)/((L+1) prod(L_i+1/3)) sqrt(prod(L_i+1/6)/(L+1/6)).
 * Only the triangle condition is applied here; parity is left to the
 * caller. */
double oracle_gosper_threej000_sq(int l1, int l2, int l3) {
  if (l3 > l1 + l2 || l1 > l2 + l3 || l2 > l1 + l3) return 0.0;
  double L = (double)(l1 + l2 + l3);
  double L1 = L - 2.0 * l1, L2 = L - 2.0 * l2, L3 = L - 2.0 * l3;
  double v = (2.0 / ORACLE_PI) * (L + 1.0 / 3.0) /
             ((L + 1.0) * (L1 + 1.0 / 3.0) * (L2 + 1.0 / 3.0) * (L3 + 1.0 / 3.0));
  v *= sqrt((L1 + 1.0 / 6.0) * (L2 + 1.0 / 6.0) * (L3 + 1.0 / 6.0) / (L + 1.0 / 6.0));
  return v;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights (Section 2.2: the mu integral of Eq. 2D  */
/* is done by GL quadrature, exact for polynomial integrands).  Newton's     */
/* method on P_n, evaluated by the three-term recurrence                     */
/*   (k+1) P_{k+1} = (2k+1) mu P_k - k P_{k-1},                              */
/* in long double; derivative P_n' = n (mu P_n - P_{n-1}) / (mu^2 - 1);      */
/* weight 2 / ((1 - mu^2) P_n'(mu)^2).  Nodes are returned ascending.        */
/* ------------------------------------------------------------------------ */
static void legendre_pair_ld(int n, ld x, ld *pn, ld *pnm1) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) { *pn = 1.0L; *pnm1 = 0.0L; return; }
  for (int k = 1; k < n; ++k) {
    ld p2 = ((ld)(2 * k + 1) * x * p1 - (ld)k * p0) / (ld)(k + 1);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

void oracle_gl_nodes(int n, double *mu, double *om) {
  const ld pi = 3.141592653589793238462643383279502884L;
  int half = (n + 1) / 2;
  for (int i = 0; i < half; ++i) {
    /* i-th largest root, classic starting guess */
    ld x = cosl(pi * ((ld)i + 0.75L) / ((ld)n + 0.5L));
    ld pn = 0, pm = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      legendre_pair_ld(n, x, &pn, &pm);
      dp = (ld)n * (x * pn - pm) / (x * x - 1.0L);
      ld dx = pn / dp;
      x -= dx;
      if (fabsl(dx) <= 4.0L * LDBL_EPSILON * fabsl(x) + 1e-300L) break;
    }
    legendre_pair_ld(n, x, &pn, &pm);
    dp = (ld)n * (x * pn - pm) / (x * x - 1.0L);
    ld w = 2.0L / ((1.0L - x * x) * dp * dp);
    /* ascending order: the largest root goes last */
    mu[n - 1 - i] = (double)x;
    om[n - 1 - i] = (double)w;
    mu[i] = (double)(-x);
    om[i] = (double)w;
  }
  if (n & 1) mu[n / 2] = 0.0; /* exact centre node for odd n */
}

/* P_0..P_lmax at one mu (double, forward recurrence). */
void oracle_legendre_row(int lmax, double mu, double *P) {
  P[0] = 1.0;
  if (lmax >= 1) P[1] = mu;
  for (int k = 1; k < lmax; ++k)
    P[k + 1] = ((2.0 * k + 1.0) * mu * P[k] - (double)k * P[k - 1]) / (double)(k + 1);
}

/* ------------------------------------------------------------------------ */
/* Radial weights W_x for "int r^2 dr" of Eq. 3D / Eq. 2D.                   */
/* kind 0: the trapezium rule the paper settles on (Section 3.2.4) times x^2. */
/* kind 1: the local Hermite-cubic integrator of Section 3.2.4 with the       */
/*         derivative estimate p'(r_k) = forward difference, integrated      */
/*         exactly over each interval, times x^2.  Per interval k:            */
/*   dr_k/2 (y_k + y_{k+1}) + dr_k^2/12 (D_k - D_{k+1}),  D_k = dy_k/dr_k,    */
/*         with D at the last node taken equal to the last interval's.       */
/*         The rule is linear in y, so it is a weight vector.                */
/* ------------------------------------------------------------------------ */
void oracle_x_weights(int kind, int nx, const double *x, double *w) {
  for (int k = 0; k < nx; ++k) w[k] = 0.0;
  if (nx < 2) { if (nx == 1) w[0] = 0.0; return; }
  if (kind == 0) {
    for (int k = 0; k + 1 < nx; ++k) {
      double h = x[k + 1] - x[k];
      w[k] += 0.5 * h;
      w[k + 1] += 0.5 * h;
    }
  } else {
    /* unit-response construction: W_m = integral of the rule applied to e_m */
    double *y = (double *)calloc((size_t)nx, sizeof(double));
    for (int m = 0; m < nx; ++m) {
      for (int k = 0; k < nx; ++k) y[k] = (k == m) ? 1.0 : 0.0;
      double s = 0.0;
      for (int k = 0; k + 1 < nx; ++k) {
        double h = x[k + 1] - x[k];
        double Dk = (y[k + 1] - y[k]) / h;
        double Dk1;
        if (k + 2 < nx) Dk1 = (y[k + 2] - y[k + 1]) / (x[k + 2] - x[k + 1]);
        else Dk1 = Dk;
        s += 0.5 * h * (y[k] + y[k + 1]) + h * h / 12.0 * (Dk - Dk1);
      }
      w[m] = s;
    }
    free(y);
  }
  for (int k = 0; k < nx; ++k) w[k] *= x[k] * x[k];
}

/* ------------------------------------------------------------------------ */
/* Permanent of the 3x3 block of M picked by a late triple and a primordial */
/* triple: the six products s1..s6 of the gamma_pt listing in Section 3.1.  */
/* ------------------------------------------------------------------------ */
static double perm3(const double *M, int nbp, const int *r, const int *c) {
  double m00 = M[r[0] * nbp + c[0]], m01 = M[r[0] * nbp + c[1]], m02 = M[r[0] * nbp + c[2]];
  double m10 = M[r[1] * nbp + c[0]], m11 = M[r[1] * nbp + c[1]], m12 = M[r[1] * nbp + c[2]];
  double m20 = M[r[2] * nbp + c[0]], m21 = M[r[2] * nbp + c[1]], m22 = M[r[2] * nbp + c[2]];
  double s1 = m00 * m11 * m22;
  double s2 = m00 * m12 * m21;
  double s3 = m01 * m10 * m22;
  double s4 = m01 * m12 * m20;
  double s5 = m02 * m10 * m21;
  double s6 = m02 * m11 * m20;
  return s1 + s2 + s3 + s4 + s5 + s6;
}

/* The same six products in magnitude: the summation-error scale of perm3. */
static double perm3_abs(const double *M, int nbp, const int *r, const int *c) {
  double m[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m[i][j] = fabs(M[r[i] * nbp + c[j]]);
  return m[0][0] * m[1][1] * m[2][2] + m[0][0] * m[1][2] * m[2][1] + m[0][1] * m[1][0] * m[2][2] +
         m[0][1] * m[1][2] * m[2][0] + m[0][2] * m[1][0] * m[2][1] + m[0][2] * m[1][1] * m[2][0];
}

/* P_{ii'}(x, mu) of Eq. legendre for every (a, p) flagged in need_a x need_p:
 *   M[a][p] = sum_l wl[l] P_l(mu) q_a(l) q~_p(l, x). */
static void legendre_table_M(int l_min, int L, int nbl, int nbp, const double *q,
                             const double *qt_x, const double *wl, const double *P,
                             const unsigned char *need_a, const unsigned char *need_p,
                             double *M) {
  for (int a = 0; a < nbl; ++a) {
    for (int p = 0; p < nbp; ++p) {
      double s = 0.0;
      if (need_a[a] && need_p[p]) {
        const double *qa = q + (size_t)a * L;
        const double *qp = qt_x + (size_t)p * L;
        for (int l = 0; l < L; ++l) s += wl[l] * P[l_min + l] * qa[l] * qp[l];
      }
      M[a * nbp + p] = s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Separable projection, Eq. 2D with Eq. legendre (Section 2.2):             */
/*   Gamma'_{nn'} = 1/(48 pi) int r^2 dr int dmu                             */
/*                  (P_{ii'} P_{jj'} P_{kk'} + 5 perms),                      */
/* the mu integral by the caller's GL rule, done first for each x (the      */
/* paper requires mu before r), then the radial sum with weights xw.         */
/* Only the (a, p) pairs used by the given mode lists are formed, so a       */
/* caller may ask for a few rows/columns of a large problem.                  */
/* ------------------------------------------------------------------------ */
static void separable_impl(int l_min, int l_max, int nbl, int nbp, int nx,
                           const double *q, const double *qt, const double *wl,
                           const double *xw, int nmu, const double *mu, const double *om,
                           int nlate, const int *late, int nprim, const int *prim,
                           double *gamma, int magnitudes) {
  int L = l_max - l_min + 1;
  unsigned char *need_a = (unsigned char *)calloc((size_t)nbl, 1);
  unsigned char *need_p = (unsigned char *)calloc((size_t)nbp, 1);
  for (int n = 0; n < nlate * 3; ++n) need_a[late[n]] = 1;
  for (int n = 0; n < nprim * 3; ++n) need_p[prim[n]] = 1;
  double *inner = (double *)calloc((size_t)nlate * nprim, sizeof(double));
  double *Mall = (double *)malloc(sizeof(double) * (size_t)nmu * nbl * nbp);
  double *Pall = (double *)malloc(sizeof(double) * (size_t)nmu * (l_max + 1));
  for (size_t i = 0; i < (size_t)nlate * nprim; ++i) gamma[i] = 0.0;
  for (int j = 0; j < nmu; ++j) oracle_legendre_row(l_max, mu[j], Pall + (size_t)j * (l_max + 1));
  for (int x = 0; x < nx; ++x) {
    const double *qt_x = qt + (size_t)x * nbp * L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < nmu; ++j)
      legendre_table_M(l_min, L, nbl, nbp, q, qt_x, wl, Pall + (size_t)j * (l_max + 1),
                       need_a, need_p, Mall + (size_t)j * nbl * nbp);
    /* mu integral for this x: inner[n][n'] = sum_j om_j perm(M(x, mu_j)) */
#pragma omp parallel for schedule(static)
    for (int n = 0; n < nlate; ++n) {
      for (int m = 0; m < nprim; ++m) {
        double s = 0.0;
        for (int j = 0; j < nmu; ++j)
          s += magnitudes ? fabs(om[j]) * perm3_abs(Mall + (size_t)j * nbl * nbp, nbp, late + 3 * n, prim + 3 * m)
                          : om[j] * perm3(Mall + (size_t)j * nbl * nbp, nbp, late + 3 * n, prim + 3 * m);
        inner[(size_t)n * nprim + m] = s;
      }
    }
    const double wx = magnitudes ? fabs(xw[x]) : xw[x];
    for (size_t i = 0; i < (size_t)nlate * nprim; ++i) gamma[i] += wx * inner[i];
  }
  const double pref = 1.0 / (48.0 * ORACLE_PI);
  for (size_t i = 0; i < (size_t)nlate * nprim; ++i) gamma[i] *= pref;
  free(need_a); free(need_p); free(inner); free(Mall); free(Pall);
}

void oracle_separable(int l_min, int l_max, int nbl, int nbp, int nx,
                      const double *q, const double *qt, const double *wl,
                      const double *xw, int nmu, const double *mu, const double *om,
                      int nlate, const int *late, int nprim, const int *prim,
                      double *gamma) {
  separable_impl(l_min, l_max, nbl, nbp, nx, q, qt, wl, xw, nmu, mu, om, nlate, late, nprim, prim, gamma, 0);
}

/* The same sum with every term in magnitude -- |om_j|, |W_x| and the six   */
/* |products| of P_{ii'} entries -- the scale of the rounding error of each */
/* entry of Gamma' (the conditioned entrywise check).                        */
void oracle_separable_abs(int l_min, int l_max, int nbl, int nbp, int nx,
                          const double *q, const double *qt, const double *wl,
                          const double *xw, int nmu, const double *mu, const double *om,
                          int nlate, const int *late, int nprim, const int *prim,
                          double *gamma) {
  separable_impl(l_min, l_max, nbl, nbp, nx, q, qt, wl, xw, nmu, mu, om, nlate, late, nprim, prim, gamma, 1);
}

/* ------------------------------------------------------------------------ */
/* Direct (non-separable) projection, Eq. 3D (Section 2.1), on a grid of     */
/* multipoles l_grid[0..ng-1] (strictly increasing, inside [l_min, l_max]),   */
/* each standing for l_dw[i] dense multipoles (1 on a dense grid).            */
/* Summand over the cube, with w = (2l+1)/(v sqrt C) and the inner-product    */
/* definitions of Appendix A (Q_n and Q~_n carry 1/6, h^2 carries 1/(4 pi)):  */
/*   w1 w2 w3 3j^2/(4 pi) * (1/6 sum_pi q q q) * (1/6 int r^2 dr sum_s q~q~q~) */
/* = w1 w2 w3 3j^2 / (144 pi) * Y_n * X_n'.  The summand is symmetric in the */
/* l_i, so the cube sum is the sorted (l1 <= l2 <= l3) sum weighted by the    */
/* number of distinct orderings (6, 3 or 1), as in the Modal3D listing's     */
/* l2 >= l1, l3 >= l2 loop bounds.                                            */
/* weight_mode 0 (EXACT): exact 3j^2 (zero off triangle and odd parity).     */
/* weight_mode 1 (SMOOTH): 1/2 x Gosper 3j^2, triangle only (parity averaged) */
/*   -- an approximation of the dense sum on sparse grids.                   */
/* ------------------------------------------------------------------------ */
void oracle_direct(int l_min, int l_max, int nbl, int nbp, int nx, const double *q,
                   const double *qt, const double *wl, const double *xw, int ng,
                   const int *l_grid, const double *l_dw, int weight_mode, int nlate,
                   const int *late, int nprim, const int *prim, double *gamma) {
  (void)nbl;
  int L = l_max - l_min + 1;
  int cmax = 3 * l_max / 2 + 2;
  ld *ctab = (ld *)malloc(sizeof(ld) * (size_t)(cmax + 1));
  ctab[0] = 1.0L;
  for (int k = 1; k <= cmax; ++k) ctab[k] = ctab[k - 1] * (1.0L - 1.0L / (2.0L * (ld)k));
  for (size_t i = 0; i < (size_t)nlate * nprim; ++i) gamma[i] = 0.0;
  double *X = (double *)malloc(sizeof(double) * (size_t)nprim);
  double *Y = (double *)malloc(sizeof(double) * (size_t)nlate);
  const double pref = 1.0 / (144.0 * ORACLE_PI);
  for (int i1 = 0; i1 < ng; ++i1) {
    for (int i2 = i1; i2 < ng; ++i2) {
      for (int i3 = i2; i3 < ng; ++i3) {
        int l1 = l_grid[i1], l2 = l_grid[i2], l3 = l_grid[i3];
        if (l3 > l1 + l2) break; /* triangle (sorted, so this is the only test) */
        double H;
        if (weight_mode == 0) {
          H = threej_tab(ctab, l1, l2, l3);
          if (H == 0.0) continue;
        } else {
          H = 0.5 * oracle_gosper_threej000_sq(l1, l2, l3);
        }
        int mult = (l1 == l2 && l2 == l3) ? 1 : ((l1 == l2 || l2 == l3) ? 3 : 6);
        int k1 = l1 - l_min, k2 = l2 - l_min, k3 = l3 - l_min;
        double z = pref * (double)mult * l_dw[i1] * l_dw[i2] * l_dw[i3] *
                   wl[k1] * wl[k2] * wl[k3] * H;
        /* late side: sum over the 6 assignments of (i,j,k) to (l1,l2,l3) */
#pragma omp parallel for schedule(static)
        for (int n = 0; n < nlate; ++n) {
          int a = late[3 * n], b = late[3 * n + 1], c = late[3 * n + 2];
          const double *qa = q + (size_t)a * L, *qb = q + (size_t)b * L, *qc = q + (size_t)c * L;
          Y[n] = qa[k1] * qb[k2] * qc[k3] + qa[k1] * qc[k2] * qb[k3] +
                 qb[k1] * qa[k2] * qc[k3] + qb[k1] * qc[k2] * qa[k3] +
                 qc[k1] * qa[k2] * qb[k3] + qc[k1] * qb[k2] * qa[k3];
        }
        /* primordial side: radial integral of the symmetrised product */
#pragma omp parallel for schedule(static)
        for (int m = 0; m < nprim; ++m) {
          int p = prim[3 * m], r = prim[3 * m + 1], s = prim[3 * m + 2];
          double acc = 0.0;
          for (int x = 0; x < nx; ++x) {
            const double *base = qt + (size_t)x * nbp * L;
            const double *tp = base + (size_t)p * L, *tr = base + (size_t)r * L,
                         *ts = base + (size_t)s * L;
            double v = tp[k1] * tr[k2] * ts[k3] + tp[k1] * ts[k2] * tr[k3] +
                       tr[k1] * tp[k2] * ts[k3] + tr[k1] * ts[k2] * tp[k3] +
                       ts[k1] * tp[k2] * tr[k3] + ts[k1] * tr[k2] * tp[k3];
            acc += xw[x] * v;
          }
          X[m] = acc;
        }
#pragma omp parallel for schedule(static)
        for (int n = 0; n < nlate; ++n) {
          double zy = z * Y[n];
          for (int m = 0; m < nprim; ++m) gamma[(size_t)n * nprim + m] += zy * X[m];
        }
      }
    }
  }
  free(ctab); free(X); free(Y);
}

/* ------------------------------------------------------------------------ */
/* Adjoint of oracle_separable (not in the paper; derived from Eq. 2D and    */
/* Eq. legendre).  Given gbar = dL/dGamma' [nlate][nprim]:                   */
/*   dL/dM_ap(x,mu_j) = xw_x om_j /(48 pi) sum_{n,n'} gbar[n][n']             */
/*                      sum_{i,k: late[n][i]=a, prim[n'][k]=p} perm2(minor_ik) */
/* (the derivative of a permanent w.r.t. one entry is the permanent of its  */
/* complementary 2x2 minor), then through Eq. legendre                       */
/*   dL/dq~_p(l,x) = sum_{a,j} dL/dM_ap(x,mu_j) wl P_l(mu_j) q_a(l),          */
/*   dL/dq_a(l)    = sum_{x,j,p} dL/dM_ap(x,mu_j) wl P_l(mu_j) q~_p(l,x).     */
/* dq may be NULL.                                                            */
/* ------------------------------------------------------------------------ */
void oracle_backward(int l_min, int l_max, int nbl, int nbp, int nx, const double *q,
                     const double *qt, const double *wl, const double *xw, int nmu,
                     const double *mu, const double *om, int nlate, const int *late,
                     int nprim, const int *prim, const double *gbar, double *dqt,
                     double *dq) {
  int L = l_max - l_min + 1;
  unsigned char *all_a = (unsigned char *)malloc((size_t)nbl);
  unsigned char *all_p = (unsigned char *)malloc((size_t)nbp);
  memset(all_a, 1, (size_t)nbl);
  memset(all_p, 1, (size_t)nbp);
  double *P = (double *)malloc(sizeof(double) * (size_t)(l_max + 1));
  double *M = (double *)malloc(sizeof(double) * (size_t)nbl * nbp);
  double *dM = (double *)malloc(sizeof(double) * (size_t)nbl * nbp);
  for (size_t i = 0; i < (size_t)nx * nbp * L; ++i) dqt[i] = 0.0;
  if (dq) for (size_t i = 0; i < (size_t)nbl * L; ++i) dq[i] = 0.0;
  const double pref = 1.0 / (48.0 * ORACLE_PI);
  for (int x = 0; x < nx; ++x) {
    const double *qt_x = qt + (size_t)x * nbp * L;
    for (int j = 0; j < nmu; ++j) {
      oracle_legendre_row(l_max, mu[j], P);
      legendre_table_M(l_min, L, nbl, nbp, q, qt_x, wl, P, all_a, all_p, M);
      for (int i = 0; i < nbl * nbp; ++i) dM[i] = 0.0;
      double c = pref * xw[x] * om[j];
      for (int n = 0; n < nlate; ++n) {
        const int *R = late + 3 * n;
        for (int m = 0; m < nprim; ++m) {
          const int *C = prim + 3 * m;
          double g = c * gbar[(size_t)n * nprim + m];
          if (g == 0.0) continue;
          for (int i = 0; i < 3; ++i) {
            int r0 = R[(i + 1) % 3], r1 = R[(i + 2) % 3];
            for (int k = 0; k < 3; ++k) {
              int c0 = C[(k + 1) % 3], c1 = C[(k + 2) % 3];
              double p2 = M[r0 * nbp + c0] * M[r1 * nbp + c1] + M[r0 * nbp + c1] * M[r1 * nbp + c0];
              dM[R[i] * nbp + C[k]] += g * p2;
            }
          }
        }
      }
      for (int p = 0; p < nbp; ++p) {
        double *d = dqt + ((size_t)x * nbp + p) * L;
        for (int a = 0; a < nbl; ++a) {
          double g = dM[a * nbp + p];
          if (g == 0.0) continue;
          const double *qa = q + (size_t)a * L;
          for (int l = 0; l < L; ++l) d[l] += g * wl[l] * P[l_min + l] * qa[l];
        }
      }
      if (dq) {
        for (int a = 0; a < nbl; ++a) {
          double *d = dq + (size_t)a * L;
          for (int p = 0; p < nbp; ++p) {
            double g = dM[a * nbp + p];
            if (g == 0.0) continue;
            const double *tp = qt_x + (size_t)p * L;
            for (int l = 0; l < L; ++l) d[l] += g * wl[l] * P[l_min + l] * tp[l];
          }
        }
      }
    }
  }
  free(all_a); free(all_p); free(P); free(M); free(dM);
}

/* ------------------------------------------------------------------------ */
/* The table P_{ii'}(x, mu_j) of Eq. legendre on every slice, by plain       */
/* loops: M[x][j][a][p] = sum_l wl[l] P_l(mu_j) q_a(l) q~_p(l, x).           */
/* ------------------------------------------------------------------------ */
void oracle_M(int l_min, int l_max, int nbl, int nbp, int nx, const double *q,
              const double *qt, const double *wl, int nmu, const double *mu, double *M) {
  int L = l_max - l_min + 1;
  unsigned char *all_a = (unsigned char *)malloc((size_t)nbl);
  unsigned char *all_p = (unsigned char *)malloc((size_t)nbp);
  memset(all_a, 1, (size_t)nbl);
  memset(all_p, 1, (size_t)nbp);
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < nmu; ++j) {
    double *P = (double *)malloc(sizeof(double) * (size_t)(l_max + 1));
    oracle_legendre_row(l_max, mu[j], P);
    for (int x = 0; x < nx; ++x)
      legendre_table_M(l_min, L, nbl, nbp, q, qt + (size_t)x * nbp * L, wl, P, all_a, all_p,
                       M + (((size_t)x * nmu + j) * nbl) * nbp);
    free(P);
  }
  free(all_a);
  free(all_p);
}
