/*
 * modal.h -- C ABI of libmodal, a GB300 (sm_103a) implementation of the
 * Modal Gamma' projection of arXiv 1503.08809 (Briggs, Pennycook,
 * Fergusson, Jaykka, Shellard): the matrix that projects primordial modes
 * (p,r,s), carried through the radial integral by q~_p(l,x), onto late-time
 * CMB modes (a,b,c) over the triangle- and parity-bounded (l1,l2,l3) domain
 * weighted by (l1 l2 l3; 0 0 0)^2.
 *
 * Conventions (every call):
 *  - Arrays are row-major and contiguous.  Unless marked "host", a pointer
 *    is a DEVICE pointer owned by the caller; the library never frees it.
 *  - l runs over the dense range l_min..l_max (L = l_max - l_min + 1).
 *    The paper's sums start at l = 2 (Eq. 3D), so l_min = 2 is the usual
 *    choice; any l_min >= 0 is accepted.
 *  - Calls are asynchronous on `stream` (NULL = legacy default stream)
 *    unless documented otherwise.  The handle owns all scratch memory
 *    (grown on demand with cudaMalloc, released by modal_handle_destroy);
 *    concurrent calls on one handle are not allowed.
 *  - Every call returns a status code (MODAL_OK = 0).  On error nothing is
 *    aborted or thrown; modal_last_error() gives a one-line reason.
 *  - Gamma'[n][n'] is FP64 with rows n = late-time modes and columns
 *    n' = primordial modes; it includes the 1/(48 pi) prefactor of Eq. 2D.
 */
#ifndef MODAL_H
#define MODAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* same type as cudaStream_t */
typedef struct CUstream_st *modal_stream_t;

/* status codes */
#define MODAL_OK 0
#define MODAL_EINVAL 1        /* bad argument (null pointer, size, mode index, ...) */
#define MODAL_ENOMEM 2        /* device allocation for the handle's scratch failed */
#define MODAL_ECUDA 3         /* a CUDA runtime/launch error (message has the CUDA text) */
#define MODAL_ETIMEOUT 4      /* a bounded device-side wait gave up */
#define MODAL_EUNSUPPORTED 5  /* valid request the library or the device cannot serve */

/* arithmetic of the separable path (modal_opts.precision) */
#define MODAL_PREC_FP64 0        /* FP64 everywhere (CUDA cores) */
#define MODAL_PREC_FP32 1        /* FP32 products, FP32 sums over short chunks,
                                    FP64 accumulation of the chunk sums */
#define MODAL_PREC_OZAKI_BF16 2  /* tcgen05 tensor cores: operands split into
                                    exponent-aligned BF16 slices, exact FP32
                                    chunk sums, FP64 accumulation */
#define MODAL_PREC_TF32 3        /* l contraction on tcgen05 in TF32 (kind::tf32,
                                    one product, FP32 accumulation); triple
                                    product of the FP64 M as MODAL_PREC_OZAKI_BF16
                                    (exact slicing: the error is the l
                                    contraction's) */
#define MODAL_PREC_BF16X3 4      /* l contraction on tcgen05 with BF16 hi/lo
                                    operands, hi hi' + hi lo' + lo hi' (FP32
                                    accumulation); triple product as for TF32 */

/* radial quadrature (modal_x_weights) */
#define MODAL_XW_TRAPEZOID 0  /* trapezium rule (Section 3.2.4), times x^2 */
#define MODAL_XW_HERMITE 1    /* local Hermite-cubic rule (Section 3.2.4), times x^2 */

/* weights of the direct sum (modal_project_direct) */
#define MODAL_W_EXACT_3J 0       /* exact (l1 l2 l3;000)^2: triangle + parity */
#define MODAL_W_SMOOTH_GOSPER 1  /* 1/2 x Gosper form, triangle only (sparse grids) */

typedef struct modal_handle modal_handle;

/* One projection problem (Eq. 3D / Eq. 2D / Eq. legendre).  The struct itself
 * lives in host memory; its array members are device pointers. */
typedef struct modal_problem {
  int32_t l_min, l_max;       /* dense l range of the tables */
  int32_t nb_late, nb_prim;   /* sizes of the late-time and primordial 1D bases */
  int32_t n_x;                /* radial points */
  int32_t n_late, n_prim;     /* number of late / primordial 3D modes */
  int32_t reserved0;
  const double *q;            /* [nb_late][L]       q_a(l)              (Eq. 3D) */
  const double *qt;           /* [n_x][nb_prim][L]  q~_p(l, x)           (Eq. 3D) */
  const double *w_l;          /* [L] (2l+1)/(v_l sqrt(C_l))        (Eq. legendre) */
  const double *x_w;          /* [n_x] radial weights incl. x^2 (modal_x_weights) */
  const int32_t *late_modes;  /* [n_late][3] index triples (a,b,c), any order,
                                 each < nb_late (Appendix A's n -> ijk map) */
  const int32_t *prim_modes;  /* [n_prim][3] index triples (p,r,s), each < nb_prim */
} modal_problem;

typedef struct modal_opts {
  int32_t n_mu;              /* GL order; 0 = ceil((3 l_max + 1)/2), the smallest
                                order exact for P_l1 P_l2 P_l3 (Section 2.2) */
  int32_t precision;         /* MODAL_PREC_* */
  int32_t allow_inexact_gl;  /* nonzero: accept n_mu below that bound */
  int32_t x_chunk;           /* radial points per streamed chunk; 0 = automatic */
  double *error_estimate;    /* optional, modal_project_separable only: device
                                [n_late][n_prim] output (overwritten) of the
                                same projection with every M replaced by |M|
                                and every weight by its magnitude, i.e.
                                1/(48 pi) sum_x |W_x| sum_j om_j sum of the six
                                |products| -- the scale of the rounding error
                                of each entry; |error| <= tol * estimate is
                                the conditioned entrywise check.  Costs one
                                more triple product.  NULL: not computed. */
} modal_opts;

/* ---- handle ------------------------------------------------------------ */
int modal_handle_create(modal_handle **out);
int modal_handle_destroy(modal_handle *h);
/* One-line reason of the last failing call on h (h may be NULL: last
 * failure of modal_handle_create on this thread).  Never NULL. */
const char *modal_last_error(const modal_handle *h);
/* Device scratch bytes modal_project_separable / _backward will hold for this
 * problem and options (host pointers; no device work). */
int modal_workspace_size(const modal_problem *prob, const modal_opts *opts,
                         int for_backward, size_t *bytes);
/* Pre-grow the handle's scratch to at least `bytes` (call before capturing a
 * CUDA graph so that no allocation happens during capture). */
int modal_handle_reserve(modal_handle *h, size_t bytes);

/* Waits for the work of earlier calls on this handle that carries a device
 * status word and returns MODAL_ETIMEOUT if any bounded device-side wait of
 * the tensor-core kernels gave up, MODAL_EUNSUPPORTED if the tensor-core form
 * met values outside its exponent range (|M| >= 1e37 or sqrt(om W)|M| >= 1e18;
 * use MODAL_PREC_FP64 then) -- in both cases the results are not valid --
 * and MODAL_OK otherwise.  Kernels never trap or spin forever: each wait on an
 * mbarrier is bounded (default ~2 s of SM clock) and on give-up the CTA
 * stops issuing work, waits for its own copies in flight, frees its tensor
 * memory and returns. */
int modal_handle_status(modal_handle *h);
/* Tunables of the tensor-core form for later calls on this handle.
 * MODAL_OPT_TC_TRIPLE_FUSED: 0 (default) writes the BF16 slices of the Y
 *   operand of the triple product to device memory and runs a TMA-fed GEMM;
 *   1 forms Y in shared memory inside the GEMM (no Y traffic through HBM);
 *   2 does so with sixteen warps from a TMA-staged tile of M~ rows (bases of
 *   up to ~21 functions; larger ones use 0).  All give the same results to
 *   rounding; 0 is the fastest at the sizes measured.
 * MODAL_OPT_TC_SPLIT_K: K splits of the triple GEMM (0 = automatic): of the
 *   shared-memory variants, and (1 .. 4) of the one-CTA-per-tile form, whose
 *   automatic choice models the waves of tiles on the SMs.
 * MODAL_OPT_TC_PAIR: 1 runs the triple-product GEMM of MODAL_OPT_TC_TRIPLE_FUSED = 0
 *   on CTA pairs (clusters of two, 2-SM tcgen05 MMA with M = 256: each SM
 *   reads half of the B operand); 0 on single CTAs.  Same results to rounding.
 * MODAL_OPT_TC_QUEUE: 1 runs that GEMM as a persistent kernel (one CTA per
 *   SM) whose CTAs take work items -- (G tile, range of exact K chunks) --
 *   from a device queue in order of decreasing modelled cost; tiles are split
 *   into K ranges (summed with FP64 atomics) when there are fewer than two per
 *   SM.  0: one CTA per tile.  Same results to rounding.
 * MODAL_OPT_TC_AUTOTUNE: 1 (default): the first batched call for a problem
 *   set times the tensor-core triple GEMM's tile shapes -- one CTA per tile,
 *   or the queue form with column tiles of at most 128 or 64 and with or
 *   without K splits -- on one radial chunk of the first problem of each
 *   bucket (l_max in steps of 250, both basis sizes, n_x in steps of 100)
 *   that has no choice yet, keeps the fastest per bucket on the handle and
 *   blocks until done; later calls (batched or single) of a bucket use it.
 *   0: no timing, the other options decide (and the choices are dropped).
 * MODAL_OPT_TC_OVERLAP: n > 0 runs the Y pass of each radial chunk on a
 *   second stream beside the previous chunk's GEMM, which then runs as the
 *   queue form on all but n SMs (two scratch sets; single-problem calls
 *   without error_estimate; implies MODAL_OPT_TC_QUEUE).  0 (default): off.
 * MODAL_OPT_TC_OVERLAP_TAIL: 1 (default) runs the operand and Y passes of
 *   each radial chunk on a second stream beside the previous chunk's GEMM,
 *   which runs one CTA per tile (or K range of one) on a high-priority
 *   stream: the passes take the SMs that the GEMM's last wave leaves idle
 *   (two scratch sets; single-problem calls without error_estimate and
 *   with the default GEMM form).  0: one stream.  Same results to rounding.
 * MODAL_OPT_DIRECT_TENSOR: 1 runs the Gamma' update of modal_project_direct
 *   (Gamma' += Y^T diag(z) X over each batch of triples, the reduction of
 *   Eq. 3D) on the tensor cores with exponent-aligned BF16 slices (errors of
 *   ~1e-10 of max|Gamma'| instead of FP64 rounding; the radial integrals X
 *   stay FP64); 2 also forms the radial integrals there (triples grouped by
 *   (l2, l3): one GEMM of the grid's q~ rows with that pair's products
 *   W_x q~_u(l2) q~_v(l3) per pair, and the l1 sums of each pair before a
 *   GEMM over pairs; bases of up to 32 functions on either side, larger
 *   ones run as 1).  The call's status then also covers those GEMMs'
 *   bounded waits and the exponent range of their operands
 *   (modal_handle_status).  0 (default): FP64 throughout.
 * MODAL_OPT_BATCH_STREAMS: concurrent streams of modal_project_separable_batched
 *   (1 .. 8), or 0 (default): the first call for a problem set captures one
 *   graph each for 1, 2, 4 and 8 streams (as far as their scratch fits),
 *   replays each twice, keeps the fastest and blocks until that is done. */
#define MODAL_OPT_TC_TRIPLE_FUSED 1
#define MODAL_OPT_TC_SPLIT_K 2
#define MODAL_OPT_BATCH_STREAMS 3
#define MODAL_OPT_TC_PAIR 4
#define MODAL_OPT_TC_QUEUE 5
#define MODAL_OPT_TC_AUTOTUNE 6
#define MODAL_OPT_TC_OVERLAP 7
#define MODAL_OPT_DIRECT_TENSOR 8
#define MODAL_OPT_TC_OVERLAP_TAIL 9
int modal_handle_set_option(modal_handle *h, int32_t option, int64_t value);

/* Bound (in SM clock cycles) of those device-side waits for later calls on
 * this handle; 0 restores the default.  A tiny bound makes the waits give up
 * on purpose (used by the tests of the status path). */
int modal_handle_set_wait_limit(modal_handle *h, int64_t cycles);

/* Opt-in per-kernel timing: while enabled, the library records a CUDA event
 * pair on the call's stream around each kernel it launches (negligible
 * overhead; no synchronisation at record time).  modal_profile_read waits
 * for the recorded events, then reports per kernel name the launch count and
 * the summed device time since the last reset, and clears the records.
 * names: host [max_entries][32] chars; launches, total_ms: host [max_entries]. */
int modal_profile_enable(modal_handle *h, int32_t enable);
int modal_profile_read(modal_handle *h, int32_t max_entries, char *names, int64_t *launches,
                       double *total_ms, int32_t *n_out);

/* ---- individual steps of the separable path ----------------------------- */

/* Gauss-Legendre nodes (ascending) and weights of order n_mu, for the mu
 * integral of Eq. 2D (Section 2.2: library nodes were not accurate enough,
 * so the nodes are refined in double-double and rounded once to FP64).
 * mu, om: device [n_mu].  1 <= n_mu <= 6400 (MODAL_EUNSUPPORTED above). */
int modal_gl_nodes(modal_handle *h, int32_t n_mu, double *mu, double *om,
                   modal_stream_t stream);

/* Legendre table with the l weight folded in (the `factor` array of the
 * Modal2D listing, Section 3.1): A[j][l - l_min] = w_l P_l(mu_j) for
 * l = l_min..l_max, by the three-term recurrence in FP64.
 * mu: device [n_mu]; w_l: device [L] or NULL (then w_l = 1); A: device [n_mu][L]. */
int modal_legendre_table(modal_handle *h, int32_t n_mu, const double *mu, int32_t l_min,
                         int32_t l_max, const double *w_l, double *A, modal_stream_t stream);

/* Radial weights W_x of "int r^2 dr" (Eq. 3D), including x^2 (Section 3.2.4).
 * x: device [n_x] strictly increasing; w: device [n_x]. */
int modal_x_weights(modal_handle *h, int32_t kind, int32_t n_x, const double *x, double *w,
                    modal_stream_t stream);

/* l contraction of Eq. legendre for every (x, mu_j) slice:
 *   M[x][j][a][p] = sum_l A[j][l] q_a(l) q~_p(l, x),   A from modal_legendre_table.
 * A: device [n_mu][L]; M: device [n_x][n_mu][nb_late][nb_prim] FP64.
 * precision: MODAL_PREC_FP64 (CUDA cores), MODAL_PREC_OZAKI_BF16 (tcgen05
 * with exponent-aligned BF16 slices; ~1e-11 normwise), MODAL_PREC_TF32 or
 * MODAL_PREC_BF16X3 (tcgen05 with FP32 accumulation; ~1e-3 and ~1e-5).
 * (prob->late_modes/prim_modes/x_w are not used.) */
int modal_contract_l(modal_handle *h, const modal_problem *prob, int32_t n_mu,
                     const double *A, int32_t precision, double *M, modal_stream_t stream);

/* ---- the projection ------------------------------------------------------ */

/* Separable projection, Eq. 2D (Section 2.2):
 *   Gamma'[n][n'] = 1/(48 pi) sum_x W_x sum_j om_j perm3(M(x, mu_j)[n, n'])
 * where perm3 is the permanent of the 3x3 block of M picked by the late
 * triple (rows) and the primordial triple (columns) -- the six products of
 * the Modal2D listing.  gamma: device [n_late][n_prim] FP64 (overwritten).
 * Exact (up to rounding) when n_mu >= (3 l_max + 1)/2; smaller n_mu is
 * rejected with MODAL_EINVAL unless opts->allow_inexact_gl. opts may be NULL
 * (FP64, automatic n_mu).  Stream-ordered, no host synchronisation; a call
 * that runs passes on the handle's own streams (MODAL_OPT_TC_OVERLAP_TAIL)
 * forks from and joins the caller's stream with events, so the call can be
 * captured in a CUDA graph once the handle has served a call of the same
 * sizes (its scratch is then allocated). */
int modal_project_separable(modal_handle *h, const modal_problem *prob,
                            const modal_opts *opts, double *gamma, modal_stream_t stream);

/* Direct (non-separable) projection, Eq. 3D (Section 2.1), on a multipole
 * grid: the sum over sorted triples l1 <= l2 <= l3 from l_grid (device [n_grid],
 * strictly increasing, inside [l_min, l_max]) with weight
 *   mult(l) * dw1 dw2 dw3 * w_l1 w_l2 w_l3 * H(l) / (144 pi)
 * times (sum over the 6 assignments of q_a q_b q_c) times (sum_x W_x times the
 * 6 assignments of q~_p q~_r q~_s); mult = number of distinct orderings of
 * (l1,l2,l3) (6, 3 or 1).  H = exact 3j^2 (MODAL_W_EXACT_3J) or 1/2 x the
 * Gosper form with the triangle condition only (MODAL_W_SMOOTH_GOSPER).
 * l_dw: device [n_grid] multipoles represented by each grid point (1 on a
 * dense grid; NULL = all 1).  On a dense grid with EXACT weights this equals
 * modal_project_separable.  gamma: device [n_late][n_prim] (overwritten).
 * Stream-ordered, no host synchronisation: the triples are counted on the
 * device and processed in batches sized on the host from the bound
 * C(n_grid + 2, 3); batches past the true count do no work.  The call can be
 * captured in a CUDA graph once the handle has served a call with the same
 * n_grid and sizes (its scratch is then allocated). */
int modal_project_direct(modal_handle *h, const modal_problem *prob, const int32_t *l_grid,
                         const double *l_dw, int32_t n_grid, int32_t weight_mode,
                         double *gamma, modal_stream_t stream);

/* Adjoint of modal_project_separable (not in the paper; it follows from
 * Eq. 2D and Eq. legendre): given dL_dgamma = dL/dGamma' (device
 * [n_late][n_prim]) writes dL/dq~ (device [n_x][nb_prim][L], overwritten)
 * and, if dL_dq is not NULL, dL/dq (device [nb_late][L], overwritten).
 * M slices are recomputed, not stored.  opts as for the forward call:
 * MODAL_PREC_FP64 and MODAL_PREC_FP32 run on CUDA cores;
 * MODAL_PREC_OZAKI_BF16 runs the three contractions on tcgen05 with the
 * forward's exact slicing -- dL/dM as one GEMM per radial chunk over the
 * 2 x 2 minors of the permanent (dL/dM_xy = sum over the minors' rows
 * (a <= b, {u, v}) of Gfull[row][(x, y)] w (M_au M_bv + M_av M_bu), Gfull
 * collecting dL/dGamma' / (48 pi) over the nine positions of (x, y) in each
 * mode pair), then dL/dq~ and dL/dq -- and reports device-side status
 * through modal_handle_status; TF32 and BF16X3 use the FP32 adjoint. */
int modal_project_backward(modal_handle *h, const modal_problem *prob, const modal_opts *opts,
                           const double *dL_dgamma, double *dL_dqt, double *dL_dq,
                           modal_stream_t stream);

/* Many independent problems of uneven size in one call (host array `probs`
 * of n problem descriptors, host array `gammas` of n device outputs).  Each
 * result equals modal_project_separable on that problem with these opts.
 * The problems are spread over S concurrent streams (largest first, each to
 * the least loaded stream; each stream has its own scratch) so that small
 * problems fill the GPU side by side, and the launches of the whole batch
 * are captured once into one CUDA graph, cached on the handle under the
 * problem set (descriptors, pointers, opts, tunables) and replayed on
 * `stream` by later calls with the same set; the data may change between
 * calls, the pointers and sizes may not.  S comes from
 * MODAL_OPT_BATCH_STREAMS; by default the first call for a set times the
 * candidates and blocks until done.  Scratch growth on the handle drops the
 * cached graphs. */
int modal_project_separable_batched(modal_handle *h, int32_t n, const modal_problem *probs,
                                    const modal_opts *opts, double *const *gammas,
                                    modal_stream_t stream);

/* ---- the full Gamma (Appendix A) ------------------------------------------ */

/* Gram matrix of the late basis, <Q_n, Q_r> with the inner product of
 * Appendix A (weight (h_l1l2l3 / v_l1 v_l2 v_l3)^2 over all l triples):
 *   gram[n][r] = 1/(144 pi) sum_{l1,l2,l3} w_l1 w_l2 w_l3 (l1 l2 l3; 0 0 0)^2
 *                 (sum of the 6 assignments of q_a q_b q_c) (same for r)
 * with w_l = w_gram[l - l_min], which for the paper's inner product is
 * (2l+1)/v_l^2 = (2l+1)^(2/3).  It is the separable projection (Eq. 2D) of a
 * problem whose projected basis is q itself at one radial point of unit
 * weight and whose primordial modes are the late modes, so it runs on the
 * same kernels and honours opts (precision, n_mu; error_estimate receives the
 * symmetrised magnitude form).  Reads prob's l range, nb_late, q, n_late and
 * late_modes; ignores qt, w_l, x_w and the primordial side.  w_gram: device
 * [L].  gram: device [n_late][n_late] (overwritten), symmetrised as
 * (G + G^T)/2.  Stream-ordered, no host synchronisation. */
int modal_gram(modal_handle *h, const modal_problem *prob, const double *w_gram,
               const modal_opts *opts, double *gram, modal_stream_t stream);

/* x = gram^{-1} rhs by a Cholesky factorisation gram = L L^T (FP64, blocks of
 * 64) and two triangular solves: with gram from modal_gram and rhs = Gamma'
 * from modal_project_separable (or _direct), x is the full
 *   Gamma_nm = sum_r <Q_n, Q_r>^{-1} <Q_r, Q~_m>           (Appendix A).
 * gram: device [n][n] row-major, only entries i >= j are read (not
 * modified).  rhs, x: device [n][m] row-major; x may be rhs (solved in
 * place) but not gram.  info: device int32 or NULL; it receives 0, or k > 0
 * if the k-th pivot is not above n 2^-52 times gram[k-1][k-1] or is not a
 * number: the leading minor of order k is not positive definite, or is
 * singular to working precision (e.g. a mode listed twice) -- then x is
 * filled with NaN.  m = 0 factors only (info still set).  The factor lives in the handle's scratch.  Stream-ordered, no
 * host synchronisation: read info after the stream. */
int modal_gram_solve(modal_handle *h, int32_t n, int32_t m, const double *gram, const double *rhs,
                     double *x, int32_t *info, modal_stream_t stream);

/* Allocation-free form of modal_project_separable, for callers that cannot
 * allocate device memory: programs that hand all of a GPU's memory to their
 * own allocator or budget, plugins whose host forbids cudaMalloc, and
 * latency-critical loops where cudaMalloc (which may synchronise the device)
 * is not acceptable.  The paper has no counterpart; this is an interface
 * convenience.
 *  - Same problem, opts and output as modal_project_separable, but no handle:
 *    it calls no cudaMalloc, cudaFree or allocating library routine.
 *  - Scratch lives in a fixed 48 MiB device array compiled into the library;
 *    every GPU that loads the library holds it until the process exits.
 *    Radial points are streamed in the largest chunk (at most opts->x_chunk
 *    when that is set) whose scratch fits, so a caller's x_chunk may be
 *    reduced; problems that do not fit even one radial point at a time are
 *    rejected with MODAL_EINVAL and a message giving the bytes needed; e.g.
 *    20-function bases (the 52 MB triple-product table alone) do not fit.
 *  - precision: MODAL_PREC_FP64 or MODAL_PREC_FP32 (the tensor-core form
 *    needs more scratch than the fixed buffer).
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it with the id of the device's current
 *    context; a call that finds a different context (after cudaDeviceReset,
 *    or on a thread without one) looks it up again.  Make the first call on a
 *    device, and the first after a reset, before any stream capture begins.
 *  - All calls share the one buffer and it keeps the last call's contents
 *    (everything a call reads is written first).  Calls that overlap on the
 *    GPU -- on different streams, or from different threads, without
 *    ordering between them -- race on it: order them (one stream, or events).
 *  - Errors: status codes as elsewhere; modal_last_error(NULL) gives the reason. */
int modal_project_separable_noalloc(const modal_problem *prob, const modal_opts *opts, double *gamma,
                                    modal_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MODAL_H */
