// modal_abi.cu -- the extern "C" boundary of libmodal: handle, scratch,
// argument validation and the drivers that chain the kernels of the
// separable path (rows a1-a7), the direct path (a8), the adjoint (a9) and
// the batched form (a10).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda.h>

#include "common.cuh"
#include "direct.cuh"
#include "kernels.cuh"
#include "tc.cuh"
#include "backward.cuh"
#include "batch_plan.h"
#include "gram.cuh"
#include "profile.cuh"

using namespace modal;

constexpr int MAX_BATCH_STREAMS = 8;

struct modal_handle {
  int device = 0;
  int num_sms = 0;
  std::string err;
  void *slot_ptr[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t slot_bytes[4] = {0, 0, 0, 0};
  int64_t *pinned_i64 = nullptr;  // host-pinned block: a spare word, then the error words below
  int *pinned_err = nullptr;      // host-pinned copies of the tensor path's device error words
  int n_err_words = 1;            // how many of them the last call filled
  cudaEvent_t err_event = nullptr;
  bool err_pending = false;
  long long wait_cycles = TC_DEFAULT_WAIT_CYCLES;
  int opt_triple_variant = TC_TRIPLE_MATERIALISED;
  int opt_split_k = 0;
  int opt_pair = 0;               // the triple GEMM on CTA pairs (2-SM MMA)
  int opt_queue = 0;              // the triple GEMM as a persistent kernel over a work queue
  int opt_autotune = 1;           // batched calls time the triple GEMM's tile shapes per bucket
  int opt_overlap = 0;            // SMs left to the Y pass beside the queue GEMM (0: no overlap)
  int opt_direct_tensor = 0;      // the direct form's Gamma update on the tensor cores
  int opt_overlap_tail = 1;       // operand and Y passes beside the previous chunk's GEMM (its last wave)
  cudaStream_t ovl_stream = nullptr;
  cudaStream_t ovl_hi = nullptr;  // high-priority stream of the GEMMs in the tail-overlap form
  cudaEvent_t ovl_ev[6] = {};     // fork, l contraction done, side done, prep[2] / gemm[2] (below)
  cudaEvent_t ovl_prep[2] = {}, ovl_gemm[2] = {};
  cudaEvent_t ovl_prep2[2] = {};  // tail form: the second half of a chunk's Y rows is ready
  // tile shape chosen per problem bucket (tile_bucket): 0 = one CTA per tile,
  // 1 + tune = the queue form with that tile shape
  std::unordered_map<uint64_t, int> tile_choice;
  int opt_batch_streams = 0;      // 0: chosen by timing on the first call for a problem set
  Profiler prof;
  // batched calls: graphs of all launches, keyed by the problem set; the
  // capture forks onto side streams so that small problems run side by side
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side[MAX_BATCH_STREAMS] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[MAX_BATCH_STREAMS] = {};
  struct BatchGraph {
    cudaGraphExec_t exec;
    int streams;
  };
  std::unordered_map<uint64_t, BatchGraph> graphs;
  void clear_graphs() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
};

// time the launch(es) of the enclosing block when profiling is on
#define PROF(h, name, st) ProfScope _prof_scope(((h) && (h)->prof.on) ? &(h)->prof : nullptr, name, st)
#define PROFN(h, name, st, n) ProfScope _prof_scope(((h) && (h)->prof.on) ? &(h)->prof : nullptr, name, st, n)

static thread_local std::string g_err_nohandle;

static int fail(modal_handle *h, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_err_nohandle = buf;
  return code;
}

#define CK(expr)                                                                              \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess) return fail(h, MODAL_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Grow-only device scratch per slot (0: general, 1: direct-path triples,
// 2: batched problem table, 3: the Cholesky factor of modal_gram_solve).
// Growing frees the old block (cudaFree waits for the device), so pointers
// from an earlier call must not be reused.
static int ws_get(modal_handle *h, int slot, size_t bytes, void **out) {
  if (bytes == 0) bytes = 256;
  if (h->slot_bytes[slot] < bytes) {
    h->clear_graphs();  // captured graphs point into the old block
    if (h->slot_ptr[slot]) cudaFree(h->slot_ptr[slot]);
    h->slot_ptr[slot] = nullptr;
    h->slot_bytes[slot] = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MODAL_ENOMEM, "cudaMalloc(%zu bytes) for scratch failed: %s", bytes,
                  cudaGetErrorString(e));
    }
    h->slot_ptr[slot] = p;
    h->slot_bytes[slot] = bytes;
  }
  *out = h->slot_ptr[slot];
  return MODAL_OK;
}

struct Bump {
  char *p;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    T *r = reinterpret_cast<T *>(p + off);
    off += align256(sizeof(T) * (n ? n : 1));
    return r;
  }
};

static int check_handle(modal_handle *h) {
  if (!h) return fail(nullptr, MODAL_EINVAL, "null handle");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
    return fail(h, MODAL_EINVAL, "handle was created on device %d, current device is %d", h->device, dev);
  return MODAL_OK;
}

static int n_mu_exact(int l_max) { return (3 * l_max + 2) / 2; }

static int validate_problem(modal_handle *h, const modal_problem *p, bool need_modes, bool need_xw) {
  if (!p) return fail(h, MODAL_EINVAL, "null problem");
  if (p->l_min < 0 || p->l_max < p->l_min)
    return fail(h, MODAL_EINVAL, "bad l range [%d, %d]", p->l_min, p->l_max);
  if (p->nb_late < 1 || p->nb_prim < 1 || p->nb_late > 64 || p->nb_prim > 64)
    return fail(h, MODAL_EINVAL, "basis sizes must be in [1, 64] (got %d, %d)", p->nb_late, p->nb_prim);
  if (p->n_x < 0 || p->n_late < 0 || p->n_prim < 0)
    return fail(h, MODAL_EINVAL, "negative size");
  if (!p->q || !p->w_l) return fail(h, MODAL_EINVAL, "null q or w_l");
  if (p->n_x > 0 && !p->qt) return fail(h, MODAL_EINVAL, "null qt");
  if (need_xw && p->n_x > 0 && !p->x_w) return fail(h, MODAL_EINVAL, "null x_w");
  if (need_modes && ((p->n_late && !p->late_modes) || (p->n_prim && !p->prim_modes)))
    return fail(h, MODAL_EINVAL, "null mode list");
  return MODAL_OK;
}

static int resolve_opts(modal_handle *h, const modal_problem *p, const modal_opts *o, int &n_mu, int &prec,
                        int &x_chunk) {
  n_mu = (o && o->n_mu > 0) ? o->n_mu : n_mu_exact(p->l_max);
  prec = o ? o->precision : MODAL_PREC_FP64;
  x_chunk = o ? o->x_chunk : 0;
  if (o && o->n_mu < 0) return fail(h, MODAL_EINVAL, "n_mu < 0");
  if (n_mu < n_mu_exact(p->l_max) && !(o && o->allow_inexact_gl))
    return fail(h, MODAL_EINVAL,
                "n_mu = %d is below ceil((3 l_max + 1)/2) = %d: the Gauss-Legendre rule would not be exact "
                "(set allow_inexact_gl to accept)",
                n_mu, n_mu_exact(p->l_max));
  if (n_mu > 6400) return fail(h, MODAL_EUNSUPPORTED, "n_mu > 6400 (l_max > 4266) is not supported");
  if (prec < MODAL_PREC_FP64 || prec > MODAL_PREC_BF16X3) return fail(h, MODAL_EINVAL, "unknown precision %d", prec);
  if (x_chunk < 0) return fail(h, MODAL_EINVAL, "x_chunk < 0");
  return MODAL_OK;
}

extern "C" {

int modal_handle_create(modal_handle **out) {
  if (!out) return fail(nullptr, MODAL_EINVAL, "null output pointer");
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, MODAL_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return fail(nullptr, MODAL_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  modal_handle *h = new modal_handle();
  h->device = dev;
  h->num_sms = prop.multiProcessorCount;
  e = cudaMallocHost((void **)&h->pinned_i64, sizeof(int64_t) + MAX_BATCH_STREAMS * sizeof(int));
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, MODAL_ENOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
  }
  h->pinned_err = (int *)(h->pinned_i64 + 1);
  for (int i = 0; i < MAX_BATCH_STREAMS; ++i) h->pinned_err[i] = 0;
  e = cudaEventCreateWithFlags(&h->err_event, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFreeHost(h->pinned_i64);
    delete h;
    return fail(nullptr, MODAL_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
  }
  *out = h;
  return MODAL_OK;
}

int modal_handle_destroy(modal_handle *h) {
  if (!h) return MODAL_OK;
  for (int s = 0; s < 4; ++s)
    if (h->slot_ptr[s]) cudaFree(h->slot_ptr[s]);
  h->clear_graphs();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int i = 0; i < MAX_BATCH_STREAMS; ++i) {
    if (h->side[i]) cudaStreamDestroy(h->side[i]);
    if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->ovl_stream) cudaStreamDestroy(h->ovl_stream);
  if (h->ovl_hi) cudaStreamDestroy(h->ovl_hi);
  for (int i = 0; i < 6; ++i)
    if (h->ovl_ev[i]) cudaEventDestroy(h->ovl_ev[i]);
  for (int i = 0; i < 2; ++i) {
    if (h->ovl_prep[i]) cudaEventDestroy(h->ovl_prep[i]);
    if (h->ovl_prep2[i]) cudaEventDestroy(h->ovl_prep2[i]);
    if (h->ovl_gemm[i]) cudaEventDestroy(h->ovl_gemm[i]);
  }
  if (h->err_event) cudaEventDestroy(h->err_event);
  if (h->pinned_i64) cudaFreeHost(h->pinned_i64);
  tc_release(h->device);
  delete h;
  return MODAL_OK;
}

const char *modal_last_error(const modal_handle *h) {
  if (!h) return g_err_nohandle.c_str();
  return h->err.c_str();
}

int modal_profile_enable(modal_handle *h, int32_t enable) {
  if (int r = check_handle(h)) return r;
  h->prof.on = enable != 0;
  return MODAL_OK;
}

int modal_profile_read(modal_handle *h, int32_t max_entries, char *names, int64_t *launches,
                       double *total_ms, int32_t *n_out) {
  if (int r = check_handle(h)) return r;
  if (max_entries < 0 || (max_entries > 0 && (!names || !launches || !total_ms)) || !n_out)
    return fail(h, MODAL_EINVAL, "bad output arrays");
  auto m = h->prof.drain();
  int n = 0;
  for (auto &kv : m) {
    if (n >= max_entries) break;
    strncpy(names + 32 * n, kv.first.c_str(), 31);
    names[32 * n + 31] = 0;
    launches[n] = kv.second.first;
    total_ms[n] = kv.second.second;
    ++n;
  }
  *n_out = n;
  return MODAL_OK;
}

int modal_handle_status(modal_handle *h) {
  if (int r = check_handle(h)) return r;
  if (!h->err_pending) return MODAL_OK;
  cudaError_t e = cudaEventSynchronize(h->err_event);
  if (e != cudaSuccess) return fail(h, MODAL_ECUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
  h->err_pending = false;
  int word = 0;
  for (int i = 0; i < h->n_err_words; ++i) {
    word |= h->pinned_err[i];
    h->pinned_err[i] = 0;
  }
  if (word & 1) return fail(h, MODAL_ETIMEOUT, "a bounded device-side wait of the tensor-core kernels gave up");
  if (word & 2)
    return fail(h, MODAL_EUNSUPPORTED,
                "values outside the range of the tensor-core form (|M| < 1e37, sqrt(w)|M| < 1e18, "
                "|w_l P_l q| < 1e37); use MODAL_PREC_FP64");
  return MODAL_OK;
}

int modal_handle_set_option(modal_handle *h, int32_t option, int64_t value) {
  if (int r = check_handle(h)) return r;
  switch (option) {
    case MODAL_OPT_TC_TRIPLE_FUSED:
      if (value < 0 || value > 2) return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_TRIPLE_FUSED takes 0, 1 or 2");
      h->opt_triple_variant = value == 2 ? TC_TRIPLE_FUSED2 : value ? TC_TRIPLE_FUSED : TC_TRIPLE_MATERIALISED;
      return MODAL_OK;
    case MODAL_OPT_TC_SPLIT_K:
      if (value < 0 || value > 4096) return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_SPLIT_K out of range");
      h->opt_split_k = (int)value;
      return MODAL_OK;
    case MODAL_OPT_TC_PAIR:
      if (value < 0 || value > 1) return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_PAIR takes 0 or 1");
      h->opt_pair = (int)value;
      return MODAL_OK;
    case MODAL_OPT_TC_QUEUE:
      if (value < 0 || value > 1) return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_QUEUE takes 0 or 1");
      h->opt_queue = (int)value;
      return MODAL_OK;
    case MODAL_OPT_TC_AUTOTUNE:
      if (value < 0 || value > 1) return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_AUTOTUNE takes 0 or 1");
      h->opt_autotune = (int)value;
      if (!value) h->tile_choice.clear();
      return MODAL_OK;
    case MODAL_OPT_TC_OVERLAP:
      if (value < 0 || value > h->num_sms / 2)
        return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_OVERLAP takes 0 .. %d", h->num_sms / 2);
      h->opt_overlap = (int)value;
      return MODAL_OK;
    case MODAL_OPT_TC_OVERLAP_TAIL:
      if (value < 0 || value > 1) return fail(h, MODAL_EINVAL, "MODAL_OPT_TC_OVERLAP_TAIL takes 0 or 1");
      h->opt_overlap_tail = (int)value;
      return MODAL_OK;
    case MODAL_OPT_DIRECT_TENSOR:
      if (value < 0 || value > 2) return fail(h, MODAL_EINVAL, "MODAL_OPT_DIRECT_TENSOR takes 0, 1 or 2");
      h->opt_direct_tensor = (int)value;
      return MODAL_OK;
    case MODAL_OPT_BATCH_STREAMS:
      if (value < 0 || value > MAX_BATCH_STREAMS)
        return fail(h, MODAL_EINVAL, "MODAL_OPT_BATCH_STREAMS takes 0 .. %d", MAX_BATCH_STREAMS);
      h->opt_batch_streams = (int)value;
      return MODAL_OK;
    default:
      return fail(h, MODAL_EINVAL, "unknown option %d", option);
  }
}

int modal_handle_set_wait_limit(modal_handle *h, int64_t cycles) {
  if (int r = check_handle(h)) return r;
  if (cycles < 0) return fail(h, MODAL_EINVAL, "negative wait limit");
  h->wait_cycles = cycles == 0 ? TC_DEFAULT_WAIT_CYCLES : (long long)cycles;
  return MODAL_OK;
}

int modal_handle_reserve(modal_handle *h, size_t bytes) {
  if (int r = check_handle(h)) return r;
  void *p;
  return ws_get(h, 0, bytes, &p);
}

int modal_gl_nodes(modal_handle *h, int32_t n_mu, double *mu, double *om, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (n_mu < 1) return fail(h, MODAL_EINVAL, "n_mu must be >= 1");
  if (n_mu > 6400) return fail(h, MODAL_EUNSUPPORTED, "n_mu > 6400 is not supported");
  if (!mu || !om) return fail(h, MODAL_EINVAL, "null output");
  CK(launch_gl_nodes(n_mu, mu, om, (cudaStream_t)stream));
  return MODAL_OK;
}

int modal_legendre_table(modal_handle *h, int32_t n_mu, const double *mu, int32_t l_min, int32_t l_max,
                         const double *w_l, double *A, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (n_mu < 0 || l_min < 0 || l_max < l_min) return fail(h, MODAL_EINVAL, "bad sizes");
  if (!mu || !A) return fail(h, MODAL_EINVAL, "null pointer");
  if (n_mu == 0) return MODAL_OK;
  CK(launch_legendre_table(n_mu, mu, l_min, l_max, w_l, A, (cudaStream_t)stream));
  return MODAL_OK;
}

int modal_x_weights(modal_handle *h, int32_t kind, int32_t n_x, const double *x, double *w,
                    modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (kind != MODAL_XW_TRAPEZOID && kind != MODAL_XW_HERMITE) return fail(h, MODAL_EINVAL, "unknown kind");
  if (n_x < 0) return fail(h, MODAL_EINVAL, "n_x < 0");
  if (n_x == 0) return MODAL_OK;
  if (!x || !w) return fail(h, MODAL_EINVAL, "null pointer");
  CK(launch_x_weights(kind, n_x, x, w, (cudaStream_t)stream));
  return MODAL_OK;
}

int modal_contract_l(modal_handle *h, const modal_problem *p, int32_t n_mu, const double *A, int32_t precision,
                     double *M, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (int r = validate_problem(h, p, false, false)) return r;
  if (n_mu < 0 || !A || !M) return fail(h, MODAL_EINVAL, "bad A/M/n_mu");
  if (precision != MODAL_PREC_FP64 && precision != MODAL_PREC_OZAKI_BF16 && precision != MODAL_PREC_TF32 &&
      precision != MODAL_PREC_BF16X3)
    return fail(h, MODAL_EINVAL, "modal_contract_l supports FP64, OZAKI_BF16, TF32 and BF16X3");
  if (n_mu == 0 || p->n_x == 0) return MODAL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SepShape s{p->l_min, p->l_max, p->l_max - p->l_min + 1, p->nb_late, p->nb_prim, p->n_x, n_mu};
  if (precision == MODAL_PREC_FP64) {
    PROF(h, "contract_l_f64", st);
    CK(launch_contract_l<double>(s, A, p->q, p->qt, 0, p->n_x, M, st));
    return MODAL_OK;
  }
  void *scratch;
  if (precision == MODAL_PREC_TF32 || precision == MODAL_PREC_BF16X3) {
    const int kind = precision == MODAL_PREC_TF32 ? TC_FORM_TF32 : TC_FORM_BF16X3;
    if (int r = ws_get(h, 0, fa_scratch_bytes(s, p->n_x), &scratch)) return r;
    Profiler *prof = h->prof.on ? &h->prof : nullptr;
    if (int r = fa_prepare_l(kind, s, A, p->q, scratch, p->n_x, st, prof)) return fail(h, r, "%s", fa_last_error());
    if (int r = fa_contract_l(kind, s, p->qt, 0, p->n_x, p->n_x, M, true, scratch, h->wait_cycles, st, prof))
      return fail(h, r, "%s", fa_last_error());
    CK(cudaMemcpyAsync(h->pinned_err, fa_error_word(scratch), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->err_event, st));
    h->n_err_words = 1;
    h->err_pending = true;
    return MODAL_OK;
  }
  if (int r = ws_get(h, 0, tc_scratch_bytes(s, p->n_x, 1, TC_TRIPLE_FUSED), &scratch)) return r;
  {
    PROF(h, "tc_contract_l", st);
    if (int r = tc_prepare_l(s, A, p->q, scratch, p->n_x, st)) return fail(h, r, "%s", tc_last_error());
    if (int r = tc_contract_l(s, p->qt, 0, p->n_x, p->n_x, M, scratch, h->wait_cycles, st))
      return fail(h, r, "%s", tc_last_error());
  }
  CK(cudaMemcpyAsync(h->pinned_err, tc_error_word(scratch), sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(h->err_event, st));
  h->n_err_words = 1;
  h->err_pending = true;
  return MODAL_OK;
}

// ---------------------------------------------------------------------------
// separable projection (Eq. 2D)
// ---------------------------------------------------------------------------
struct SepPlan {
  SepShape s;
  int prec;
  int variant;  // tensor-core triple-product variant
  int tune = 0; // tile shape of the queue variant (tc.cuh tune_wmax / tune_split)
  int overlap = 0;  // > 0: Y pass beside the queue GEMM, which keeps num_sms - overlap SMs
  bool tail = false;  // operand and Y passes on a low-priority stream beside the one-CTA-per-tile GEMM
  int nxl;      // radial points per l-contraction chunk (tensor-core form; = nxc otherwise)
  int nxc;      // radial points per chunk
  int ksplit;   // K split of the SIMT triple product
  size_t elem;  // bytes per M element
  int64_t Gsize;
  double *est;  // error-scale output (opts->error_estimate) or NULL
  size_t bytes;
};

// Bucket of a problem for the tile autotuner: l_max in steps of 250, both
// basis sizes, and the radial count in steps of 100.
static uint64_t tile_bucket(const modal_problem *p) {
  return (uint64_t)(p->l_max / 250) << 40 | (uint64_t)p->nb_late << 28 | (uint64_t)p->nb_prim << 16 |
         (uint64_t)(p->n_x / 100);
}

static int plan_separable(modal_handle *h, const modal_problem *p, const modal_opts *o, SepPlan &pl,
                          int num_sms) {
  pl.variant = h ? h->opt_triple_variant : TC_TRIPLE_MATERIALISED;
  if (pl.variant == TC_TRIPLE_FUSED2 && !tc_fused2_fits(p->nb_late, p->nb_prim)) pl.variant = TC_TRIPLE_MATERIALISED;
  if (pl.variant == TC_TRIPLE_MATERIALISED && h && h->opt_pair) pl.variant = TC_TRIPLE_PAIR;
  else if (pl.variant == TC_TRIPLE_MATERIALISED && h && (h->opt_queue || h->opt_overlap)) pl.variant = TC_TRIPLE_QUEUE;
  if ((pl.variant == TC_TRIPLE_MATERIALISED || pl.variant == TC_TRIPLE_QUEUE) && h && h->opt_autotune) {
    auto it = h->tile_choice.find(tile_bucket(p));
    if (it != h->tile_choice.end()) {  // the autotuner's choice for this bucket
      pl.variant = it->second == 0 ? TC_TRIPLE_MATERIALISED : TC_TRIPLE_QUEUE;
      pl.tune = it->second == 0 ? 0 : it->second - 1;
    }
  }
  const bool y_hbm = pl.variant == TC_TRIPLE_MATERIALISED || pl.variant == TC_TRIPLE_PAIR ||
                     pl.variant == TC_TRIPLE_QUEUE;
  int n_mu, prec, xch;
  if (int r = resolve_opts(h, p, o, n_mu, prec, xch)) return r;
  pl.s = SepShape{p->l_min, p->l_max, p->l_max - p->l_min + 1, p->nb_late, p->nb_prim, p->n_x, n_mu};
  pl.prec = prec;
  // the TF32 / BF16x3 l contractions hand FP64 M to the tensor-core triple product
  const bool fa_form = prec == MODAL_PREC_TF32 || prec == MODAL_PREC_BF16X3;
  const bool m_f32 = prec == MODAL_PREC_FP32;
  pl.elem = m_f32 ? sizeof(float) : sizeof(double);
  const int64_t nblp = (int64_t)p->nb_late * p->nb_prim;
  if (xch > 0) {
    pl.nxc = xch < p->n_x ? xch : p->n_x;
  } else if (prec == MODAL_PREC_OZAKI_BF16 || fa_form) {
    // per radial point: M (FP64), its double-FP32 copy and its 5 BF16 slices,
    // the 5 slices of the q~ rows of the l contraction and, unless Y is formed
    // in shared memory, the 5 BF16 slices of Y (which then dominate)
    const int64_t L = p->l_max - p->l_min + 1;
    int64_t per_x = 26 * (int64_t)n_mu * nblp + 10 * (int64_t)p->nb_prim * L;
    int64_t budget = (int64_t)2 << 30;
    if (y_hbm || fa_form) {
      // 11 GiB: eight radial points per chunk at Planck size, where the
      // per-launch set-up of the GEMM tiles and the Y pass amortise best
      // (measured: 4.06 M slices/s against 3.99 M with four and 3.95 M with 16)
      const int64_t P2 = (int64_t)p->nb_prim * (p->nb_prim + 1) / 2;
      per_x += 10 * P2 * p->nb_late * (p->nb_late + 1) / 2 * (int64_t)n_mu;
      budget = (int64_t)11 << 30;
    }
    int64_t c = budget / (per_x > 0 ? per_x : 1);
    if (c > 64) c = 64;
    pl.nxc = (int)(c < 1 ? 1 : (c > p->n_x ? p->n_x : c));
  } else {
    const int64_t budget = (int64_t)2 << 30;  // 2 GiB of M per chunk
    int64_t per_x = (int64_t)n_mu * nblp * (int64_t)pl.elem;
    int64_t c = budget / (per_x > 0 ? per_x : 1);
    pl.nxc = (int)(c < 1 ? 1 : (c > p->n_x ? p->n_x : c));
  }
  if (pl.nxc < 1) pl.nxc = 1;
  pl.nxl = pl.nxc;
  if (prec == MODAL_PREC_OZAKI_BF16 && y_hbm) {
    // the l contraction runs on up to 64 radial points at once (M <= 1 GiB),
    // a whole number of triple-product chunks
    int64_t c = ((int64_t)1 << 30) / ((int64_t)n_mu * nblp * 8);
    if (c > 64) c = 64;
    if (c > p->n_x) c = p->n_x;
    c = c / pl.nxc * pl.nxc;
    pl.nxl = (int)(c < pl.nxc ? pl.nxc : c);
  }
  GLayout g = make_glayout(p->nb_late, p->nb_prim);
  pl.Gsize = g.size();
  pl.est = o ? o->error_estimate : nullptr;
  pl.ksplit = triple_ksplit(pl.s, pl.nxc, num_sms);
  const int nchunks = p->n_x > 0 ? (p->n_x + pl.nxc - 1) / pl.nxc : 0;
  const bool need_part = pl.ksplit > 1 || nchunks > 1;
  pl.overlap = (prec == MODAL_PREC_OZAKI_BF16 && pl.variant == TC_TRIPLE_QUEUE && h && h->opt_overlap > 0 &&
                !pl.est) ? h->opt_overlap : 0;
  pl.tail = prec == MODAL_PREC_OZAKI_BF16 && pl.variant == TC_TRIPLE_MATERIALISED && h && h->opt_overlap_tail &&
            !pl.est && !pl.overlap;
  size_t b = 0;
  b += 2 * align256(sizeof(double) * n_mu);                      // mu, om
  b += align256(sizeof(double) * (size_t)n_mu * pl.s.L);          // A
  b += align256(pl.elem * (size_t)pl.nxl * n_mu * nblp) * (pl.tail ? 2 : 1);  // M chunk(s)
  b += align256(sizeof(double) * (size_t)pl.Gsize);               // G
  if (pl.est) b += align256(sizeof(double) * (size_t)pl.Gsize);   // G of |M| (error scale)
  if (need_part) b += align256(sizeof(double) * (size_t)pl.Gsize * pl.ksplit);
  if (prec == MODAL_PREC_OZAKI_BF16)
    b += (pl.overlap || pl.tail) ? tc_ovl_scratch_bytes(pl.s, pl.nxl, pl.nxc)
                                 : tc_scratch_bytes(pl.s, pl.nxl, pl.nxc, pl.variant);
  if (fa_form)  // the l contraction's scratch (status word first), then the triple product's
    b += align256(fa_scratch_bytes(pl.s, pl.nxc)) + tc_scratch_bytes(pl.s, pl.nxc, pl.nxc, TC_TRIPLE_MATERIALISED);
  pl.bytes = b + 1024;
  return MODAL_OK;
}

// The tensor-core form with the Y pass of each radial chunk beside the GEMM
// of the previous one: the l contraction and the queue GEMM (on
// num_sms - overlap SMs) on the call's stream, the operand passes (column
// statistics, M~ and B slices, Y slices) on a second stream, two scratch
// sets alternating between chunks:
//   main: [l contraction L] -> GEMM(c) after prep(c)      (records gemm[c % 2])
//   side: prep(c) after the l contraction of its l-chunk and after GEMM(c - 2)
//   main waits for the side's last prep of l-chunk L before l contraction L + 1.
static int run_tc_overlap(modal_handle *h, int num_sms, const modal_problem *p, const SepPlan &pl, void *tcs,
                          double *M, double *M2, const double *om, const double *A, double *G, cudaStream_t st,
                          bool first_in_call) {
  const SepShape &s = pl.s;
  if (!h->ovl_stream) CK(cudaStreamCreateWithFlags(&h->ovl_stream, cudaStreamNonBlocking));
  if (pl.tail && !h->ovl_hi) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&h->ovl_hi, cudaStreamNonBlocking, greatest));
  }
  for (int i = 0; i < 5; ++i)
    if (!h->ovl_ev[i]) CK(cudaEventCreateWithFlags(&h->ovl_ev[i], cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) {
    if (!h->ovl_prep[i]) CK(cudaEventCreateWithFlags(&h->ovl_prep[i], cudaEventDisableTiming));
    if (!h->ovl_prep2[i]) CK(cudaEventCreateWithFlags(&h->ovl_prep2[i], cudaEventDisableTiming));
    if (!h->ovl_gemm[i]) CK(cudaEventCreateWithFlags(&h->ovl_gemm[i], cudaEventDisableTiming));
  }
  cudaStream_t side = h->ovl_stream;
  Profiler *prof = h->prof.on ? &h->prof : nullptr;
  const long long wc = h->wait_cycles;
  const int grid_sms = num_sms - pl.overlap;
  // the tail form runs the l contraction and the GEMMs on a high-priority
  // stream, so that the side stream's blocks take only the SMs that the
  // GEMM's last wave leaves idle; the call's stream waits for both at the end
  cudaStream_t user = st;
  if (pl.tail) {
    CK(cudaEventRecord(h->ovl_ev[3], user));
    CK(cudaStreamWaitEvent(h->ovl_hi, h->ovl_ev[3], 0));
    st = h->ovl_hi;
  }
  if (int r = tc_prepare_l(s, A, p->q, tcs, pl.nxl, st, prof, first_in_call))
    return fail(h, r, "tensor-core operand split failed: %s", tc_last_error());
  // l-chunk L's M: one buffer, or (tail form) two used in turn, so that the
  // next l contraction can run before the last GEMM of the current l-chunk
  // and the side stream prepares the next chunk's operands during that GEMM
  auto mbuf = [&](int L) { return (pl.tail && M2 && (L & 1)) ? M2 : M; };
  auto lcontract = [&](int L) -> int {
    const int x0 = L * pl.nxl, nl = (p->n_x - x0) < pl.nxl ? (p->n_x - x0) : pl.nxl;
    if (int r = tc_contract_l(s, p->qt, x0, nl, pl.nxl, mbuf(L), tcs, wc, st, prof))
      return fail(h, r, "tensor-core l contraction failed: %s", tc_last_error());
    return cudaEventRecord(h->ovl_ev[1], st) == cudaSuccess ? MODAL_OK
                                                              : fail(h, MODAL_ECUDA, "event record failed");
  };
  const int nL = (p->n_x + pl.nxl - 1) / pl.nxl;
  const bool ahead = pl.tail && M2;  // the next l contraction is issued before the last GEMM of an l-chunk
  int gc = 0;  // chunk count
  if (ahead && nL > 0)
    if (int r = lcontract(0)) return r;
  for (int L = 0; L < nL; ++L) {
    const int x0 = L * pl.nxl, nl = (p->n_x - x0) < pl.nxl ? (p->n_x - x0) : pl.nxl;
    if (!ahead) {
      if (L > 0) CK(cudaStreamWaitEvent(st, h->ovl_ev[2], 0));  // the side has read the previous M
      if (int r = lcontract(L)) return r;
    }
    CK(cudaStreamWaitEvent(side, h->ovl_ev[1], 0));  // l-chunk L's M is ready
    const double *Mc = mbuf(L);
    for (int xs = x0; xs < x0 + nl; xs += pl.nxc, ++gc) {
      const int ns = (x0 + nl - xs) < pl.nxc ? (x0 + nl - xs) : pl.nxc;
      const int set = gc & 1;
      const double *Ms = Mc + (size_t)(xs - x0) * s.n_mu * s.nbl * s.nbp;
      if (gc >= 2) CK(cudaStreamWaitEvent(side, h->ovl_gemm[set], 0));  // GEMM(gc - 2) used this set
      // tail form: the Y rows in two halves (the G blocks of each expansion),
      // so that the GEMM of the first half runs while the second is formed
      if (int r = tc_triple_prep(s, Ms, om, p->x_w, xs, ns, pl.nxl, pl.nxc, tcs, set, pl.tail ? 0 : -1, side,
                                 prof))
        return fail(h, r, "tensor-core triple product failed: %s", tc_last_error());
      CK(cudaEventRecord(h->ovl_prep[set], side));
      if (pl.tail) {
        if (int r = tc_triple_prep(s, Ms, om, p->x_w, xs, ns, pl.nxl, pl.nxc, tcs, set, 1, side, prof))
          return fail(h, r, "tensor-core triple product failed: %s", tc_last_error());
        CK(cudaEventRecord(h->ovl_prep2[set], side));
      }
      if (ahead && xs + pl.nxc >= x0 + nl && L + 1 < nL) {
        // before this l-chunk's last GEMM: the next l contraction, into the
        // other M buffer once the side has read it (l-chunk L - 1)
        if (L > 0) CK(cudaStreamWaitEvent(st, h->ovl_ev[2], 0));
        if (int r = lcontract(L + 1)) return r;
      }
      CK(cudaStreamWaitEvent(st, h->ovl_prep[set], 0));
      if (int r = tc_triple_gemm(s, ns, pl.nxl, pl.nxc, G, gc > 0, tcs, set, wc, grid_sms, pl.tune, pl.tail,
                                 h->opt_split_k, pl.tail ? 0 : -1, st, prof))
        return fail(h, r, "tensor-core triple product failed: %s", tc_last_error());
      if (pl.tail) {
        CK(cudaStreamWaitEvent(st, h->ovl_prep2[set], 0));
        if (int r = tc_triple_gemm(s, ns, pl.nxl, pl.nxc, G, true, tcs, set, wc, grid_sms, pl.tune, true,
                                   h->opt_split_k, 1, st, prof))
          return fail(h, r, "tensor-core triple product failed: %s", tc_last_error());
      }
      CK(cudaEventRecord(h->ovl_gemm[set], st));
    }
    CK(cudaEventRecord(h->ovl_ev[2], side));
  }
  CK(cudaStreamWaitEvent(st, h->ovl_ev[2], 0));  // nothing of the side stream outlives the call
  if (pl.tail) {  // back on the call's stream
    CK(cudaEventRecord(h->ovl_ev[4], st));
    CK(cudaStreamWaitEvent(user, h->ovl_ev[4], 0));
  }
  return MODAL_OK;
}

static int run_separable(modal_handle *h, int num_sms, const modal_problem *p, const SepPlan &pl,
                         double *gamma, cudaStream_t st, void *scratch, bool first_in_call = true,
                         bool capturing = false) {
  const SepShape &s = pl.s;
  Bump bp{(char *)scratch};
  // the tensor-core scratch comes first, so that its status words sit at the
  // same address for every problem of a batch
  const bool fa = pl.prec == MODAL_PREC_TF32 || pl.prec == MODAL_PREC_BF16X3;
  const int fa_kind = pl.prec == MODAL_PREC_TF32 ? TC_FORM_TF32 : TC_FORM_BF16X3;
  void *tcs = (pl.prec == MODAL_PREC_OZAKI_BF16)
                  ? bp.take<char>((pl.overlap || pl.tail) ? tc_ovl_scratch_bytes(s, pl.nxl, pl.nxc)
                                                          : tc_scratch_bytes(s, pl.nxl, pl.nxc, pl.variant))
                  : fa ? bp.take<char>(fa_scratch_bytes(s, pl.nxc)) : nullptr;
  // TF32 / BF16x3: the tensor-core triple product's scratch after the l contraction's
  void *fa_tc = fa ? bp.take<char>(tc_scratch_bytes(s, pl.nxc, pl.nxc, TC_TRIPLE_MATERIALISED)) : nullptr;
  double *mu = bp.take<double>(s.n_mu), *om = bp.take<double>(s.n_mu);
  double *A = bp.take<double>((size_t)s.n_mu * s.L);
  void *M = bp.take<char>(pl.elem * (size_t)pl.nxl * s.n_mu * s.nbl * s.nbp);
  void *M2 = pl.tail ? bp.take<char>(pl.elem * (size_t)pl.nxl * s.n_mu * s.nbl * s.nbp) : nullptr;
  double *G = bp.take<double>((size_t)pl.Gsize);
  double *Gabs = pl.est ? bp.take<double>((size_t)pl.Gsize) : nullptr;
  const int nchunks = (p->n_x + pl.nxc - 1) / pl.nxc;
  const bool need_part = pl.ksplit > 1 || nchunks > 1;
  double *Gpart = need_part ? bp.take<double>((size_t)pl.Gsize * pl.ksplit) : nullptr;

  {
    PROF(h, "gl_nodes", st);
    CK(launch_gl_nodes(s.n_mu, mu, om, st));                                   // a1
  }
  {
    PROF(h, "legendre_table", st);
    CK(launch_legendre_table(s.n_mu, mu, s.l_min, s.l_max, p->w_l, A, st));      // a2
  }
  if (p->n_x == 0) {
    PROFN(h, "zero_G", st, Gabs ? 2 : 1);
    CK(launch_zero(G, (size_t)pl.Gsize, st));
    if (Gabs) CK(launch_zero(Gabs, (size_t)pl.Gsize, st));
  }
  for (int c = 0; c < nchunks; ++c) {
    const int x0 = c * pl.nxc;
    const int nxc = (p->n_x - x0) < pl.nxc ? (p->n_x - x0) : pl.nxc;
    if (pl.prec == MODAL_PREC_FP64) {
      {
        PROF(h, "contract_l_f64", st);
        CK(launch_contract_l<double>(s, A, p->q, p->qt, x0, nxc, (double *)M, st));         // a4+a5
      }
      {
        PROFN(h, "triple_f64", st, triple_launches(s, nxc, pl.ksplit, c > 0));
        CK(launch_triple<double>(s, (double *)M, om, p->x_w, x0, nxc, pl.ksplit, G, Gpart, c > 0,
                                 num_sms, st));                                             // a6
      }
      if (Gabs) {
        PROFN(h, "triple_abs_f64", st, triple_launches(s, nxc, pl.ksplit, c > 0));
        CK(launch_triple<double>(s, (double *)M, om, p->x_w, x0, nxc, pl.ksplit, Gabs, Gpart, c > 0,
                                 num_sms, st, true));
      }
    } else if (fa) {
      // the l contraction on the tensor cores with FP32 accumulation (FP64
      // M), then the exact-slicing triple product of the tensor-core form
      Profiler *prof = (h && h->prof.on && !capturing) ? &h->prof : nullptr;
      const long long wc = h ? h->wait_cycles : TC_DEFAULT_WAIT_CYCLES;
      if (c == 0) {
        if (int r = fa_prepare_l(fa_kind, s, A, p->q, tcs, pl.nxc, st, prof, first_in_call))
          return fail(h, r, "tensor-core operand split failed: %s", fa_last_error());
        CK(tc_init_words(fa_tc, s, pl.nxc, 1, st));
      }
      if (int r = fa_contract_l(fa_kind, s, p->qt, x0, nxc, pl.nxc, M, true, tcs, wc, st, prof))
        return fail(h, r, "tensor-core l contraction failed: %s", fa_last_error());
      CK(tc_init_words(fa_tc, s, pl.nxc, 0, st));
      int r = tc_triple_chunk(s, (const double *)M, om, p->x_w, x0, nxc, pl.nxc, G, c > 0, fa_tc, wc, num_sms,
                              TC_TRIPLE_MATERIALISED, h ? h->opt_split_k : 0, st, prof, false, 0);
      if (!r && Gabs)
        r = tc_triple_chunk(s, (const double *)M, om, p->x_w, x0, nxc, pl.nxc, Gabs, c > 0, fa_tc, wc, num_sms,
                            TC_TRIPLE_MATERIALISED, h ? h->opt_split_k : 0, st, prof, true, 0);
      if (r) return fail(h, r, "tensor-core triple product failed: %s", tc_last_error());
    } else if (pl.prec == MODAL_PREC_FP32) {
      {
        PROF(h, "contract_l_f32", st);
        CK(launch_contract_l<float>(s, A, p->q, p->qt, x0, nxc, (float *)M, st));
      }
      {
        PROFN(h, "triple_f32", st, triple_launches(s, nxc, pl.ksplit, c > 0));
        CK(launch_triple<float>(s, (float *)M, om, p->x_w, x0, nxc, pl.ksplit, G, Gpart, c > 0,
                                num_sms, st));
      }
      if (Gabs) {
        PROFN(h, "triple_abs_f32", st, triple_launches(s, nxc, pl.ksplit, c > 0));
        CK(launch_triple<float>(s, (float *)M, om, p->x_w, x0, nxc, pl.ksplit, Gabs, Gpart, c > 0,
                                num_sms, st, true));
      }
    } else {
      // tensor-core form: the l contraction over an l-chunk of nxl points,
      // then the triple product over its chunks of nxc points
      if ((pl.overlap || pl.tail) && h && !capturing) {  // every chunk, Y pass beside the GEMM
        if (int r = run_tc_overlap(h, num_sms, p, pl, tcs, (double *)M, (double *)M2, om, A, G, st,
                                   first_in_call))
          return r;
        break;
      }
      if (x0 % pl.nxl != 0) continue;
      Profiler *prof = (h && h->prof.on && !capturing) ? &h->prof : nullptr;
      if (c == 0) {
        int r = tc_prepare_l(s, A, p->q, tcs, pl.nxl, st, prof, first_in_call);
        if (r) return fail(h, r, "tensor-core operand split failed: %s", tc_last_error());
      }
      const int nl = (p->n_x - x0) < pl.nxl ? (p->n_x - x0) : pl.nxl;
      const long long wc = h ? h->wait_cycles : TC_DEFAULT_WAIT_CYCLES;
      if (int r = tc_contract_l(s, p->qt, x0, nl, pl.nxl, (double *)M, tcs, wc, st, prof))
        return fail(h, r, "tensor-core l contraction failed: %s", tc_last_error());
      for (int xs = x0; xs < x0 + nl; xs += pl.nxc) {
        const int ns = (x0 + nl - xs) < pl.nxc ? (x0 + nl - xs) : pl.nxc;
        const double *Ms = (const double *)M + (size_t)(xs - x0) * s.n_mu * s.nbl * s.nbp;
        int r = tc_triple_chunk(s, Ms, om, p->x_w, xs, ns, pl.nxl, G, xs > 0, tcs, wc, num_sms, pl.variant,
                                h ? h->opt_split_k : 0, st, prof, false, pl.tune);
        if (r) return fail(h, r, "tensor-core triple product failed: %s", tc_last_error());
        if (Gabs) {
          r = tc_triple_chunk(s, Ms, om, p->x_w, xs, ns, pl.nxl, Gabs, xs > 0, tcs, wc, num_sms, pl.variant,
                              h ? h->opt_split_k : 0, st, prof, true, pl.tune);
          if (r) return fail(h, r, "tensor-core triple product (error scale) failed: %s", tc_last_error());
        }
      }
    }
  }
  if (fa && nchunks > 0)  // the triple product's status joins the l contraction's word
    CK(tc_or_status(fa_error_word(tcs), fa_tc, st));
  if ((pl.prec == MODAL_PREC_OZAKI_BF16 || fa) && nchunks > 0 && !capturing && h) {
    // surface a bounded-wait give-up through modal_handle_status (no sync here)
    CK(cudaMemcpyAsync(h->pinned_err, fa ? fa_error_word(tcs) : tc_error_word(tcs), sizeof(int),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->err_event, st));
    h->n_err_words = 1;
    h->err_pending = true;
  }
  PROFN(h, "gather", st, Gabs ? 2 : 1);
  // the tensor-core triple product's layout of G depends on its variant
  const GLayout gl = pl.prec == MODAL_PREC_OZAKI_BF16 ? tc_triple_glayout(s, pl.variant)
                     : fa ? tc_triple_glayout(s, TC_TRIPLE_MATERIALISED) : make_glayout(s.nbl, s.nbp);
  CK(launch_gather(s, G, p->late_modes, p->prim_modes, p->n_late, p->n_prim, 1.0 / (48.0 * MODAL_PI), gamma,
                   st, &gl));                                                               // a7
  if (Gabs)
    CK(launch_gather(s, Gabs, p->late_modes, p->prim_modes, p->n_late, p->n_prim, 1.0 / (48.0 * MODAL_PI),
                     pl.est, st, &gl));
  return MODAL_OK;
}

int modal_workspace_size(const modal_problem *p, const modal_opts *o, int for_backward, size_t *bytes) {
  if (!bytes) return fail(nullptr, MODAL_EINVAL, "null output");
  if (int r = validate_problem(nullptr, p, false, false)) return r;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  SepPlan pl;
  if (int r = plan_separable(nullptr, p, o, pl, sms)) return r;
  size_t b = pl.bytes;
  if (for_backward) {
    size_t bb = pl.prec == MODAL_PREC_OZAKI_BF16 ? tc_backward_scratch_bytes(pl.s, tc_backward_nxc(pl.s, sms))
                                                 : backward_scratch_bytes(pl.s, pl.nxc, pl.prec);
    b = bb > b ? bb : b;
  }
  *bytes = b;
  return MODAL_OK;
}

int modal_project_separable(modal_handle *h, const modal_problem *p, const modal_opts *o, double *gamma,
                            modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (int r = validate_problem(h, p, true, true)) return r;
  if ((int64_t)p->n_late * p->n_prim == 0) return MODAL_OK;
  if (!gamma) return fail(h, MODAL_EINVAL, "null gamma");
  SepPlan pl;
  if (int r = plan_separable(h, p, o, pl, h->num_sms)) return r;
  void *scratch;
  if (int r = ws_get(h, 0, pl.bytes, &scratch)) return r;
  return run_separable(h, h->num_sms, p, pl, gamma, (cudaStream_t)stream, scratch);
}

// ---------------------------------------------------------------------------
// Gram matrix <Q_n, Q_r> and the full Gamma (Appendix A)
// ---------------------------------------------------------------------------
int modal_gram(modal_handle *h, const modal_problem *p, const double *w_gram, const modal_opts *o,
               double *gram, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (!p) return fail(h, MODAL_EINVAL, "null problem");
  if (p->l_min < 0 || p->l_max < p->l_min) return fail(h, MODAL_EINVAL, "bad l range [%d, %d]", p->l_min, p->l_max);
  if (p->nb_late < 1 || p->nb_late > 64)
    return fail(h, MODAL_EINVAL, "nb_late must be in [1, 64] (got %d)", p->nb_late);
  if (p->n_late < 0) return fail(h, MODAL_EINVAL, "negative size");
  if (p->n_late == 0) return MODAL_OK;
  if (!p->q || !p->late_modes || !w_gram || !gram) return fail(h, MODAL_EINVAL, "null q, late_modes, w_gram or gram");
  // the late basis projected on itself: q~ := q at one radial point of unit
  // weight, l weight w_gram, primordial modes := late modes
  modal_problem g = *p;
  g.nb_prim = p->nb_late;
  g.n_x = 1;
  g.qt = p->q;
  g.w_l = w_gram;
  g.n_prim = p->n_late;
  g.prim_modes = p->late_modes;
  g.x_w = nullptr;
  SepPlan pl;
  if (int r = plan_separable(h, &g, o, pl, h->num_sms)) return r;
  void *scratch;
  if (int r = ws_get(h, 0, align256(pl.bytes) + 256, &scratch)) return r;
  double *one = (double *)((char *)scratch + align256(pl.bytes));  // the unit radial weight
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_fill(one, 1, 1.0, st));
  g.x_w = one;
  if (int r = run_separable(h, h->num_sms, &g, pl, gram, st, scratch)) return r;
  PROFN(h, "gram_symmetrise", st, pl.est ? 2 : 1);
  CK(launch_symmetrise(gram, p->n_late, st));
  if (pl.est) CK(launch_symmetrise(pl.est, p->n_late, st));
  return MODAL_OK;
}

int modal_gram_solve(modal_handle *h, int32_t n, int32_t m, const double *gram, const double *rhs, double *x,
                     int32_t *info, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (n < 0 || m < 0) return fail(h, MODAL_EINVAL, "negative size");
  if (n > 0 && !gram) return fail(h, MODAL_EINVAL, "null gram");
  if (n > 0 && m > 0 && (!rhs || !x)) return fail(h, MODAL_EINVAL, "null rhs or x");
  if (n > 0 && m > 0 && x == gram) return fail(h, MODAL_EINVAL, "x must not alias gram");
  void *scratch;
  if (int r = ws_get(h, 3, gram_solve_scratch_bytes(n), &scratch)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  PROFN(h, "gram_solve", st, gram_solve_launches(n, m));
  CK(gram_solve(n, m, gram, rhs, x, scratch, (int *)info, st));
  return MODAL_OK;
}

// FNV-1a over the bytes of the problem set: the key of a captured graph
static uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
  const unsigned char *c = (const unsigned char *)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ULL;
  }
  return h;
}

// Work estimate of one problem (for spreading a batch over streams): the
// triple product's MACs plus the l contraction's, per slice, times slices.
static double problem_cost(const modal_problem *p, int n_mu) {
  const GLayout g = make_glayout(p->nb_late, p->nb_prim);
  const double L = (double)(p->l_max - p->l_min + 1);
  return ((double)g.size() + L * p->nb_late * p->nb_prim) * (double)p->n_x * (double)n_mu;
}

// A batch spread over `ns` streams (batch_plan.h: longest first, each to
// the least loaded stream; one scratch block per stream)
using BatchLayout = batch::Layout;
static_assert(batch::MAX_STREAMS == MAX_BATCH_STREAMS, "one stream limit");
static BatchLayout batch_layout(int n, const modal_problem *probs, const std::vector<SepPlan> &plans, int ns) {
  std::vector<double> cost(n);
  std::vector<size_t> bytes(n);
  for (int i = 0; i < n; ++i) {
    cost[i] = problem_cost(&probs[i], plans[i].s.n_mu);
    bytes[i] = plans[i].bytes;
  }
  return batch::layout(n, cost.data(), bytes.data(), ns);
}

// Capture every launch of the batch into one graph, the problems of stream k
// on side stream k (forked from and joined back into the capture stream).
static int capture_batch(modal_handle *h, int n, const modal_problem *probs, const std::vector<SepPlan> &plans,
                         double *const *gammas, const BatchLayout &bl, char *scratch, cudaGraphExec_t *out) {
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (!h->fork_ev) CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
  for (int k = 1; k < bl.ns; ++k) {
    if (!h->side[k]) CK(cudaStreamCreateWithFlags(&h->side[k], cudaStreamNonBlocking));
    if (!h->join_ev[k]) CK(cudaEventCreateWithFlags(&h->join_ev[k], cudaEventDisableTiming));
  }
  const bool prof_on = h->prof.on;
  h->prof.on = false;  // no event records inside the capture
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
  int rr = MODAL_OK;
  cudaError_t ce = cudaSuccess;
  if (bl.ns > 1) {
    ce = cudaEventRecord(h->fork_ev, h->cap_stream);
    for (int k = 1; k < bl.ns && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(h->side[k], h->fork_ev, 0);
  }
  bool first[MAX_BATCH_STREAMS];
  for (int k = 0; k < MAX_BATCH_STREAMS; ++k) first[k] = true;
  for (int i = 0; i < n && rr == MODAL_OK && ce == cudaSuccess; ++i) {
    if ((int64_t)probs[i].n_late * probs[i].n_prim == 0) continue;
    const int k = bl.stream_of[i];
    cudaStream_t sk = k == 0 ? h->cap_stream : h->side[k];
    rr = run_separable(h, h->num_sms, &probs[i], plans[i], gammas[i], sk, scratch + bl.off[k], first[k], true);
    first[k] = false;
  }
  for (int k = 1; k < bl.ns && ce == cudaSuccess; ++k) {
    ce = cudaEventRecord(h->join_ev[k], h->side[k]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->cap_stream, h->join_ev[k], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &graph);
  h->prof.on = prof_on;
  if (rr != MODAL_OK || ce != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (rr != MODAL_OK) return rr;
    return fail(h, MODAL_ECUDA, "graph capture: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  }
  ce = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(h, MODAL_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
  return MODAL_OK;
}

// The tile autotuner: times the triple GEMM's candidate shapes -- one CTA
// per tile; the queue form with column tiles of at most 128 (K split, or
// not) or 64 -- on one radial chunk of problem p (second of two runs each,
// CUDA events on the call's stream, blocking) and keeps the fastest for p's
// bucket.  gamma (p's output) receives scratch results.
static int tune_tiles(modal_handle *h, const modal_problem *p, const modal_opts *o, double *gamma,
                      cudaStream_t st) {
  static const int cands[] = {0, 1 + 0, 1 + (8 | 16), 1 + 4};
  modal_problem sub = *p;
  SepPlan pl;
  if (int r = plan_separable(h, &sub, o, pl, h->num_sms)) return r;
  sub.n_x = pl.nxc < p->n_x ? pl.nxc : p->n_x;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_c = 0, rr = MODAL_OK;
  for (int c : cands) {
    SepPlan q;
    if ((rr = plan_separable(h, &sub, o, q, h->num_sms)) != MODAL_OK) break;
    q.variant = c == 0 ? TC_TRIPLE_MATERIALISED : TC_TRIPLE_QUEUE;
    q.tune = c == 0 ? 0 : c - 1;
    q.tail = false;  // the GEMM's own time, as the batched graph runs it
    void *scr;
    if ((rr = ws_get(h, 0, q.bytes, &scr)) != MODAL_OK) break;
    if ((rr = run_separable(h, h->num_sms, &sub, q, gamma, st, scr)) != MODAL_OK) break;
    cudaError_t ce = cudaEventRecord(e0, st);
    if (ce == cudaSuccess && (rr = run_separable(h, h->num_sms, &sub, q, gamma, st, scr)) != MODAL_OK) break;
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce != cudaSuccess) {
      rr = fail(h, MODAL_ECUDA, "timing the tile shapes: %s", cudaGetErrorString(ce));
      break;
    }
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rr != MODAL_OK) return rr;
  h->tile_choice[tile_bucket(p)] = best_c;
  return MODAL_OK;
}

int modal_project_separable_batched(modal_handle *h, int32_t n, const modal_problem *probs,
                                    const modal_opts *o, double *const *gammas, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (n < 0) return fail(h, MODAL_EINVAL, "n < 0");
  if (n == 0) return MODAL_OK;
  if (!probs || !gammas) return fail(h, MODAL_EINVAL, "null probs/gammas");
  if (o && o->error_estimate) return fail(h, MODAL_EINVAL, "error_estimate is for single-problem calls");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<SepPlan> plans(n);
  bool any_tc = false;
  for (int i = 0; i < n; ++i) {
    if (int r = validate_problem(h, &probs[i], true, true)) return fail(h, r, "problem %d: %s", i, h->err.c_str());
    if (int r = plan_separable(h, &probs[i], o, plans[i], h->num_sms))
      return fail(h, r, "problem %d: %s", i, h->err.c_str());
    if ((int64_t)probs[i].n_late * probs[i].n_prim > 0 && !gammas[i])
      return fail(h, MODAL_EINVAL, "null gamma for problem %d", i);
    any_tc = any_tc || plans[i].prec == MODAL_PREC_OZAKI_BF16 || plans[i].prec == MODAL_PREC_TF32 ||
             plans[i].prec == MODAL_PREC_BF16X3;  // their status word heads each stream's scratch
  }
  // tile shapes: time the buckets that have no choice yet, then plan with the choices
  if (h->opt_autotune) {
    bool tuned = false;
    for (int i = 0; i < n; ++i) {
      const modal_problem &pp = probs[i];
      if (plans[i].prec != MODAL_PREC_OZAKI_BF16) continue;
      if (plans[i].variant != TC_TRIPLE_MATERIALISED && plans[i].variant != TC_TRIPLE_QUEUE) continue;
      if ((int64_t)pp.n_late * pp.n_prim == 0 || pp.n_x == 0) continue;
      if (h->tile_choice.count(tile_bucket(&pp))) continue;
      if (int r = tune_tiles(h, &pp, o, gammas[i], st)) return fail(h, r, "tile autotuner, problem %d: %s", i,
                                                                    h->err.c_str());
      tuned = true;
    }
    if (tuned)
      for (int i = 0; i < n; ++i)
        if (int r = plan_separable(h, &probs[i], o, plans[i], h->num_sms)) return r;
  }
  // stream counts to consider: the fixed option, or 1, 2, 4, 8 (at most n)
  // while their scratch fits in half of the free device memory
  std::vector<BatchLayout> cands;
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) freeb = 0;
  for (int ns = 1; ns <= MAX_BATCH_STREAMS; ns *= 2) {
    if (h->opt_batch_streams > 0 && ns != h->opt_batch_streams) continue;
    if (ns > 1 && ns > n) break;
    BatchLayout bl = batch_layout(n, probs, plans, ns);
    const size_t cap = freeb / 2 < ((size_t)64 << 30) ? freeb / 2 : ((size_t)64 << 30);
    if (ns > 1 && h->opt_batch_streams == 0 && bl.off[ns] > h->slot_bytes[0] && bl.off[ns] > cap) break;
    cands.push_back(bl);
  }
  if (h->opt_batch_streams > 0 && cands.empty()) {
    const int ns = h->opt_batch_streams < n ? h->opt_batch_streams : n;
    cands.push_back(batch_layout(n, probs, plans, ns));
  }
  size_t need = 0;
  for (auto &bl : cands) need = bl.off[bl.ns] > need ? bl.off[bl.ns] : need;
  void *scratch;
  if (int r = ws_get(h, 0, need, &scratch)) return r;  // before capture: no allocation inside
  uint64_t key = 1469598103934665603ULL;
  key = fnv1a(key, &n, sizeof n);
  key = fnv1a(key, probs, sizeof(modal_problem) * (size_t)n);
  if (o) key = fnv1a(key, o, sizeof *o);
  key = fnv1a(key, gammas, sizeof(double *) * (size_t)n);
  key = fnv1a(key, &scratch, sizeof scratch);
  key = fnv1a(key, &h->opt_triple_variant, sizeof(int));
  key = fnv1a(key, &h->opt_split_k, sizeof(int));
  key = fnv1a(key, &h->opt_pair, sizeof(int));
  key = fnv1a(key, &h->opt_queue, sizeof(int));
  for (int i = 0; i < n; ++i) {  // the tile shapes chosen per problem
    key = fnv1a(key, &plans[i].variant, sizeof(int));
    key = fnv1a(key, &plans[i].tune, sizeof(int));
  }
  key = fnv1a(key, &h->opt_batch_streams, sizeof(int));
  key = fnv1a(key, &h->wait_cycles, sizeof(long long));
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    // capture one graph per candidate; with several, replay each twice and
    // keep the one whose second replay is fastest (blocks this first call)
    std::vector<cudaGraphExec_t> execs;
    for (auto &bl : cands) {
      cudaGraphExec_t ex = nullptr;
      if (int r = capture_batch(h, n, probs, plans, gammas, bl, (char *)scratch, &ex)) {
        for (auto x : execs) cudaGraphExecDestroy(x);
        return r;
      }
      execs.push_back(ex);
    }
    int best = 0;
    if (execs.size() > 1) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      float best_ms = 1e30f;
      for (size_t c = 0; c < execs.size(); ++c) {
        cudaError_t ce = cudaGraphLaunch(execs[c], st);
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
        if (ce == cudaSuccess) ce = cudaGraphLaunch(execs[c], st);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          for (auto x : execs) cudaGraphExecDestroy(x);
          return fail(h, MODAL_ECUDA, "timing the batched graphs: %s", cudaGetErrorString(ce));
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = (int)c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    for (size_t c = 0; c < execs.size(); ++c)
      if ((int)c != best) cudaGraphExecDestroy(execs[c]);
    it = h->graphs.emplace(key, modal_handle::BatchGraph{execs[best], cands[best].ns}).first;
  }
  CK(cudaGraphLaunch(it->second.exec, st));
  if (any_tc) {
    const int ns = it->second.streams;
    const BatchLayout bl = batch_layout(n, probs, plans, ns);
    for (int k = 0; k < ns; ++k)
      CK(cudaMemcpyAsync(h->pinned_err + k, tc_error_word((char *)scratch + bl.off[k]), sizeof(int),
                         cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->err_event, st));
    h->n_err_words = ns;
    h->err_pending = true;
  }
  return MODAL_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of modal_project_separable.  Its scratch is this
// file-scope device array (present on every GPU that loads the library, for
// the life of the process).  In host code the array's name is only a
// host-side stand-in, so the device address is taken with
// cudaGetSymbolAddress at set-up -- once per device, in its current context,
// and again only if that context was replaced (a cudaDeviceReset reloads the
// module, and the array may then sit elsewhere) -- and kernels receive it.
// ---------------------------------------------------------------------------
#define MODAL_NOALLOC_SCRATCH_BYTES ((size_t)48 << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[MODAL_NOALLOC_SCRATCH_BYTES];

namespace {
struct NoallocDevice {
  void *scratch = nullptr;
  int num_sms = 0;
  unsigned long long ctx_id = 0;  // context the address belongs to
  bool ready = false;
};
constexpr int NOALLOC_MAX_DEVICES = 64;
NoallocDevice g_noalloc_dev[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;
}  // namespace

extern "C" int modal_project_separable_noalloc(const modal_problem *p, const modal_opts *o, double *gamma,
                                               modal_stream_t stream) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, MODAL_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return fail(nullptr, MODAL_EUNSUPPORTED, "device ordinal %d beyond %d", dev, NOALLOC_MAX_DEVICES);
  // the unique id of the thread's current context (never reused within the
  // process); 0 if none is current yet
  // (driver entry points resolved through the runtime, so that loading the
  // library needs no libcuda on machines without a GPU)
  typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
  typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
  static const CtxGetCurrentFn get_current = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
               ? (CtxGetCurrentFn)p
               : (CtxGetCurrentFn) nullptr;
  }();
  static const CtxGetIdFn get_id = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
               ? (CtxGetIdFn)p
               : (CtxGetIdFn) nullptr;
  }();
  auto current_ctx_id = []() -> unsigned long long {
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
      return 0;
    return id;
  };
  const unsigned long long ctx_id = current_ctx_id();
  NoallocDevice nd;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocDevice &slot = g_noalloc_dev[dev];
    if (!slot.ready || ctx_id == 0 || slot.ctx_id != ctx_id) {  // set-up on this device / context (no allocation)
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // also makes the device's context current
      if (e != cudaSuccess)
        return fail(nullptr, MODAL_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
      slot.ctx_id = current_ctx_id();
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess)
        return fail(nullptr, MODAL_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
      slot.scratch = ptr;
      slot.num_sms = sms;
      slot.ready = true;
    }
    nd = slot;
  }
  if (int r = validate_problem(nullptr, p, true, true)) return r;
  if ((int64_t)p->n_late * p->n_prim == 0) return MODAL_OK;
  if (!gamma) return fail(nullptr, MODAL_EINVAL, "null gamma");
  const int prec = o ? o->precision : MODAL_PREC_FP64;
  if (prec != MODAL_PREC_FP64 && prec != MODAL_PREC_FP32)
    return fail(nullptr, MODAL_EINVAL, "the allocation-free entry point serves MODAL_PREC_FP64 and MODAL_PREC_FP32");
  // the largest radial chunk (at most the caller's or the automatic one)
  // whose scratch fits the static buffer
  modal_opts oo = o ? *o : modal_opts{0, MODAL_PREC_FP64, 0, 0, nullptr};
  SepPlan pl;
  if (int r = plan_separable(nullptr, p, &oo, pl, nd.num_sms)) return r;
  for (int nxc = pl.nxc - 1; pl.bytes > MODAL_NOALLOC_SCRATCH_BYTES && nxc >= 1; --nxc) {
    oo.x_chunk = nxc;
    if (int r = plan_separable(nullptr, p, &oo, pl, nd.num_sms)) return r;
  }
  if (pl.bytes > MODAL_NOALLOC_SCRATCH_BYTES)
    return fail(nullptr, MODAL_EINVAL,
                "problem needs %zu bytes of scratch; the allocation-free entry point's static scratch holds %zu",
                pl.bytes, MODAL_NOALLOC_SCRATCH_BYTES);
  return run_separable(nullptr, nd.num_sms, p, pl, gamma, (cudaStream_t)stream, nd.scratch);
}

// ---------------------------------------------------------------------------
// direct projection (Eq. 3D)
// ---------------------------------------------------------------------------
int modal_project_direct(modal_handle *h, const modal_problem *p, const int32_t *l_grid, const double *l_dw,
                         int32_t ng, int32_t mode, double *gamma, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (int r = validate_problem(h, p, true, true)) return r;
  if (mode != MODAL_W_EXACT_3J && mode != MODAL_W_SMOOTH_GOSPER) return fail(h, MODAL_EINVAL, "unknown weight mode");
  if (ng < 0) return fail(h, MODAL_EINVAL, "n_grid < 0");
  if ((int64_t)p->n_late * p->n_prim == 0) return MODAL_OK;
  if (!gamma) return fail(h, MODAL_EINVAL, "null gamma");
  cudaStream_t st = (cudaStream_t)stream;
  const int L = p->l_max - p->l_min + 1;
  if (ng == 0 || p->n_x == 0) {
    CK(launch_zero(gamma, (size_t)p->n_late * p->n_prim, st));
    return MODAL_OK;
  }
  if (!l_grid) return fail(h, MODAL_EINVAL, "null l_grid");
  if (p->l_max > 21000) return fail(h, MODAL_EUNSUPPORTED, "l_max > 21000 is not supported by the direct form");
  if (h->opt_direct_tensor == 2 && tc_direct_supported(p->nb_late, p->nb_prim)) {
    // radial integrals and Gamma' update on the tensor cores
    void *scratch;
    if (int r = ws_get(h, 0, tc_direct_scratch_bytes(p, ng), &scratch)) return r;
    Profiler *prof = h->prof.on ? &h->prof : nullptr;
    if (int r = tc_project_direct(p, l_grid, l_dw, ng, mode, gamma, scratch, h->num_sms, h->wait_cycles, st, prof))
      return fail(h, r, "tensor-core direct form failed: %s", tc_last_error());
    CK(cudaMemcpyAsync(h->pinned_err, tc_error_word(scratch), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->err_event, st));
    h->n_err_words = 1;
    h->err_pending = true;
    return MODAL_OK;
  }
  const int64_t npairs = (int64_t)ng * ng;
  const int cmax = 3 * p->l_max / 2 + 2;
  // The triple count is known only on the device.  Batches of T triples are
  // sized on the host from the bound C(ng + 2, 3) (every sorted triple of
  // grid points); each kernel reads the true count and batches past it do no
  // work, so the call never waits for the device.
  const int64_t ntri_max = (int64_t)ng * (ng + 1) * (ng + 2) / 6;
  int T = 32768;
  {
    int64_t cap = ((int64_t)1 << 30) / (8 * (int64_t)(p->n_late + p->n_prim));
    if (cap < 256) cap = 256;
    if (T > cap) T = (int)(cap / 32 * 32);
    if (T > ntri_max) T = (int)ntri_max;
  }
  const int64_t nbatch = cdiv64(ntri_max, T);
  size_t scan_b = scan_tmp_bytes(npairs);
  size_t b1 = 0;
  b1 += align256(sizeof(double) * (size_t)L * p->n_x * p->nb_prim);     // qt transposed
  b1 += 2 * align256(sizeof(int64_t) * (size_t)npairs);                 // counts, offsets
  b1 += align256(sizeof(double) * (size_t)(cmax + 1));                  // 3j product table
  b1 += align256(sizeof(int64_t));                                      // triple count
  b1 += align256(scan_b);
  b1 += align256(sizeof(int) * 3 * (size_t)T) + align256(sizeof(double) * (size_t)T);  // batch triples, weights
  b1 += align256(sizeof(double) * (size_t)T * p->n_late) + align256(sizeof(double) * (size_t)T * p->n_prim);
  b1 += 1024;
  void *s1, *tcs = nullptr;
  if (int r = ws_get(h, 1, b1, &s1)) return r;
  if (h->opt_direct_tensor)
    if (int r = ws_get(h, 0, tc_gemm_batch_scratch_bytes(p->n_late, p->n_prim, T), &tcs)) return r;
  Bump bp{(char *)s1};
  double *qtT = bp.take<double>((size_t)L * p->n_x * p->nb_prim);
  int64_t *counts = bp.take<int64_t>((size_t)npairs);
  int64_t *offs = bp.take<int64_t>((size_t)npairs);
  double *ctab = bp.take<double>((size_t)cmax + 1);
  int64_t *ntri = bp.take<int64_t>(1);
  void *scan_tmp = bp.take<char>(scan_b);
  int *tri = bp.take<int>(3 * (size_t)T);
  double *z = bp.take<double>((size_t)T);
  double *Yb = bp.take<double>((size_t)T * p->n_late);
  double *Xb = bp.take<double>((size_t)T * p->n_prim);

  {
    PROFN(h, "direct_setup", st, 6);  // transpose, 3j table, counts, scan (2), total
    int64_t rows = (int64_t)p->n_x * p->nb_prim, cols = L;
    dim3 grid((unsigned)cdiv64(cols, 32), (unsigned)cdiv64(rows, 32));
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(p->qt, rows, cols, qtT);
    CK(cudaGetLastError());
    CK(launch_threej_table(cmax, ctab, st));
    k_direct_count<<<(unsigned)cdiv64(npairs, 256), 256, 0, st>>>(ng, l_grid, mode, counts);
    CK(cudaGetLastError());
    CK(scan_exclusive_i64(scan_tmp, scan_b, counts, offs, npairs, st));
    k_direct_total<<<1, 32, 0, st>>>(counts, offs, npairs, ntri);
    CK(cudaGetLastError());
  }
  const int nbp = p->nb_prim, P2 = nbp * (nbp + 1) / 2;
  int xc = 16;
  size_t smem = 0;
  for (;; xc /= 2) {
    smem = sizeof(double) * ((size_t)nbp * P2 + (size_t)xc * P2 + 3 * (size_t)xc * nbp);
    if (smem <= 200 * 1024 || xc == 1) break;
  }
  if (smem > 200 * 1024) return fail(h, MODAL_EUNSUPPORTED, "primordial basis too large for the direct path");
  CK(cudaFuncSetAttribute(k_direct_X, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int64_t bi = 0; bi < nbatch; ++bi) {
    const int64_t t0 = bi * T;
    {
      PROF(h, "direct_fill", st);
      k_direct_fill_batch<<<(unsigned)cdiv(T, 256), 256, 0, st>>>(ng, l_grid, l_dw, p->w_l, p->l_min, ctab, mode,
                                                                  offs, ntri, t0, T, tri, z);
      CK(cudaGetLastError());
    }
    {
      PROF(h, "direct_X", st);
      k_direct_X<<<T, 256, smem, st>>>(nbp, p->n_x, p->l_min, qtT, p->x_w, tri, 0, T, xc, p->prim_modes,
                                       p->n_prim, Xb, ntri, t0);
      CK(cudaGetLastError());
    }
    {
      PROF(h, "direct_Y", st);
      int64_t ny = (int64_t)p->n_late * T;
      k_direct_Y<<<(unsigned)cdiv64(ny, 256), 256, 0, st>>>(p->nb_late, L, p->l_min, p->q, tri, z, 0, T, ntri, t0,
                                                            p->late_modes, p->n_late, Yb);
      CK(cudaGetLastError());
    }
    if (tcs) {
      // Gamma' += Y X^T over the batch's triples on the exact-slicing GEMM
      // (Gamma' zeroed before the first batch; batches past the end do nothing)
      if (bi == 0) CK(launch_zero(gamma, (size_t)p->n_late * p->n_prim, st));
      Profiler *prof = h->prof.on ? &h->prof : nullptr;
      if (int r = tc_gemm_batch(p->n_late, p->n_prim, T, Yb, Xb, ntri, t0, gamma, p->n_prim, tcs, bi == 0,
                                h->wait_cycles, st, prof))
        return fail(h, r, "tensor-core direct update failed: %s", tc_last_error());
    } else {
      PROF(h, "direct_gemm", st);
      CK(launch_gemm_nt_f64(p->n_late, p->n_prim, T, Yb, T, Xb, T, gamma, p->n_prim, bi > 0, st, ntri, t0));
    }
  }
  if (tcs) {
    CK(cudaMemcpyAsync(h->pinned_err, tc_error_word(tcs), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->err_event, st));
    h->n_err_words = 1;
    h->err_pending = true;
  }
  return MODAL_OK;
}

// ---------------------------------------------------------------------------
// adjoint (not in the paper; from Eq. 2D and Eq. legendre)
// ---------------------------------------------------------------------------
int modal_project_backward(modal_handle *h, const modal_problem *p, const modal_opts *o,
                           const double *dL_dgamma, double *dL_dqt, double *dL_dq, modal_stream_t stream) {
  if (int r = check_handle(h)) return r;
  if (int r = validate_problem(h, p, true, true)) return r;
  if (!dL_dgamma || !dL_dqt) return fail(h, MODAL_EINVAL, "null dL_dgamma or dL_dqt");
  SepPlan pl;
  if (int r = plan_separable(h, p, o, pl, h->num_sms)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (pl.prec == MODAL_PREC_OZAKI_BF16) {  // the adjoint's three contractions on the tensor cores
    int nxc = tc_backward_nxc(pl.s, h->num_sms);
    if (o && o->x_chunk > 0 && o->x_chunk < nxc) nxc = o->x_chunk;  // a smaller chunk on request
    void *scratch;
    if (int r = ws_get(h, 0, tc_backward_scratch_bytes(pl.s, nxc), &scratch)) return r;
    Profiler *prof = h->prof.on ? &h->prof : nullptr;
    if (int r = tc_backward(pl.s, nxc, p, dL_dgamma, dL_dqt, dL_dq, scratch, h->wait_cycles, st, prof))
      return fail(h, r, "tensor-core adjoint failed: %s", tc_last_error());
    if (pl.s.n_x > 0 && (int64_t)p->n_late * p->n_prim > 0) {
      CK(cudaMemcpyAsync(h->pinned_err, tc_error_word(scratch), sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(h->err_event, st));
      h->n_err_words = 1;
      h->err_pending = true;
    }
    return MODAL_OK;
  }
  size_t bytes = backward_scratch_bytes(pl.s, pl.nxc, pl.prec);
  void *scratch;
  if (int r = ws_get(h, 0, bytes, &scratch)) return r;
  int r = run_backward(pl.s, pl.nxc, pl.prec, p, dL_dgamma, dL_dqt, dL_dq, scratch, h->num_sms, st);
  if (r) return fail(h, r, "adjoint failed: %s", backward_last_error());
  return MODAL_OK;
}

}  // extern "C"
