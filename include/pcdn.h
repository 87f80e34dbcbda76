/*
 * pcdn.h -- C ABI of the GB300 PCDN solver.
 *
 * Parallel Coordinate Descent Newton (Bian, Li, Liu, Yang, arXiv:1306.4080)
 * for L1-regularised logistic regression and L1-regularised L2-loss SVM:
 *
 *     min_w  F(w) = c * sum_i phi(w; x_i, y_i) + ||w||_1          (Section 2, Eq. 1)
 *     phi = log(1 + exp(-y_i w^T x_i))                                (Eq. 2)
 *     phi = max(0, 1 - y_i w^T x_i)^2                                 (Eq. 3)
 *
 * Notation: n_samples = the paper's s, n_features = the paper's n.  X is
 * n_samples x n_features, sparse, compressed by columns (CSC).
 *
 * Every entry point returns an int status (PCDN_OK = 0, < 0 error, > 0 a
 * completed call with a caveat) and records a message readable with
 * pcdn_last_error() (thread-local).  No entry point throws or aborts.
 * Host pointers are read during the call only and never retained, unless a
 * comment says otherwise.  All device work runs in the library's CUDA
 * kernels; there is no CPU fallback.  A call that needs a GPU fails with
 * PCDN_ECUDA when none is present.
 */
#ifndef PCDN_H
#define PCDN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define PCDN_OK 0
#define PCDN_EINVAL (-1)        /* bad argument: malformed CSC, label not +/-1, C <= 0, P out of [1, n_features], ... */
#define PCDN_ENOMEM (-2)        /* a device or host allocation failed */
#define PCDN_ECUDA (-3)         /* a CUDA call failed (no device, launch error, ...) */
#define PCDN_ENUMERIC (-4)      /* a non-finite gradient, Hessian, objective change or maintained quantity */
#define PCDN_ETIMEOUT (-5)      /* a device-side wait between thread blocks gave up (bounded spin) */
#define PCDN_ENOTCONVERGED 1    /* max_epochs reached before the tolerance; outputs are still written */

typedef enum { PCDN_LOSS_LOGISTIC = 0, PCDN_LOSS_L2SVM = 1 } pcdn_loss;

/* PCDN_PREC_FP64: all arithmetic in FP64 (X values are stored as FP32 and widened).
 * PCDN_PREC_MIXED: X, g, h, d and the per-sample line-search curvature terms in
 *   FP32; the step's first-order term, Delta, the line-search sums, the maintained
 *   quantities, w and the KKT test in FP64. */
typedef enum { PCDN_PREC_FP64 = 0, PCDN_PREC_MIXED = 1 } pcdn_precision;

/* Sparse X by columns.  Column j holds rows row_idx[col_ptr[j] .. col_ptr[j+1])
 * strictly ascending, with values val[...].  col_ptr[0] == 0, col_ptr[n_features] == nnz.
 * Pointers are host memory for pcdn_create and device memory for pcdn_create_device. */
typedef struct {
  int64_t n_samples;
  int64_t n_features;
  int64_t nnz;
  const int64_t* col_ptr; /* [n_features + 1] */
  const int32_t* row_idx; /* [nnz] */
  const float* val;       /* [nnz], finite */
} pcdn_csc;

/* Solver options; fill with pcdn_default_opts() and override fields. */
typedef struct {
  double sigma;       /* Armijo sufficient-decrease factor, Eq. 6 (default 0.01, Section 5.1) */
  double beta;        /* backtracking factor, Eq. 6 (default 0.5, Section 5.1) */
  double gamma;       /* weight of d^T H d in Delta, Eq. 7 (default 0, Section 5.1) */
  double nu;          /* replaces a Hessian diagonal <= 0 (default 1e-12, Appendix A, proof of Lemma 1(b)) */
  int32_t q_max;      /* backtracking cap; at the cap the bundle is left unchanged (default 30) */
  int32_t ls_batch;   /* step sizes beta^q evaluated per pass over the touched samples (1..8; 0 = default: 1 on the first pass, 4 after) */
  int64_t max_epochs; /* outer-iteration cap (default 1000) */
  pcdn_precision prec;
  int32_t warm_start; /* 0: the solve starts from w = 0 (Algorithm 3); 1: from the problem's current w */
  int32_t grid_ctas;  /* thread blocks of the bundle walker; 0 = one group covering the whole GPU */
  int32_t refresh;    /* 1 (default): recompute the maintained quantities from z = Xw after each outer iteration */
  uint32_t spin_limit;/* iterations a device-side wait may spin before PCDN_ETIMEOUT (0 = default) */
} pcdn_opts;

/* Per-solve statistics (written by pcdn_solve). */
typedef struct {
  int64_t epochs;        /* outer iterations run */
  int64_t bundles;       /* inner iterations (bundles) processed */
  int64_t coord_updates; /* features visited = sum of bundle sizes */
  int64_t ls_steps;      /* step sizes tested, summed over bundles with a nonzero direction */
  int64_t ls_cap_hits;   /* bundles whose backtracking reached q_max */
  int64_t ls_passes;     /* passes over touched samples (each tests up to ls_batch step sizes) */
  int64_t nnz_visited;   /* sum over bundles of the bundle's nonzeros */
  int64_t rows_touched;  /* sum over bundles of the number of touched samples */
  int64_t kernel_launches; /* CUDA kernels this library launched during the solve */
  double F_final;        /* objective (Eq. 1) at the returned w */
  double kkt_rel;        /* ||v(w)||_1 / ||v(0)||_1, v the minimum-norm subgradient */
  double kkt0;           /* ||v(w0)||_1 at the start point */
  double wall_s;         /* host wall time of the solve */
  double walk_s;         /* device time of the bundle-walker launches (CUDA events) */
  double bytes_model;    /* algorithmic bytes of the bundle steps: sum of 16 nnz_B + 33 |U_B| + 16 P */
  int32_t converged;     /* kkt_rel <= eps */
  int32_t walk_grid;     /* thread blocks of the bundle walker (last launch) */
} pcdn_stats;

/* Optional per-bundle / per-epoch record of a solve (caller-owned host arrays,
 * each may be NULL; entries beyond the capacities are not written). */
typedef struct {
  int64_t bundle_cap;
  int32_t* q;        /* [bundle_cap] accepted q (q_max at the cap) */
  double* alpha;     /* [bundle_cap] accepted step (0 at the cap, 1 when d = 0) */
  double* Delta;     /* [bundle_cap] Eq. 7 */
  double* dF;        /* [bundle_cap] F(w + alpha d) - F(w) as evaluated by the line search */
  int64_t epoch_cap;
  double* epoch_kkt; /* [epoch_cap] relative KKT after each outer iteration */
} pcdn_trace;

typedef struct pcdn_problem pcdn_problem;

/* Default options (see field comments). */
void pcdn_default_opts(pcdn_opts* opts);

/* Copy X (host CSC), y (host, n_samples entries in {-1, +1}) to the device and
 * build the row-major mirror of X used for z = Xw.  C > 0 is the loss weight c
 * of Eq. 1.  The problem starts at w = 0 and owns its device memory until
 * pcdn_destroy.  Errors: PCDN_EINVAL (columns not ascending, row out of range,
 * non-finite value, label not +/-1, C <= 0), PCDN_ENOMEM, PCDN_ECUDA. */
int pcdn_create(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, pcdn_problem** out);

/* As pcdn_create, but X's arrays and y are device pointers (e.g. from PyTorch)
 * that the caller keeps alive and unchanged until pcdn_destroy; they are read,
 * never written.  `stream` (a cudaStream_t, may be NULL = the library's own
 * stream) orders the library's work after the caller's producers. Validation
 * runs on the device. */
int pcdn_create_device(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, void* stream,
                       pcdn_problem** out);

/* Algorithm 3 (with Algorithm 4): outer iterations of a fresh random partition
 * (Eq. 8) into bundles of P features (the last one m mod P when P does not
 * divide m), each bundle stepped in turn, until the relative minimum-norm
 * subgradient (recomputed after every outer iteration) is <= eps or
 * max_epochs is reached.  The partition of outer iteration k orders the
 * features by splitmix64 keys of (seed, k), ties by index.  w_out (host,
 * n_features entries, may be NULL) receives w; stats (may be NULL) and trace
 * (may be NULL) are filled.  Returns PCDN_OK, PCDN_ENOTCONVERGED, or an error. */
int pcdn_solve(pcdn_problem* prob, int32_t P, double eps, uint64_t seed, const pcdn_opts* opts,
               double* w_out, pcdn_stats* stats, pcdn_trace* trace);

/* One inner iteration of Algorithm 3 on the caller's bundle (host array of P
 * distinct feature indices), from w_in (host, n_features entries; NULL = the
 * problem's current w, whose maintained quantities are then used as they are).
 * Outputs (host, each may be NULL): g[P], h[P] (Eq. 11 / generalised Hessian,
 * h <= 0 replaced by nu), d[P] (Eq. 5), Delta (Eq. 7), q and alpha = beta^q
 * (Eq. 6; q = q_max and alpha = 0 at the cap), dF (the line search's value of
 * F(w + alpha d) - F(w)).  The problem's w and maintained quantities advance. */
int pcdn_bundle_step(pcdn_problem* prob, const double* w_in, const int32_t* bundle, int32_t P,
                     const pcdn_opts* opts, double* g, double* h, double* d, double* Delta, int32_t* q,
                     double* alpha, double* dF);

/* Set w (host, n_features entries) and recompute the maintained quantities. */
int pcdn_set_w(pcdn_problem* prob, const double* w);
/* Copy the current w to the host (n_features entries). */
int pcdn_get_w(pcdn_problem* prob, double* w);
/* Objective F(w) (Eq. 1) at the current w, from z = Xw. */
int pcdn_objective(pcdn_problem* prob, double* F);
/* ||v(w)||_1 of the minimum-norm subgradient at the current w (fresh gradient). */
int pcdn_kkt(pcdn_problem* prob, double* kkt_l1);
/* The feature order of outer iteration `epoch` (host, n_features entries), as
 * pcdn_solve draws it on the device. */
int pcdn_permutation(pcdn_problem* prob, uint64_t seed, int64_t epoch, int32_t* perm);
/* Device-resident sizes (bytes) held by the problem. */
int pcdn_memory(pcdn_problem* prob, int64_t* bytes);

/* Objective without allocation.
 *
 * For callers that may not allocate device memory (an application that owns all GPU memory
 * through its own pool or budget, or a request loop that allows no allocator calls): the
 * objective F(w) = C * sum_i phi(w; x_i, y_i) + ||w||_1 from the caller's device buffers,
 * with no cudaMalloc, cudaFree or other allocating call.  The paper has no counterpart; the
 * value equals pcdn_objective's for the same X, y, C, loss and w (up to summation order).
 *
 * X's arrays, y (n_samples labels in {-1, +1}), w (n_features doubles) and F (one double,
 * written) are device pointers; the call only enqueues work on `stream` (a cudaStream_t, NULL =
 * the legacy default stream) and returns: F is ready once that stream has reached this work.
 * Its scratch (z = Xw and per-block partial sums) is one fixed array of about 2 MiB inside the
 * library, held on every GPU that loads the library until the process exits; hence
 * n_samples <= PCDN_NOALLOC_MAX_SAMPLES, larger problems return PCDN_EINVAL.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress) and keeps it: make
 * that first call before any stream capture.  All calls share the array, so calls that may
 * run at the same time on the GPU race: order them (one stream, or events).  A row index
 * outside [0, n_samples) makes F NaN.  Errors: PCDN_EINVAL, PCDN_ECUDA. */
#define PCDN_NOALLOC_MAX_SAMPLES 262144
int pcdn_objective_noalloc(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, const double* w,
                           double* F, void* stream);

void pcdn_destroy(pcdn_problem* prob);
/* Message of the last failed call on this thread ("" if none). */
const char* pcdn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PCDN_H */
