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
#define PCDN_ENUMERIC (-4)      /* a non-finite gradient, Hessian, objective change or maintained quantity;
                                   FP64 mode keeps e^{w^T x_i} (Algorithm 4) and so also fails once some
                                   |w^T x_i| passes about 699, where mixed precision (which keeps w^T x_i)
                                   goes on */
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
  int32_t shrink;     /* 1: shrinking between outer iterations (default 0: every outer iteration visits every
                         feature, Algorithm 3).  The first outer iteration visits every feature; outer
                         iteration k >= 1 visits, in its random order (Eq. 8), only the features with
                         w_j != 0 or |g_j| >= 1 - M/n_samples at the stopping test of iteration k-1
                         (M = max_j |v_j|, v the minimum-norm subgradient).  The stopping test still
                         covers every feature.  Solves that shrink are not captured as CUDA graphs. */
  int64_t epoch0;     /* index of the first outer iteration (its partition, Eq. 8, is drawn with this index; default 0) */
  double kkt_ref;     /* > 0: relative KKT measured against this ||v||_1 instead of the start point's (default 0).
                         A solve stopped after k outer iterations resumes exactly with warm_start = 1 from its w,
                         epoch0 = k and kkt_ref = its stats.kkt0 */
  int32_t layout;     /* how d^T x_i (Algorithm 4) reaches the samples: PCDN_LAYOUT_AUTO (default), _SCATTER or _ROWS */
} pcdn_opts;

/* PCDN_LAYOUT_ROWS: per outer iteration the entries of every bundle's columns are regrouped by
 *   sample; the thread that owns a sample sums its d^T x_i in a fixed order, and the step's full
 *   update is written before the step-size decision (two grid barriers per bundle on the usual
 *   path).  Every sum has a fixed order: FP64 results repeat bit for bit for a given walker grid.
 * PCDN_LAYOUT_SCATTER: each block adds d_j x_ij into a dense vector with atomic adds (results
 *   repeat up to rounding); no regrouping pass.
 * PCDN_LAYOUT_AUTO: rows for FP64 solves whose walker spans several thread blocks, scatter otherwise. */
#define PCDN_LAYOUT_AUTO 0
#define PCDN_LAYOUT_SCATTER 1
#define PCDN_LAYOUT_ROWS 2

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
  int64_t* epoch_features; /* [epoch_cap] features visited by each outer iteration (n_features unless shrinking) */
} pcdn_trace;

typedef struct pcdn_problem pcdn_problem;

/* Default options (see field comments; the Armijo parameters are Section 5.1's sigma = 0.01,
 * beta = 0.5, gamma = 0). */
void pcdn_default_opts(pcdn_opts* opts);

/* Copy X (host CSC), y (host, n_samples entries in {-1, +1}) to the device and
 * build the row-major mirror of X used for z = Xw.  C > 0 is the loss weight c
 * of Eq. 1.  The problem starts at w = 0 and owns its device memory until
 * pcdn_destroy.  Errors: PCDN_EINVAL (columns not ascending, row out of range,
 * non-finite value, label not +/-1, C <= 0), PCDN_ENOMEM, PCDN_ECUDA. */
int pcdn_create(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, pcdn_problem** out);

/* The problem of Eq. 1 as pcdn_create, but X's arrays and y are device pointers (e.g. from PyTorch)
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

/* Set w (host, n_features entries) and recompute the maintained quantities of Section 3.1
 * (e^{w^T x_i} for the logistic loss, b_i = 1 - y_i w^T x_i for the L2-SVM) from z = Xw. */
int pcdn_set_w(pcdn_problem* prob, const double* w);
/* Change the loss weight c of Eq. 1 (C > 0, finite).  w and the maintained quantities are kept
 * (neither depends on c), so a following pcdn_solve with opts.warm_start = 1 continues from the
 * current w: one step of a warm-started regularisation path.  Errors: PCDN_EINVAL. */
int pcdn_set_C(pcdn_problem* prob, double C);
/* Separable penalty (the concluding remarks' generalisation to a convex twice-differentiable loss
 * plus a separable regulariser): the problem becomes
 *   min_w  c sum_i phi(w; x_i, y_i) + l1 ||w||_1 + (l2/2) ||w||_2^2,
 * L1 (the paper's problem, l1 = 1, l2 = 0: the default), ridge (l1 = 0) or elastic net.  Every
 * step uses the smooth part's gradient g + l2 w and Hessian diagonal h + l2; the direction is Eq. 5
 * with l1 in place of 1; Delta (Eq. 7) takes l1 times the L1 change; the line search adds the
 * penalty's change; pcdn_objective, pcdn_kkt and the stopping test use the penalised objective
 * (shrinking's bound becomes l1 - M/n_samples).  w and the maintained quantities are kept.
 * Errors: PCDN_EINVAL (l1 or l2 negative or not finite, both zero). */
int pcdn_set_penalty(pcdn_problem* prob, double l1, double l2);
/* Copy the current w, the iterate of Algorithm 3, to the host (n_features entries); library
 * management, no passage of its own. */
int pcdn_get_w(pcdn_problem* prob, double* w);
/* Objective F(w) (Eq. 1, with the problem's penalty) at the current w, from z = Xw. */
int pcdn_objective(pcdn_problem* prob, double* F);
/* ||v(w)||_1 of the minimum-norm subgradient at the current w (fresh gradient): the quantity of
 * the stopping test (Section 5.1 names newGLMNET's outer condition; this library's reading is the
 * relative l1 norm of the minimum-norm subgradient). */
int pcdn_kkt(pcdn_problem* prob, double* kkt_l1);
/* The feature order of outer iteration `epoch` (host, n_features entries), as
 * pcdn_solve draws it on the device: the random partition of Eq. 8 and Algorithm 3. */
int pcdn_permutation(pcdn_problem* prob, uint64_t seed, int64_t epoch, int32_t* perm);
/* Device-resident sizes (bytes) held by the problem; library management, no passage. */
int pcdn_memory(pcdn_problem* prob, int64_t* bytes);

/* ---- many solves on one GPU ----------------------------------------------------------------
 *
 * The paper solves one problem at a time (Algorithm 3).  These calls run many independent solves
 * concurrently on one GPU; each solve runs exactly pcdn_solve's stages, kernels and stop rule on
 * its problem's own stream, so solves of different problems overlap on the device while each
 * advances at its own pace.  A solve's bundle walker is one thread block, or several (a
 * cooperative launch) when its bundles are large and the GPU has blocks to spare: the walker
 * blocks of all concurrent multi-block walkers are kept within what the GPU holds resident.  Each
 * solve's outer iterations are replayed from a CUDA graph captured at its first one. */

/* One job of a batch: a problem solved along a regularisation path. */
typedef struct {
  pcdn_problem* prob;   /* from pcdn_create / pcdn_create_device; distinct for every job */
  int32_t P;            /* bundle size in [1, n_features], or 0: chosen by the autotuner (below) */
  double eps;           /* relative KKT tolerance of every solve of the job */
  uint64_t seed;        /* partition seed (Eq. 8) of every solve */
  int32_t n_C;          /* >= 1 */
  const double* C_path; /* host [n_C]: C_path[0] is solved from opts->warm_start's start point,
                           each later C from the previous solution (warm start) */
  double* w_out;        /* host [n_C * n_features] (row k = w at C_path[k]), may be NULL */
  pcdn_stats* stats;    /* host [n_C], may be NULL */
  int32_t status;       /* out: PCDN_OK, PCDN_ENOTCONVERGED (some solve hit max_epochs) or the error
                           that ended the job */
  int32_t P_used;       /* out: the bundle size the job's path ran with */
  int32_t layout_used;  /* out: the walker layout of its path (PCDN_LAYOUT_*; AUTO = the library's choice) */
} pcdn_batch_job;

typedef struct {
  int32_t max_inflight;   /* jobs in flight at once (0 = one per hardware work queue: CUDA_DEVICE_MAX_CONNECTIONS,
                             CUDA's default 8, at most 32; set it before the process creates its CUDA context) */
  int32_t threads;        /* host threads driving them (0 = 4) */
  double probe_eps;       /* autotuner: relative KKT a probe solve aims at (0 = 0.1) */
  int32_t probe_epochs;   /* autotuner: outer-iteration cap of a probe solve (0 = no cap beyond opts) */
  int32_t n_candidates;   /* autotuner: bundle sizes to try (0 = powers of 4 from 16 to min(4096, n_features)) */
  const int32_t* candidates;
  int32_t no_graphs;      /* 1: issue every outer iteration's kernels directly instead of replaying a graph */
  int32_t tune_layout;    /* autotuner: 1 also probes, for each candidate bundle size whose walker
                             takes more than one block, the walker layout the library would not pick
                             (PCDN_LAYOUT_ROWS for mixed precision, SCATTER for FP64); only when
                             opts->layout is PCDN_LAYOUT_AUTO */
} pcdn_batch_opts;

typedef struct {
  double wall_s;          /* host wall time of the whole batch */
  int64_t solves;         /* path solves completed */
  int64_t probe_solves;   /* autotuner probe solves */
  int64_t epochs;         /* outer iterations of the path solves */
  int64_t coord_updates;  /* features visited by the path solves */
  double bytes_model;     /* algorithmic bytes of the path solves' bundle steps */
  int64_t graph_solves;   /* path solves whose outer iterations replayed a captured CUDA graph */
  int64_t retries;        /* path solves of autotuned jobs repeated with a smaller bundle size after
                             reaching max_epochs (counted in solves once, with their last attempt) */
} pcdn_batch_stats;

/* Defaults: max_inflight 0, threads 0, probe_eps 0.1, probe_epochs 3, default candidates,
 * tune_layout 0 (on the 64-problem batch the extra probes cost more than the layouts they found
 * gained: 8.2 s against 7.1 to 7.5 s).  No
 * passage: the paper solves one problem at a time (Algorithm 3). */
void pcdn_default_batch_opts(pcdn_batch_opts* bopts);

/* Algorithm 3 on many problems at once (no passage: the paper solves one problem at a time; each
 * solve is exactly pcdn_solve's).  Solve every job's path (opts, may be NULL = defaults, apply to every solve; grid_ctas is
 * ignored: each solve's walker is one thread block, or several from the shared block budget when
 * its bundles hold more than about 2048 nonzeros).  A job with P = 0 first runs a short probe solve
 * from w = 0 at the geometric middle of its C path for each candidate bundle size (to probe_eps, at
 * most probe_epochs outer iterations) and keeps the one with the least walker device time per
 * decade of KKT reduction; it then needs opts->warm_start = 0.  When a solve of such a job reaches
 * max_epochs, its C is solved again from the w reached, with the next smaller candidate (and the
 * job keeps that size for the rest of its path; P_used reports it): a bundle size probed at the
 * path's middle can stall at its largest C, where the coordinates couple more strongly.  Jobs run concurrently, up to max_inflight at a time.  Returns the
 * first error of any job (with its message), else PCDN_ENOTCONVERGED if some solve reached
 * max_epochs, else PCDN_OK; every job's status is written.  Errors: PCDN_EINVAL (bad job, two jobs
 * on one problem), PCDN_ECUDA, and the solve errors of pcdn_solve. */
int pcdn_solve_batch(pcdn_batch_job* jobs, int32_t n_jobs, const pcdn_opts* opts, const pcdn_batch_opts* bopts,
                     pcdn_batch_stats* out);

/* The bundle-size autotuner (Section 5.1 and Table 3 choose P* empirically; this replaces that
 * search) on one problem (at its current C): for each candidate P (NULL/0 = the
 * defaults above), a probe solve from w = 0 to probe_eps (at most probe_epochs outer iterations;
 * 0 = opts' cap) with a one-block walker; *P_best = the candidate with the least walker device
 * time per decade of relative-KKT reduction; probe_s (may be NULL, [n_candidates or the default count]) receives each score.  The
 * problem is left at the last probe's w. */
int pcdn_autotune(pcdn_problem* prob, const int32_t* candidates, int32_t n_candidates, double probe_eps,
                  int32_t probe_epochs, uint64_t seed, const pcdn_opts* opts, int32_t* P_best, double* probe_s);

/* ---- request server: continuous batching ------------------------------------------------------
 *
 * A server owns its host threads.  The admission thread takes submitted requests in arrival
 * order, waits until a slot is free and the request's device footprint fits the memory budget
 * (a request larger than the whole budget is admitted alone) and reserves both; creator threads
 * then copy admitted requests to the device (pcdn_create), several at once.  The driver thread
 * starts each created request's solve in a free slot and advances all of them concurrently, one
 * stream each, with the walker blocks and CUDA graphs of the batch solver.  A finished request's w
 * and statistics are kept on the host until pcdn_server_wait collects them, and its device memory
 * is released at once, so waiting requests are admitted while others are still on the GPU. */
typedef struct pcdn_server pcdn_server;

typedef struct {
  int32_t slots;        /* solves in flight at once (0 = one per hardware work queue, as for batches) */
  int64_t hbm_budget;   /* device bytes the admitted requests may hold together (0 = 8 GiB) */
  pcdn_opts solve;      /* options of every solve (warm_start and grid_ctas are ignored) */
} pcdn_server_opts;

/* What pcdn_server_wait reports about a request; times are seconds since the server was created. */
typedef struct {
  int32_t status;       /* the solve's status (as pcdn_solve's return value) */
  double t_submit;      /* pcdn_server_submit returned */
  double t_admit;       /* admitted (slot and memory reserved; requests are admitted in arrival order) */
  double t_start;       /* copied to the device, solve started */
  double t_done;        /* solved, w on the host */
  int64_t bytes;        /* device footprint used for admission */
  pcdn_stats stats;     /* of the last solve; kkt_rel and kkt0 measured from w = 0 */
  int32_t P_used;       /* bundle size of the last solve */
  int32_t retries;      /* solves repeated with a smaller bundle size (below) */
} pcdn_request_info;

/* Default server options.  No passage: serving is not in the paper (each request is one solve of
 * Algorithm 3). */
void pcdn_default_server_opts(pcdn_server_opts* opts);
/* Start a server on the current device (no passage, as above).  Errors: PCDN_EINVAL, PCDN_ENOMEM,
 * PCDN_ECUDA. */
int pcdn_server_create(const pcdn_server_opts* opts, pcdn_server** out);
/* Queue one solve of Eq. 1 by Algorithm 3 (as pcdn_create + pcdn_solve from w = 0).  A solve that
 * reaches max_epochs with P above 16 goes on from the w it reached with the next smaller of the
 * bundle sizes 4096, 1024, 256, 64, 16 (its relative KKT target still measured from w = 0), so
 * that a bundle size too large for the request's C stalls no request; info reports the size used.  X and y are host arrays, copied
 * before the call returns.  *ticket identifies the request.  Full validation of X and y happens at
 * admission; a malformed request then finishes with PCDN_EINVAL.  Errors: PCDN_EINVAL (sizes, C,
 * loss, P, eps), PCDN_ENOMEM. */
int pcdn_server_submit(pcdn_server* srv, const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, int32_t P,
                       double eps, uint64_t seed, int64_t* ticket);
/* As pcdn_server_submit (one solve of Algorithm 3), but X's arrays and y are not copied: the caller keeps them valid and
 * unchanged until pcdn_server_wait has returned the request's result (a caller that already holds
 * its problems in host memory saves a copy per request). */
int pcdn_server_submit_borrowed(pcdn_server* srv, const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss,
                                int32_t P, double eps, uint64_t seed, int64_t* ticket);
/* Wait up to timeout_s seconds (<= 0: no limit) for a request (library management, no passage);
 * then w_out (host, n_features entries, may be NULL) and info (may be NULL) receive its result and
 * the request is forgotten (each ticket can be collected once).  Returns the request's status,
 * PCDN_ETIMEOUT if it did not finish in time (it can be waited for again), or PCDN_EINVAL for an
 * unknown ticket.  info is written only for a finished request: a caller that needs to tell a
 * solve that itself ended with PCDN_ETIMEOUT from a wait that timed out sets info->status to a
 * value no call returns before the call and checks it after. */
int pcdn_server_wait(pcdn_server* srv, int64_t ticket, double timeout_s, double* w_out, pcdn_request_info* info);
/* Counters (library management, no passage): requests submitted and finished so far, requests
 * holding device memory, and the device bytes they were admitted with.  Any pointer may be NULL. */
int pcdn_server_stats(pcdn_server* srv, int64_t* submitted, int64_t* finished, int32_t* in_flight,
                      int64_t* bytes_in_use);
/* Stop the server (library management, no passage): solves in flight end after their current
 * stage, uncollected results and queued requests are dropped, all device memory is released. */
void pcdn_server_destroy(pcdn_server* srv);

/* Objective without allocation.
 *
 * For callers that may not allocate device memory (an application that owns all GPU memory
 * through its own pool or budget, or a request loop that allows no allocator calls): the
 * objective F(w) = C * sum_i phi(w; x_i, y_i) + ||w||_1 from the caller's device buffers,
 * with no cudaMalloc, cudaFree or other allocating call (the paper's penalty, l1 = 1, l2 = 0).
 * The paper has no counterpart; the value equals pcdn_objective's for the same X, y, C, loss and
 * w on a problem with the default penalty (up to summation order).
 *
 * X's arrays, y (n_samples labels in {-1, +1}), w (n_features doubles) and F (one double,
 * written) are device pointers; the call only enqueues work on `stream` (a cudaStream_t, NULL =
 * the legacy default stream) and returns: F is ready once that stream has reached this work.
 * Its scratch (z = Xw and per-block partial sums) is one fixed array of about 2 MiB inside the
 * library, which a GPU holds from the first call on it until the process exits; hence
 * n_samples <= PCDN_NOALLOC_MAX_SAMPLES, larger problems return PCDN_EINVAL.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress) and keeps it; under
 * CUDA's lazy module loading (the default) that first call also loads the library's module on
 * the device and places the array there, the one allocation this entry point causes: make that
 * first call at set-up, before any stream capture, and later calls allocate nothing.  After a
 * cudaDeviceReset the kept address is stale: reload the library before calling again.  All
 * calls share the array, so calls that may run at the same time on the GPU race: order them (one
 * stream, or events).  A row index outside [0, n_samples), a column pointer outside [0, nnz) or
 * decreasing, or a label other than +/-1 makes F NaN (nothing outside the arrays is read).
 * Errors: PCDN_EINVAL, PCDN_ECUDA. */
#define PCDN_NOALLOC_MAX_SAMPLES 262144
/* F(w) of Eq. 1 without allocation (described above; the paper has no counterpart). */
int pcdn_objective_noalloc(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, const double* w,
                           double* F, void* stream);

/* Release the problem's device memory and stream (library management, no passage). */
void pcdn_destroy(pcdn_problem* prob);
/* Message of the last failed call on this thread ("" if none; library management, no passage). */
const char* pcdn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PCDN_H */
