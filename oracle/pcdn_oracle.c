/*
 * PCDN reference oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of Parallel Coordinate
 * Descent Newton (Bian, Li, Liu, Yang, arXiv:1306.4080) for L1-regularised
 * logistic regression and L1-regularised L2-loss SVM.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load this code; the
 * CUDA library never does, and the two share no code.
 *
 * Every routine follows the paper's steps in the paper's order:
 *   objective                 Section 2, Eq. 1 with the losses of Eq. 2 / Eq. 3
 *   gradient / Hessian diag   Section 3.1, Eq. 11 (logistic); Appendix A, proof of
 *                             Lemma 1(b) (generalised Hessian of the L2-loss SVM)
 *   direction                 Section 2.1, Eq. 4 solved in closed form (Eq. 5, read
 *                             with the +/-1 terms in its conditions)
 *   Armijo rule               Section 2.1, Eq. 6 and Eq. 7
 *   line search               Section 3.1, Eq. 10 and Algorithm 4
 *   bundle walk               Section 3, Eq. 8, Eq. 9 and Algorithm 3
 *   CDN                       Section 2.1, Algorithm 1 (PCDN with P = 1)
 *
 * Readings where the paper is silent or garbled (each one is also listed in
 * the design notes):
 *   - Eq. 5 prints "g <= h w" / "g >= h w"; minimising g d + h d^2/2 + |w + d|
 *     gives "g + 1 <= h w" / "g - 1 >= h w".  The corrected form is used.
 *   - The L2-SVM gradient and line-search terms are not printed; they follow by
 *     differentiating Eq. 3: g_j = -2c sum_{b_i > 0} y_i x_ij b_i with
 *     b_i = 1 - y_i w^T x_i, and the loss change of row i at step a is
 *     max(0, b_i - a y_i d^T x_i)^2 - max(0, b_i)^2.
 *   - nu = 1e-12 replaces a Hessian diagonal h <= 0 (Appendix A, proof of
 *     Lemma 1(b)); applied to both losses.
 *   - The line search is capped at q_max steps; at the cap the bundle is
 *     left unchanged (a = 0) and the cap is counted.
 *   - Random partition (Eq. 8, Algorithm 3): features sorted by 64-bit keys
 *     from splitmix64 (Steele, Lea, Flood 2014), ties by feature index; bundle
 *     t holds sorted positions [tP, min((t+1)P, m)).
 *   - Stopping rule (Section 5.1 only names newGLMNET's outer condition):
 *     after each outer iteration the maintained quantities are recomputed
 *     from z = Xw, and the solve stops once the l1 norm of the minimum-norm
 *     subgradient is at most eps times its value at w = 0.
 *   - Separable regularisers (the concluding remarks: a convex twice-
 *     differentiable loss plus a separable penalty, covering L1, L2 and
 *     their mixture): F(w) = c sum_i phi + l1 ||w||_1 + (l2/2) ||w||_2^2
 *     with l1, l2 >= 0 (the paper's problem: l1 = 1, l2 = 0).  The smooth
 *     part's gradient and Hessian diagonal are g + l2 w and h + l2 (h after
 *     the nu rule); the direction minimises the model of Eq. 4 with l1 |.|;
 *     Delta (Eq. 7) takes the smooth part's g and h and l1 times the L1
 *     change; the line search adds (l2/2)(||w + a d||^2 - ||w||^2).
 *   - Shrinking (Section 5.1 says only that the comparison's shrinking runs
 *     outside the parallel loop): optional, between outer iterations.  The
 *     first outer iteration of a solve visits every feature; outer iteration
 *     k >= 1 visits the active set of w^k (the iterate after k outer
 *     iterations, with its maintained quantities just recomputed): feature j
 *     is active unless w_j = 0 and |g_j(w^k)| < 1 - M_k / s, where M_k is the
 *     largest |v_j(w^k)| of the minimum-norm subgradient and s the number of
 *     samples (the margin of LIBLINEAR's CDN shrinking, taken from a fresh
 *     gradient).  The iteration's partition is the full random order of Eq. 8
 *     restricted to the active features, in bundles of P.  The stopping rule
 *     is unchanged (all features).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_ENOTCONVERGED 1

#define OR_LOSS_LOGISTIC 0
#define OR_LOSS_L2SVM 1

typedef struct {
  int64_t n;              /* samples (the paper's s) */
  int64_t m;              /* features (the paper's n) */
  const int64_t* col_ptr; /* [m+1] */
  const int32_t* row_idx; /* [nnz], ascending within each column */
  const float* val;       /* [nnz] */
  const int8_t* y;        /* [n], +1 / -1 */
  double c;               /* loss weight c > 0 of Eq. 1 */
  int loss;               /* OR_LOSS_* */
  double l1, l2;          /* penalty l1 ||w||_1 + (l2/2) ||w||^2 (Eq. 1: l1 = 1, l2 = 0) */
} or_problem;

typedef struct {
  double sigma, beta, gamma, nu;
  int q_max;
} or_armijo;

typedef struct {
  int64_t epochs, bundles, coord_updates, ls_steps, ls_cap_hits;
  double F_final, kkt_rel, kkt0;
  int converged;
} or_stats;

/* ------------------------------------------------------------------------- */
/* splitmix64 (Steele, Lea, Flood 2014): state advance + output mix.          */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static const uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ULL;

/* k-th output (k >= 1) of the splitmix64 stream whose state starts at s0 */
uint64_t or_splitmix64_output(uint64_t s0, uint64_t k) { return sm64_mix(s0 + k * SM64_GAMMA); }

/* sort key of feature j in outer iteration `epoch` */
uint64_t or_perm_key(uint64_t seed, int64_t epoch, int64_t j) {
  uint64_t s_epoch = or_splitmix64_output(seed ^ ((uint64_t)epoch * 0xD1B54A32D192ED03ULL), 1);
  return or_splitmix64_output(s_epoch, (uint64_t)j + 1);
}

typedef struct { uint64_t key; int32_t j; } or_keyed;

static int cmp_keyed(const void* a, const void* b) {
  const or_keyed* x = (const or_keyed*)a;
  const or_keyed* y = (const or_keyed*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->j > y->j) - (x->j < y->j);
}

/* Random disjoint partition of the features for one outer iteration
 * (Eq. 8, Algorithm 3): perm[0..m) is the feature order; bundles are
 * consecutive slices of length P. */
int or_permutation(uint64_t seed, int64_t epoch, int64_t m, int32_t* perm) {
  if (m <= 0 || !perm) return OR_EINVAL;
  or_keyed* kk = (or_keyed*)malloc(sizeof(or_keyed) * (size_t)m);
  if (!kk) return OR_ENOMEM;
  for (int64_t j = 0; j < m; ++j) { kk[j].key = or_perm_key(seed, epoch, j); kk[j].j = (int32_t)j; }
  qsort(kk, (size_t)m, sizeof(or_keyed), cmp_keyed);
  for (int64_t t = 0; t < m; ++t) perm[t] = kk[t].j;
  free(kk);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* z = X w, accumulated column by column                                      */
static void xw(const or_problem* p, const double* w, double* z) {
  for (int64_t i = 0; i < p->n; ++i) z[i] = 0.0;
  for (int64_t j = 0; j < p->m; ++j) {
    if (w[j] == 0.0) continue;
    for (int64_t k = p->col_ptr[j]; k < p->col_ptr[j + 1]; ++k) z[p->row_idx[k]] += (double)p->val[k] * w[j];
  }
}

/* F(w) = c sum_i phi(w; x_i, y_i) + ||w||_1   (Eq. 1, Eq. 2, Eq. 3) */
double or_objective(const or_problem* p, const double* w) {
  double* z = (double*)malloc(sizeof(double) * (size_t)(p->n > 0 ? p->n : 1));
  if (!z) return NAN;
  xw(p, w, z);
  double L = 0.0;
  for (int64_t i = 0; i < p->n; ++i) {
    double yz = (double)p->y[i] * z[i];
    if (p->loss == OR_LOSS_LOGISTIC) {
      /* log(1 + exp(-yz)), evaluated without overflow */
      L += (yz > 0) ? log1p(exp(-yz)) : (-yz + log1p(exp(yz)));
    } else {
      double b = 1.0 - yz;
      L += b > 0 ? b * b : 0.0;
    }
  }
  free(z);
  double r = 0.0, q = 0.0;
  for (int64_t j = 0; j < p->m; ++j) r += fabs(w[j]);
  if (p->l2 != 0.0)
    for (int64_t j = 0; j < p->m; ++j) q += w[j] * w[j];
  return p->c * L + p->l1 * r + 0.5 * p->l2 * q;
}

/* Maintained per-sample quantity from w (Section 3.1): e^{w^T x_i} for the
 * logistic loss, b_i = 1 - y_i w^T x_i for the L2-loss SVM. */
int or_refresh(const or_problem* p, const double* w, double* mq) {
  double* z = (double*)malloc(sizeof(double) * (size_t)(p->n > 0 ? p->n : 1));
  if (!z) return OR_ENOMEM;
  xw(p, w, z);
  for (int64_t i = 0; i < p->n; ++i)
    mq[i] = (p->loss == OR_LOSS_LOGISTIC) ? exp(z[i]) : 1.0 - (double)p->y[i] * z[i];
  free(z);
  return OR_OK;
}

/* Gradient and Hessian diagonal of L at feature j from the maintained
 * quantities.  Logistic: Eq. 11 with tau(s) = 1/(1+e^{-s}) written through
 * E_i = e^{w^T x_i}: tau(y_i z_i) = E_i/(1+E_i) for y_i = +1 and 1/(1+E_i)
 * for y_i = -1.  L2-SVM: generalised Hessian 2c sum_{i in I(w)} x_ij^2 with
 * I(w) = {i : y_i w^T x_i < 1} (Appendix A, proof of Lemma 1(b)), and the
 * matching gradient.  h <= 0 is replaced by nu. */
void or_grad_hess(const or_problem* p, const double* mq, int64_t j, double nu, double* g_out, double* h_out) {
  double g = 0.0, h = 0.0;
  for (int64_t k = p->col_ptr[j]; k < p->col_ptr[j + 1]; ++k) {
    int64_t i = p->row_idx[k];
    double x = (double)p->val[k];
    double y = (double)p->y[i];
    if (p->loss == OR_LOSS_LOGISTIC) {
      double E = mq[i];
      double tau = (p->y[i] > 0) ? E / (1.0 + E) : 1.0 / (1.0 + E);
      g += (tau - 1.0) * y * x;
      h += tau * (1.0 - tau) * x * x;
    } else {
      double b = mq[i];
      if (b > 0.0) {
        g += -2.0 * y * x * b;
        h += 2.0 * x * x;
      }
    }
  }
  g *= p->c;
  h *= p->c;
  if (h <= 0.0) h = nu;
  *g_out = g;
  *h_out = h;
}

/* argmin_d  g d + h d^2 / 2 + |w + d|   (Eq. 4, closed form Eq. 5 with the
 * +/-1 terms in the branch conditions) */
double or_direction_l1(double g, double h, double w, double l1) {
  if (g + l1 <= h * w) return -(g + l1) / h;
  if (g - l1 >= h * w) return -(g - l1) / h;
  return -w;
}

double or_direction(double g, double h, double w) { return or_direction_l1(g, h, w, 1.0); }

/* Gradient and Hessian diagonal of the smooth part c L(w) + (l2/2)||w||^2 at
 * feature j (the loss's after the nu rule, plus l2 w_j and l2). */
static void smooth_grad_hess(const or_problem* p, const double* mq, int64_t j, double nu, double wj, double* g,
                             double* h) {
  or_grad_hess(p, mq, j, nu, g, h);
  if (p->l2 != 0.0) {
    *g += p->l2 * wj;
    *h += p->l2;
  }
}

/* Minimum-norm subgradient of the penalised objective at one feature. */
static double min_norm_v(double g, double wj, double l1) {
  if (wj > 0) return g + l1;
  if (wj < 0) return g - l1;
  return fabs(g) > l1 ? (g > 0 ? g - l1 : g + l1) : 0.0;
}

/* Change of the penalty of one feature when w_j moves by t. */
static double penalty_change(const or_problem* p, double wj, double t) {
  double r = p->l1 * (fabs(wj + t) - fabs(wj));
  if (p->l2 != 0.0) r += 0.5 * p->l2 * ((wj + t) * (wj + t) - wj * wj);
  return r;
}

/* Minimum-norm subgradient of F at w, l1 norm, with the gradient recomputed
 * from the maintained quantities for every feature. */
double or_kkt_l1(const or_problem* p, const double* w, const double* mq, double nu) {
  double s = 0.0;
  for (int64_t j = 0; j < p->m; ++j) {
    double g, h;
    smooth_grad_hess(p, mq, j, nu, w[j], &g, &h);
    s += fabs(min_norm_v(g, w[j], p->l1));
  }
  return s;
}

/* Loss change of sample i when w moves by a d (maintained form, Eq. 10 for
 * the logistic loss; the SVM analogue for Eq. 3).  Section 3.1 states that
 * Eq. 10 is the objective change of Eq. 6 itself; its logarithm
 * log((E e^u + 1) / (E e^u + e^u)) + [y = -1] u is evaluated here in forms
 * that do not cancel.  With p = E/(1+E) and s = 1/(1+E) the per-sample
 * change is log(p e^u + s) - [y = +1] u, written as
 *   log1p(p expm1(u)) - [y = +1] u   when E <= 1 (the log1p argument >= -1/2),
 *   log1p(s expm1(-u)) + [y = -1] u  when E > 1  (the same bound),
 * and, when |u| is too large for expm1, as a log-sum-exp of log p + u and
 * log s.  (Eq. 10's log-ratio taken literally loses every digit once
 * |w^T x_i| exceeds about 37: the ratio rounds to 0 or 1.) */
static double row_loss_change(const or_problem* p, double mq_i, int8_t y_i, double u /* a d^T x_i */) {
  if (p->loss == OR_LOSS_LOGISTIC) {
    const double E = mq_i;
    if (fabs(u) < 700.0) {
      if (E <= 1.0) return log1p(E / (1.0 + E) * expm1(u)) - (y_i > 0 ? u : 0.0);
      return log1p(expm1(-u) / (1.0 + E)) + (y_i < 0 ? u : 0.0);
    }
    const double lp = log(E) - log1p(E), ls = -log1p(E);
    const double a = lp + u, b = ls;
    const double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b))) - (y_i > 0 ? u : 0.0);
  } else {
    double bn = mq_i - (double)y_i * u;
    double a = bn > 0 ? bn * bn : 0.0;
    double b = mq_i > 0 ? mq_i * mq_i : 0.0;
    return a - b;
  }
}

/* The per-sample loss change above, exported for its pin tests. */
double or_loss_change(const or_problem* p, double mq_i, int y_i, double u) {
  return row_loss_change(p, mq_i, (int8_t)y_i, u);
}

/*
 * One PCDN inner iteration (Algorithm 3 body, with Algorithm 4) on bundle
 * B = bundle[0..P).  Updates w and mq in place.
 *   direct != 0: the Armijo test evaluates F(w + a d) - F(w) from scratch
 *                (Eq. 6); otherwise through the maintained quantities (Eq. 10).
 * Outputs (any may be NULL): g[P], h[P], d[P], Delta (Eq. 7), q, alpha, dF.
 * Returns OR_OK (step accepted), 1 when the line search reached q_max
 * (a = 0, nothing changes), 2 when every direction is zero (no line search;
 * q = 0, a = 1, dF = 0), or a negative error code.
 */
int or_bundle_step(const or_problem* p, const or_armijo* ar, double* w, double* mq, const int32_t* bundle,
                   int64_t P, int direct, double* g_out, double* h_out, double* d_out, double* Delta_out,
                   int32_t* q_out, double* alpha_out, double* dF_out) {
  double* g = (double*)malloc(sizeof(double) * (size_t)P);
  double* h = (double*)malloc(sizeof(double) * (size_t)P);
  double* d = (double*)malloc(sizeof(double) * (size_t)P);
  double* dx = (double*)calloc((size_t)(p->n > 0 ? p->n : 1), sizeof(double));
  if (!g || !h || !d || !dx) { free(g); free(h); free(d); free(dx); return OR_ENOMEM; }

  /* direction for every feature of the bundle (Algorithm 3, Eq. 9) */
  int any = 0;
  for (int64_t k = 0; k < P; ++k) {
    int64_t j = bundle[k];
    smooth_grad_hess(p, mq, j, ar->nu, w[j], &g[k], &h[k]);
    d[k] = or_direction_l1(g[k], h[k], w[j], p->l1);
    if (d[k] != 0.0) any = 1;
  }
  /* Delta = grad^T d + gamma d^T H d + ||w + d||_1 - ||w||_1   (Eq. 7) */
  double Delta = 0.0;
  {
    double lin = 0.0, quad = 0.0, l1 = 0.0;
    for (int64_t k = 0; k < P; ++k) {
      int64_t j = bundle[k];
      lin += g[k] * d[k];
      quad += h[k] * d[k] * d[k];
      l1 += p->l1 * (fabs(w[j] + d[k]) - fabs(w[j]));
    }
    Delta = lin + ar->gamma * quad + l1;
  }
  /* d^T x_i for every sample (Algorithm 4, first step) */
  for (int64_t k = 0; k < P; ++k) {
    if (d[k] == 0.0) continue;
    int64_t j = bundle[k];
    for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) dx[p->row_idx[e]] += d[k] * (double)p->val[e];
  }

  int32_t q = 0;
  double alpha = 1.0, dF = 0.0;
  int capped = 0;
  if (any) {
    double* wt = NULL;
    double F0 = 0.0;
    if (direct) {
      wt = (double*)malloc(sizeof(double) * (size_t)p->m);
      if (!wt) { free(g); free(h); free(d); free(dx); return OR_ENOMEM; }
      F0 = or_objective(p, w);
    }
    /* Armijo backtracking (Eq. 6): first q with dF(beta^q) <= sigma beta^q Delta */
    double a = 1.0;
    int accepted = 0;
    for (q = 0; q < ar->q_max; ++q) {
      if (direct) {
        memcpy(wt, w, sizeof(double) * (size_t)p->m);
        for (int64_t k = 0; k < P; ++k) wt[bundle[k]] += a * d[k];
        dF = or_objective(p, wt) - F0;
      } else {
        double Ls = 0.0;
        for (int64_t i = 0; i < p->n; ++i)
          if (dx[i] != 0.0) Ls += row_loss_change(p, mq[i], p->y[i], a * dx[i]);
        double r = 0.0;
        for (int64_t k = 0; k < P; ++k) r += penalty_change(p, w[bundle[k]], a * d[k]);
        dF = p->c * Ls + r;
      }
      if (dF <= ar->sigma * a * Delta) { accepted = 1; break; }
      a *= ar->beta;
    }
    free(wt);
    if (accepted) {
      alpha = a;
      /* w <- w + a d;  maintained quantities (Algorithm 4) */
      for (int64_t k = 0; k < P; ++k) w[bundle[k]] += alpha * d[k];
      for (int64_t i = 0; i < p->n; ++i) {
        if (dx[i] == 0.0) continue;
        if (p->loss == OR_LOSS_LOGISTIC) mq[i] *= exp(alpha * dx[i]);
        else mq[i] -= alpha * (double)p->y[i] * dx[i];
      }
    } else {
      capped = 1;
      q = ar->q_max;
      alpha = 0.0;
      dF = 0.0;
    }
  }

  if (!any) capped = 2;
  if (g_out) memcpy(g_out, g, sizeof(double) * (size_t)P);
  if (h_out) memcpy(h_out, h, sizeof(double) * (size_t)P);
  if (d_out) memcpy(d_out, d, sizeof(double) * (size_t)P);
  if (Delta_out) *Delta_out = Delta;
  if (q_out) *q_out = q;
  if (alpha_out) *alpha_out = alpha;
  if (dF_out) *dF_out = dF;
  free(g); free(h); free(d); free(dx);
  return capped;
}

/* Active set for shrinking (reading above): active[j] = 1 unless w_j = 0 and
 * |g_j| < l1 - M / s (the reading's bound 1 - M / s for the paper's penalty),
 * g the smooth part's gradient, M = max_j |v_j| with v the minimum-norm subgradient.
 * Returns the number of active features; *M_out gets M. */
int64_t or_active_set(const or_problem* p, const double* w, const double* mq, double nu, uint8_t* active,
                      double* M_out) {
  double* g = (double*)malloc(sizeof(double) * (size_t)p->m);
  if (!g) return -1;
  double M = 0.0;
  for (int64_t j = 0; j < p->m; ++j) {
    double h;
    smooth_grad_hess(p, mq, j, nu, w[j], &g[j], &h);
    const double v = min_norm_v(g[j], w[j], p->l1);
    if (fabs(v) > M) M = fabs(v);
  }
  const double bound = p->l1 - M / (double)p->n;
  int64_t count = 0;
  for (int64_t j = 0; j < p->m; ++j) {
    active[j] = (w[j] != 0.0 || fabs(g[j]) >= bound) ? 1 : 0;
    count += active[j];
  }
  free(g);
  if (M_out) *M_out = M;
  return count;
}

/*
 * Algorithm 3: outer iterations k = 0, 1, ...; in each, a fresh random
 * partition and a sequential walk over its bundles.  After every outer
 * iteration the maintained quantities are recomputed from z = Xw and the
 * relative minimum-norm-subgradient test decides convergence.
 *
 * w[m] is the start point on entry (the paper starts at 0) and the result on
 * exit.  bundle_limit >= 0 stops after that many bundles (timing samples).
 * Per-bundle and per-epoch traces are written when the buffers are given.
 */
int or_solve(const or_problem* p, const or_armijo* ar, int64_t P, double eps, uint64_t seed, int64_t max_epochs,
             int direct, int64_t bundle_limit, double* w, or_stats* st,
             int64_t trace_cap, int32_t* tr_q, double* tr_alpha, double* tr_Delta, double* tr_dF,
             int64_t epoch_cap, double* ep_kkt, double* ep_F, int shrink, int64_t* ep_active) {
  if (!p || !ar || !w || !st || P < 1 || P > p->m || !(eps > 0)) return OR_EINVAL;
  memset(st, 0, sizeof(*st));
  double* mq = (double*)malloc(sizeof(double) * (size_t)(p->n > 0 ? p->n : 1));
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->m);
  uint8_t* active = shrink ? (uint8_t*)malloc((size_t)p->m) : NULL;
  if (!mq || !perm || (shrink && !active)) { free(mq); free(perm); free(active); return OR_ENOMEM; }
  int rc = or_refresh(p, w, mq);
  if (rc) { free(mq); free(perm); free(active); return rc; }
  double kkt0 = or_kkt_l1(p, w, mq, ar->nu);
  st->kkt0 = kkt0;
  st->kkt_rel = kkt0 > 0 ? 1.0 : 0.0;
  int64_t nb = (p->m + P - 1) / P;
  int64_t tcount = 0;
  int stop_early = 0;
  if (kkt0 == 0.0) st->converged = 1;
  for (int64_t k = 0; k < max_epochs && !st->converged && !stop_early; ++k) {
    rc = or_permutation(seed, k, p->m, perm);
    if (rc) break;
    int64_t npos = p->m;
    if (shrink && k > 0) {  /* the random order restricted to the active set of the current w */
      const int64_t na = or_active_set(p, w, mq, ar->nu, active, NULL);
      if (na < 0) { rc = OR_ENOMEM; break; }
      npos = 0;
      for (int64_t t = 0; t < p->m; ++t)
        if (active[perm[t]]) perm[npos++] = perm[t];
    }
    if (k < epoch_cap && ep_active) ep_active[k] = npos;
    nb = (npos + P - 1) / P;
    for (int64_t t = 0; t < nb; ++t) {
      if (bundle_limit >= 0 && tcount >= bundle_limit) { stop_early = 1; break; }
      int64_t lo = t * P, hi = lo + P < npos ? lo + P : npos;
      int32_t q;
      double alpha, Delta, dF;
      int r = or_bundle_step(p, ar, w, mq, perm + lo, hi - lo, direct, NULL, NULL, NULL, &Delta, &q, &alpha, &dF);
      if (r < 0) { rc = r; stop_early = 1; break; }
      if (r == 1) st->ls_cap_hits++;
      if (r != 2) st->ls_steps += (r == 1) ? ar->q_max : q + 1;
      if (tcount < trace_cap) {
        if (tr_q) tr_q[tcount] = q;
        if (tr_alpha) tr_alpha[tcount] = alpha;
        if (tr_Delta) tr_Delta[tcount] = Delta;
        if (tr_dF) tr_dF[tcount] = dF;
      }
      ++tcount;
      st->bundles++;
      st->coord_updates += hi - lo;
    }
    if (stop_early) break;
    st->epochs = k + 1;
    or_refresh(p, w, mq);
    double kk = or_kkt_l1(p, w, mq, ar->nu);
    st->kkt_rel = kkt0 > 0 ? kk / kkt0 : 0.0;
    if (k < epoch_cap) {
      if (ep_kkt) ep_kkt[k] = st->kkt_rel;
      if (ep_F) ep_F[k] = or_objective(p, w);
    }
    if (st->kkt_rel <= eps) st->converged = 1;
  }
  st->F_final = or_objective(p, w);
  free(mq);
  free(perm);
  free(active);
  if (rc < 0) return rc;
  return st->converged ? OR_OK : OR_ENOTCONVERGED;
}

/* Algorithm 1 (CDN): one coordinate at a time with a 1-D Armijo search,
 * visiting features in the same random order as PCDN's partition.  Kept as a
 * separately written loop so that PCDN with P = 1 can be checked against it. */
int or_cdn_epoch(const or_problem* p, const or_armijo* ar, uint64_t seed, int64_t epoch, double* w, double* mq) {
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->m);
  if (!perm) return OR_ENOMEM;
  or_permutation(seed, epoch, p->m, perm);
  for (int64_t t = 0; t < p->m; ++t) {
    int64_t j = perm[t];
    double g, h;
    smooth_grad_hess(p, mq, j, ar->nu, w[j], &g, &h);
    double d = or_direction_l1(g, h, w[j], p->l1);
    if (d == 0.0) continue;
    /* same operation order as the bundle step with P = 1 */
    double Delta = (g * d + ar->gamma * (h * d * d)) + p->l1 * (fabs(w[j] + d) - fabs(w[j]));
    double a = 1.0;
    int ok = 0;
    for (int q = 0; q < ar->q_max; ++q) {
      double Ls = 0.0;
      for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
        int64_t i = p->row_idx[e];
        double dx = d * (double)p->val[e];
        if (dx != 0.0) Ls += row_loss_change(p, mq[i], p->y[i], a * dx);
      }
      double dF = p->c * Ls + penalty_change(p, w[j], a * d);
      if (dF <= ar->sigma * a * Delta) { ok = 1; break; }
      a *= ar->beta;
    }
    if (!ok) continue;
    w[j] += a * d;
    for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
      int64_t i = p->row_idx[e];
      double dx = d * (double)p->val[e];
      if (dx == 0.0) continue;
      if (p->loss == OR_LOSS_LOGISTIC) mq[i] *= exp(a * dx);
      else mq[i] -= a * (double)p->y[i] * dx;
    }
  }
  free(perm);
  return OR_OK;
}
