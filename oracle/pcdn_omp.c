/*
 * PCDN on all host cores (OpenMP) -- a CPU BASELINE, TEST INFRASTRUCTURE ONLY.
 *
 * The paper's own parallel scheme (Section 3.1 and Section 5.1: a shared-memory implementation
 * whose threads share the work of a bundle): the directions of the bundle's features in parallel
 * (Eq. 9, Eq. 5); d^T x_i, the line search (Eq. 6 with Eq. 10) and the updates (Algorithm 4) with
 * the samples split over the threads (each thread sums its own rows' entries of the bundle's
 * columns, found by binary search, and lists its touched rows), so no atomics and no scan of all
 * samples.  Same partitions (Eq. 8), Armijo rule and stop test as the oracle, whose
 * per-feature routines it reuses; the order of the floating-point sums differs (atomic adds and
 * parallel reductions), so results agree with the oracle to rounding, not bitwise.
 *
 * Only bench.py's CPU-baseline leg and its own CPU test load this code.
 */
#include <omp.h>

#include "pcdn_oracle.c"

typedef struct {
  double* dx;      /* [n] d^T x_i of the bundle, zero outside it */
  uint8_t* mark;   /* [n] 1 for a touched sample */
  int32_t* rows;   /* [n] touched samples, thread t's in [lo_t, lo_t + cnt_t) with lo_t its first row */
  int64_t* cnt;    /* [threads] touched samples listed by each thread */
  int threads;
} omp_ws;

/* Rows of thread t: [n t / T, n (t + 1) / T). */
static int64_t row_lo(const or_problem* p, int t, int T) { return p->n * (int64_t)t / T; }

/* First entry of column j at or after row r (rows ascending within a column). */
static int64_t col_lower(const or_problem* p, int64_t j, int64_t r) {
  int64_t a = p->col_ptr[j], b = p->col_ptr[j + 1];
  while (a < b) {
    const int64_t mid = a + (b - a) / 2;
    if (p->row_idx[mid] < r) a = mid + 1;
    else b = mid;
  }
  return a;
}

static int omp_bundle_step(const or_problem* p, const or_armijo* ar, double* w, double* mq, const int32_t* bundle,
                           int64_t P, omp_ws* ws, double* g, double* h, double* d, int32_t* q_out) {
  int any = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : any)
  for (int64_t k = 0; k < P; ++k) {
    const int64_t j = bundle[k];
    or_grad_hess(p, mq, j, ar->nu, &g[k], &h[k]);
    d[k] = or_direction(g[k], h[k], w[j]);
    if (d[k] != 0.0) any = 1;
  }
  double lin = 0.0, quad = 0.0, l1 = 0.0;
  for (int64_t k = 0; k < P; ++k) {
    const int64_t j = bundle[k];
    lin += g[k] * d[k];
    quad += h[k] * d[k] * d[k];
    l1 += fabs(w[j] + d[k]) - fabs(w[j]);
  }
  const double Delta = lin + ar->gamma * quad + l1;
  *q_out = 0;
  if (!any) return 2;
  const int T = ws->threads;
  /* d^T x_i: each thread sums the entries of its own rows (no atomics) and lists them */
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num();
    const int64_t lo = row_lo(p, t, T), hi = row_lo(p, t + 1, T);
    int64_t c = 0;
    for (int64_t k = 0; k < P; ++k) {
      if (d[k] == 0.0) continue;
      const int64_t j = bundle[k];
      for (int64_t e = col_lower(p, j, lo); e < p->col_ptr[j + 1] && p->row_idx[e] < hi; ++e) {
        const int32_t i = p->row_idx[e];
        ws->dx[i] += d[k] * (double)p->val[e];
        if (!ws->mark[i]) {
          ws->mark[i] = 1;
          ws->rows[lo + c++] = i;
        }
      }
    }
    ws->cnt[t] = c;
  }
  double a = 1.0;
  int accepted = 0;
  int32_t q;
  for (q = 0; q < ar->q_max; ++q) {
    double Ls = 0.0;
#pragma omp parallel num_threads(T) reduction(+ : Ls)
    {
      const int t = omp_get_thread_num();
      const int64_t lo = row_lo(p, t, T);
      for (int64_t r = 0; r < ws->cnt[t]; ++r) {
        const int32_t i = ws->rows[lo + r];
        if (ws->dx[i] != 0.0) Ls += row_loss_change(p, mq[i], p->y[i], a * ws->dx[i]);
      }
    }
    double rr = 0.0;
    for (int64_t k = 0; k < P; ++k) {
      const int64_t j = bundle[k];
      rr += fabs(w[j] + a * d[k]) - fabs(w[j]);
    }
    const double dF = p->c * Ls + rr;
    if (dF <= ar->sigma * a * Delta) {
      accepted = 1;
      break;
    }
    a *= ar->beta;
  }
  if (accepted) {
    for (int64_t k = 0; k < P; ++k) w[bundle[k]] += a * d[k];
  }
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num();
    const int64_t lo = row_lo(p, t, T);
    for (int64_t r = 0; r < ws->cnt[t]; ++r) {
      const int32_t i = ws->rows[lo + r];
      if (accepted && ws->dx[i] != 0.0) {
        if (p->loss == OR_LOSS_LOGISTIC) mq[i] *= exp(a * ws->dx[i]);
        else mq[i] -= a * (double)p->y[i] * ws->dx[i];
      }
      ws->dx[i] = 0.0;
      ws->mark[i] = 0;
    }
  }
  *q_out = accepted ? q : ar->q_max;
  return accepted ? 0 : 1;
}

/* The maintained quantities from z = Xw, columns in parallel (atomic adds into z). */
static int omp_refresh(const or_problem* p, const double* w, double* mq) {
  double* z = (double*)calloc((size_t)(p->n > 0 ? p->n : 1), sizeof(double));
  if (!z) return OR_ENOMEM;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < p->m; ++j) {
    if (w[j] == 0.0) continue;
    for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
      const double v = (double)p->val[e] * w[j];
#pragma omp atomic
      z[p->row_idx[e]] += v;
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < p->n; ++i)
    mq[i] = (p->loss == OR_LOSS_LOGISTIC) ? exp(z[i]) : 1.0 - (double)p->y[i] * z[i];
  free(z);
  return OR_OK;
}

/* ||v||_1 of the minimum-norm subgradient, features in parallel. */
static double omp_kkt_l1(const or_problem* p, const double* w, const double* mq, double nu) {
  double s = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : s)
  for (int64_t j = 0; j < p->m; ++j) {
    double g, h;
    or_grad_hess(p, mq, j, nu, &g, &h);
    double v;
    if (w[j] > 0) v = g + 1.0;
    else if (w[j] < 0) v = g - 1.0;
    else v = fabs(g) > 1.0 ? (g > 0 ? g - 1.0 : g + 1.0) : 0.0;
    s += fabs(v);
  }
  return s;
}

int or_omp_threads(void) { return omp_get_max_threads(); }

/* Algorithm 3 as or_solve (same partitions, Armijo rule, stop test), bundles stepped with the
 * parallel scheme above.  bundle_limit >= 0 stops after that many bundles (timing samples). */
int or_solve_omp(const or_problem* p, const or_armijo* ar, int64_t P, double eps, uint64_t seed, int64_t max_epochs,
                 int64_t bundle_limit, double* w, or_stats* st) {
  if (!p || !ar || !w || !st || P < 1 || P > p->m || !(eps > 0)) return OR_EINVAL;
  if (p->l1 != 1.0 || p->l2 != 0.0) return OR_EINVAL; /* the paper's penalty only */
  memset(st, 0, sizeof(*st));
  const size_t n1 = (size_t)(p->n > 0 ? p->n : 1);
  double* mq = (double*)malloc(sizeof(double) * n1);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->m);
  double* g = (double*)malloc(sizeof(double) * (size_t)P);
  double* h = (double*)malloc(sizeof(double) * (size_t)P);
  double* d = (double*)malloc(sizeof(double) * (size_t)P);
  omp_ws ws;
  ws.threads = omp_get_max_threads();
  if (ws.threads < 1) ws.threads = 1;
  ws.dx = (double*)calloc(n1, sizeof(double));
  ws.mark = (uint8_t*)calloc(n1, 1);
  ws.rows = (int32_t*)malloc(sizeof(int32_t) * n1);
  ws.cnt = (int64_t*)calloc((size_t)ws.threads, sizeof(int64_t));
  int rc = OR_OK;
  if (!mq || !perm || !g || !h || !d || !ws.dx || !ws.mark || !ws.rows || !ws.cnt) rc = OR_ENOMEM;
  if (!rc) rc = omp_refresh(p, w, mq);
  double kkt0 = 0.0;
  if (!rc) {
    kkt0 = omp_kkt_l1(p, w, mq, ar->nu);
    st->kkt0 = kkt0;
    st->kkt_rel = kkt0 > 0 ? 1.0 : 0.0;
    if (kkt0 == 0.0) st->converged = 1;
  }
  const int64_t nb = (p->m + P - 1) / P;
  int64_t tcount = 0;
  int stop_early = 0;
  for (int64_t k = 0; !rc && k < max_epochs && !st->converged && !stop_early; ++k) {
    rc = or_permutation(seed, k, p->m, perm);
    if (rc) break;
    for (int64_t t = 0; t < nb; ++t) {
      if (bundle_limit >= 0 && tcount >= bundle_limit) {
        stop_early = 1;
        break;
      }
      const int64_t lo = t * P, hi = lo + P < p->m ? lo + P : p->m;
      int32_t q;
      const int r = omp_bundle_step(p, ar, w, mq, perm + lo, hi - lo, &ws, g, h, d, &q);
      if (r == 1) st->ls_cap_hits++;
      if (r != 2) st->ls_steps += (r == 1) ? ar->q_max : q + 1;
      ++tcount;
      st->bundles++;
      st->coord_updates += hi - lo;
    }
    if (stop_early) break;
    st->epochs = k + 1;
    rc = omp_refresh(p, w, mq);
    if (rc) break;
    const double kk = omp_kkt_l1(p, w, mq, ar->nu);
    st->kkt_rel = kkt0 > 0 ? kk / kkt0 : 0.0;
    if (st->kkt_rel <= eps) st->converged = 1;
  }
  if (!rc) st->F_final = or_objective(p, w);
  free(mq); free(perm); free(g); free(h); free(d); free(ws.dx); free(ws.mark); free(ws.rows); free(ws.cnt);
  if (rc < 0) return rc;
  return st->converged ? OR_OK : OR_ENOTCONVERGED;
}
