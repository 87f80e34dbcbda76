/*
 * Seeded synthetic sparse classification data (inputs only).
 *
 * This file produces the design matrix X (CSR and CSC), the labels y and the
 * planted weight vector w*.  It holds none of the solver's arithmetic: it is
 * the one module that both the CPU oracle tests and the CUDA path read their
 * inputs from.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Every row draws from its own stream whose
 * start state is a hash of (seed, stream tag, row), so the output does not
 * depend on how many threads run the generator.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no -ffast-math, so
 * the same inputs come out on x86-64 and aarch64 up to libm rounding).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GEN_OK 0
#define GEN_EINVAL -1
#define GEN_ENOMEM -2

static inline uint64_t sm64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* start state of stream (seed, tag, idx) */
static inline uint64_t stream_state(uint64_t seed, uint64_t tag, uint64_t idx) {
  uint64_t s = seed ^ (tag * 0xD1B54A32D192ED03ULL);
  uint64_t a = sm64_next(&s);
  uint64_t t = a ^ (idx * 0x9E3779B97F4A7C15ULL);
  return sm64_next(&t);
}

/* uniform in (0, 1): 53 random bits, never 0 */
static inline double u01(uint64_t* s) {
  return ((double)(sm64_next(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static inline uint64_t below(uint64_t* s, uint64_t bound) {
  /* multiply-shift range reduction */
  return (uint64_t)(((unsigned __int128)sm64_next(s) * bound) >> 64);
}

static double std_normal(uint64_t* s) {
  /* Box-Muller, one of the pair */
  double u1 = u01(s), u2 = u01(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static int64_t poisson_inv(uint64_t* s, double lam) {
  if (lam > 500.0) {
    /* exp(-lam) underflows beyond ~745: draw the sum of independent Poisson pieces of mean <= 500,
       which is Poisson(lam) exactly */
    const int pieces = (int)ceil(lam / 500.0);
    int64_t k = 0;
    for (int i = 0; i < pieces; ++i) k += poisson_inv(s, lam / pieces);
    return k;
  }
  /* inversion by sequential search */
  double u = u01(s);
  double p = exp(-lam), F = p;
  int64_t k = 0, kmax = (int64_t)(10.0 * lam + 50.0);
  while (u > F && k < kmax) {
    ++k;
    p *= lam / (double)k;
    F += p;
  }
  return k;
}

enum { TAG_ROWS = 1, TAG_RANKS = 2, TAG_WSTAR = 3, TAG_FLIP = 4, TAG_VALS = 5 };

/* Vose alias table over weights wt[0..m) */
static int build_alias(const double* wt, int64_t m, double* prob, int64_t* alias) {
  double tot = 0;
  for (int64_t j = 0; j < m; ++j) tot += wt[j];
  int64_t* small = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  int64_t* large = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  double* sc = (double*)malloc(sizeof(double) * (size_t)m);
  if (!small || !large || !sc) { free(small); free(large); free(sc); return GEN_ENOMEM; }
  int64_t ns = 0, nl = 0;
  for (int64_t j = 0; j < m; ++j) {
    sc[j] = wt[j] * (double)m / tot;
    if (sc[j] < 1.0) small[ns++] = j; else large[nl++] = j;
  }
  while (ns > 0 && nl > 0) {
    int64_t a = small[--ns], g = large[--nl];
    prob[a] = sc[a];
    alias[a] = g;
    sc[g] = (sc[g] + sc[a]) - 1.0;
    if (sc[g] < 1.0) small[ns++] = g; else large[nl++] = g;
  }
  while (nl > 0) { int64_t g = large[--nl]; prob[g] = 1.0; alias[g] = g; }
  while (ns > 0) { int64_t a = small[--ns]; prob[a] = 1.0; alias[a] = a; }
  free(small); free(large); free(sc);
  return GEN_OK;
}

/*
 * Row-pattern generation, pass 1 (lengths) and pass 2 (columns).
 * kind 0: every entry present independently with probability `density`
 *         (geometric skips along the row).
 * kind 1: row length max(1, Poisson(row_mean)); columns drawn without
 *         replacement with probability proportional to rank^-zipf_s, the
 *         rank of each column being a random permutation of [0, m).
 */
typedef struct {
  int64_t n, m;
  int kind;
  double density, row_mean, zipf_s;
  int value_kind; /* 0: |N(0,1)|, 1: log(1+c), c~Poisson(2)|c>=1, times idf */
  int64_t wstar_nnz;
  double flip_frac;
  uint64_t seed;
} gen_spec;

typedef struct {
  int64_t nnz;
  int64_t* row_ptr; /* n+1 */
  int32_t* col_idx; /* nnz */
  float* rval;      /* nnz, CSR values */
  int64_t* col_ptr; /* m+1 */
  int32_t* row_idx; /* nnz */
  float* cval;      /* nnz, CSC values */
  int8_t* y;        /* n */
  int32_t* wstar_idx; /* wstar_nnz */
  double* wstar_val;  /* wstar_nnz */
} gen_out;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Draw k distinct values from [0, m) (Floyd's algorithm), sorted ascending. */
static int sample_distinct(uint64_t* s, int64_t m, int64_t k, int32_t* out) {
  /* simple open-addressing set for k << m */
  int64_t cap = 16;
  while (cap < 4 * k) cap <<= 1;
  int64_t* tab = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  if (!tab) return GEN_ENOMEM;
  for (int64_t i = 0; i < cap; ++i) tab[i] = -1;
  int64_t cnt = 0;
  for (int64_t j = m - k; j < m; ++j) {
    int64_t t = (int64_t)below(s, (uint64_t)(j + 1));
    int64_t v = t;
    /* if t already present, use j */
    int64_t h = (t * 0x9E3779B1LL) & (cap - 1);
    int present = 0;
    while (tab[h] != -1) { if (tab[h] == t) { present = 1; break; } h = (h + 1) & (cap - 1); }
    if (present) {
      v = j;
      h = (j * 0x9E3779B1LL) & (cap - 1);
      while (tab[h] != -1) h = (h + 1) & (cap - 1);
    }
    tab[h] = v;
    out[cnt++] = (int32_t)v;
  }
  free(tab);
  qsort(out, (size_t)k, sizeof(int32_t), cmp_i32);
  return GEN_OK;
}

int gen_free(gen_out* o) {
  free(o->row_ptr); free(o->col_idx); free(o->rval);
  free(o->col_ptr); free(o->row_idx); free(o->cval);
  free(o->y); free(o->wstar_idx); free(o->wstar_val);
  memset(o, 0, sizeof(*o));
  return GEN_OK;
}

int gen_generate(const gen_spec* sp, gen_out* o) {
  memset(o, 0, sizeof(*o));
  const int64_t n = sp->n, m = sp->m;
  if (n <= 0 || m <= 0 || m > 2147483647LL || n > 2147483647LL) return GEN_EINVAL;
  if (sp->kind == 0 && !(sp->density > 0 && sp->density < 1)) return GEN_EINVAL;
  if (sp->kind == 1 && !(sp->row_mean > 0 && sp->row_mean <= 0.25 * (double)m && sp->zipf_s > 0)) return GEN_EINVAL;
  if (sp->wstar_nnz < 0 || sp->wstar_nnz > m || sp->flip_frac < 0 || sp->flip_frac > 1) return GEN_EINVAL;
  if (sp->kind != 0 && sp->kind != 1) return GEN_EINVAL;

  int rc = GEN_OK;
  o->row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!o->row_ptr) return GEN_ENOMEM;

  /* ---- column-rank alias table for kind 1 ---- */
  double* aprob = NULL; int64_t* aalias = NULL; int32_t* rank_to_col = NULL;
  if (sp->kind == 1) {
    double* wt = (double*)malloc(sizeof(double) * (size_t)m);
    aprob = (double*)malloc(sizeof(double) * (size_t)m);
    aalias = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    rank_to_col = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    if (!wt || !aprob || !aalias || !rank_to_col) { free(wt); rc = GEN_ENOMEM; goto fail; }
    for (int64_t r = 0; r < m; ++r) wt[r] = pow((double)(r + 1), -sp->zipf_s);
    rc = build_alias(wt, m, aprob, aalias);
    free(wt);
    if (rc) goto fail;
    /* random permutation rank -> column (Fisher-Yates) */
    uint64_t s = stream_state(sp->seed, TAG_RANKS, 0);
    for (int64_t r = 0; r < m; ++r) rank_to_col[r] = (int32_t)r;
    for (int64_t i = m - 1; i > 0; --i) {
      int64_t j = (int64_t)below(&s, (uint64_t)(i + 1));
      int32_t t = rank_to_col[i]; rank_to_col[i] = rank_to_col[j]; rank_to_col[j] = t;
    }
  }

  /* ---- pass 1: row lengths ---- */
  {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      uint64_t s = stream_state(sp->seed, TAG_ROWS, (uint64_t)i);
      int64_t k;
      if (sp->kind == 0) {
        /* count entries of the geometric-skip walk */
        double lq = log1p(-sp->density);
        int64_t c = 0, j = -1;
        for (;;) {
          double u = u01(&s);
          int64_t skip = (int64_t)floor(log(u) / lq);
          j += skip + 1;
          if (j >= m) break;
          ++c;
        }
        k = c;
      } else {
        k = poisson_inv(&s, sp->row_mean);
        if (k < 1) k = 1;
        if (k > m) k = m;
      }
      o->row_ptr[i + 1] = k;
    }
  }
  for (int64_t i = 0; i < n; ++i) o->row_ptr[i + 1] += o->row_ptr[i];
  o->nnz = o->row_ptr[n];
  {
    const int64_t nnz = o->nnz;
    o->col_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    o->rval = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    if (!o->col_idx || !o->rval) { rc = GEN_ENOMEM; goto fail; }
  }

  /* ---- pass 2: columns and raw values (replays the same streams) ---- */
  {
    int fail_flag = 0;
#pragma omp parallel
    {
      int32_t* stamp = NULL;
      if (sp->kind == 1) {
        stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
        if (!stamp) {
#pragma omp atomic write
          fail_flag = 1;
        } else {
          for (int64_t j = 0; j < m; ++j) stamp[j] = -1;
        }
      }
#pragma omp for schedule(dynamic, 1024)
      for (int64_t i = 0; i < n; ++i) {
        if (sp->kind == 1 && !stamp) continue;
        uint64_t s = stream_state(sp->seed, TAG_ROWS, (uint64_t)i);
        int64_t p0 = o->row_ptr[i], k = o->row_ptr[i + 1] - p0;
        int32_t* cols = o->col_idx + p0;
        if (sp->kind == 0) {
          double lq = log1p(-sp->density);
          int64_t c = 0, j = -1;
          for (;;) {
            double u = u01(&s);
            int64_t skip = (int64_t)floor(log(u) / lq);
            j += skip + 1;
            if (j >= m) break;
            cols[c++] = (int32_t)j;
          }
        } else {
          (void)poisson_inv(&s, sp->row_mean); /* replay the length draw */
          int64_t c = 0;
          while (c < k) {
            int64_t r = (int64_t)below(&s, (uint64_t)m);
            if (u01(&s) >= aprob[r]) r = aalias[r];
            int32_t col = rank_to_col[r];
            if (stamp[col] == (int32_t)i) continue;
            stamp[col] = (int32_t)i;
            cols[c++] = col;
          }
          qsort(cols, (size_t)k, sizeof(int32_t), cmp_i32);
        }
        /* raw values from a separate stream */
        uint64_t sv = stream_state(sp->seed, TAG_VALS, (uint64_t)i);
        for (int64_t c = 0; c < k; ++c) {
          double v;
          if (sp->value_kind == 0) {
            v = fabs(std_normal(&sv));
          } else {
            int64_t cnt;
            do { cnt = poisson_inv(&sv, 2.0); } while (cnt < 1);
            v = log1p((double)cnt);
          }
          o->rval[p0 + c] = (float)v;
        }
      }
      free(stamp);
    }
    if (fail_flag) { rc = GEN_ENOMEM; goto fail; }
  }
  free(aprob); aprob = NULL; free(aalias); aalias = NULL; free(rank_to_col); rank_to_col = NULL;

  /* ---- document frequencies, idf weights, row normalisation ---- */
  {
    const int64_t nnz = o->nnz;
    o->col_ptr = (int64_t*)calloc((size_t)m + 1, sizeof(int64_t));
    if (!o->col_ptr) { rc = GEN_ENOMEM; goto fail; }
    for (int64_t p = 0; p < nnz; ++p) o->col_ptr[o->col_idx[p] + 1]++;
    if (sp->value_kind == 1) {
      double* idf = (double*)malloc(sizeof(double) * (size_t)m);
      if (!idf) { rc = GEN_ENOMEM; goto fail; }
      for (int64_t j = 0; j < m; ++j) {
        int64_t df = o->col_ptr[j + 1];
        idf[j] = df > 0 ? log(1.0 + (double)n / (double)df) : 0.0;
      }
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < nnz; ++p) o->rval[p] = (float)((double)o->rval[p] * idf[o->col_idx[p]]);
      free(idf);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double ss = 0;
      for (int64_t p = o->row_ptr[i]; p < o->row_ptr[i + 1]; ++p) ss += (double)o->rval[p] * (double)o->rval[p];
      if (ss > 0) {
        double inv = 1.0 / sqrt(ss);
        for (int64_t p = o->row_ptr[i]; p < o->row_ptr[i + 1]; ++p) o->rval[p] = (float)((double)o->rval[p] * inv);
      }
    }
    /* ---- CSC by stable counting sort (rows stay ascending in each column) ---- */
    for (int64_t j = 0; j < m; ++j) o->col_ptr[j + 1] += o->col_ptr[j];
    o->row_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    o->cval = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    if (!o->row_idx || !o->cval || !fill) { free(fill); rc = GEN_ENOMEM; goto fail; }
    memcpy(fill, o->col_ptr, sizeof(int64_t) * (size_t)m);
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t p = o->row_ptr[i]; p < o->row_ptr[i + 1]; ++p) {
        int64_t q = fill[o->col_idx[p]]++;
        o->row_idx[q] = (int32_t)i;
        o->cval[q] = o->rval[p];
      }
    }
    free(fill);
  }

  /* ---- planted w*, labels y = sign(X w*) (sign(0)=+1), exact flips ---- */
  {
    int64_t ks = sp->wstar_nnz;
    o->wstar_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ks > 0 ? ks : 1));
    o->wstar_val = (double*)malloc(sizeof(double) * (size_t)(ks > 0 ? ks : 1));
    o->y = (int8_t*)malloc((size_t)n);
    double* wd = (double*)calloc((size_t)m, sizeof(double));
    if (!o->wstar_idx || !o->wstar_val || !o->y || !wd) { free(wd); rc = GEN_ENOMEM; goto fail; }
    uint64_t s = stream_state(sp->seed, TAG_WSTAR, 0);
    if (ks > 0 && (rc = sample_distinct(&s, m, ks, o->wstar_idx))) { free(wd); goto fail; }
    for (int64_t t = 0; t < ks; ++t) {
      o->wstar_val[t] = std_normal(&s);
      wd[o->wstar_idx[t]] = o->wstar_val[t];
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double dot = 0;
      for (int64_t p = o->row_ptr[i]; p < o->row_ptr[i + 1]; ++p) dot += (double)o->rval[p] * wd[o->col_idx[p]];
      o->y[i] = dot >= 0 ? (int8_t)1 : (int8_t)-1;
    }
    free(wd);
    int64_t nflip = (int64_t)floor(sp->flip_frac * (double)n + 0.5);
    if (nflip > 0) {
      int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)nflip);
      if (!fl) { rc = GEN_ENOMEM; goto fail; }
      uint64_t sf = stream_state(sp->seed, TAG_FLIP, 0);
      if ((rc = sample_distinct(&sf, n, nflip, fl))) { free(fl); goto fail; }
      for (int64_t t = 0; t < nflip; ++t) o->y[fl[t]] = (int8_t)(-o->y[fl[t]]);
      free(fl);
    }
  }
  return GEN_OK;

fail:
  free(aprob); free(aalias); free(rank_to_col);
  gen_free(o);
  return rc;
}

int gen_nthreads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
