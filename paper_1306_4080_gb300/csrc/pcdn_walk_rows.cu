// Bundle walker on the row-sorted layout (pcdn_rows.cu): one persistent launch steps a run of
// bundles of one outer iteration (Algorithm 3's inner loop with Algorithm 4), every thread block
// in lockstep, with two grid barriers per bundle on the usual path.
//
// Per bundle t (positions [tP, min((t+1)P, npos)) of the partition's feature order):
//   A  column pass.  The bundle's column work items (a column, or a chunk of at most kChunk
//      nonzeros of a long column) are split over the blocks in contiguous runs of balanced nonzero
//      count.  A block stages a batch of items and their row indices and values (16-byte copies),
//      gathers each entry's per-sample coefficient pair, reduces g_j, h_j (Eq. 11 / generalised
//      Hessian) one warp per item and forms d_j (Eq. 5) one thread per item.  A column cut over
//      several blocks: each block sums its own chunks in order and publishes one partial sum; the
//      block whose publication completes the column sums the partials in block order and forms
//      d_j.  Nothing in this phase waits for another block.
//   -- barrier 1 (its counter also carries "some block has a nonzero direction")
//   B  line search.  Each block owns the samples whose row segments start in its share of the
//      bundle's row-sorted entries.  One thread per sample sums d^T x_i over its segment in a fixed
//      order (no atomics), evaluates its loss change for the pass's step sizes beta^q (Eq. 10) and,
//      on the first pass, writes the sample's state after the full step alpha = 1 (Algorithm 4's
//      update), keeping the old value aside.  A block also sums Delta's parts (Eq. 7) and the
//      penalty change of each step over a fixed slice of the bundle's positions.  Per-block partial
//      sums go to global memory.
//   -- barrier 2; then every block sums the partials in block order (identical sums in every block,
//      the same bits run to run) and takes the same decision (Eq. 6).
//   If the full step is accepted (almost every bundle), the samples already hold their new state:
//   the blocks update w_B and go on to the next bundle.  Otherwise the blocks evaluate further step
//   sizes from the kept state, then write the accepted step's state (or the old state at the cap),
//   and a third barrier closes the bundle.
// A bundle whose directions are all zero ends after barrier 1.
//
// Every sum has a fixed order: d^T x_i sequential over the row's entries, lane trees, warps and
// blocks in index order.  Results are repeatable bit for bit for a given grid size.
//
// Precision.  FP64 mode computes in FP64.  Mixed mode keeps X, g, h, d, d^T x and the per-sample
// line-search remainders in FP32 and sums Delta, the line-search sums and the penalty changes in
// FP64; the maintained quantities and w stay FP64.

#include "pcdn_internal.cuh"

namespace pcdn {
namespace rows {

constexpr int kBCap = 2048;      // row-sorted entries staged per round
constexpr int kMaxGrid = 512;    // blocks of a walk (a bundle's block plan is staged in shared memory)
constexpr int kAlphaTab = 64;
constexpr int kFinCap = kICap;   // split columns a block can finish in one batch
constexpr int kFBad = 3 + 2 * kMaxK;  // partial field: a speculative update left the usable range

template <int PREC> using GHT = typename std::conditional<PREC == 0, double, float>::type;

enum { kFirst = 0, kEval = 1, kApply = 2 };

struct FxSlot {
  long long l0, l1, l2;
  unsigned fl;
};

template <int PREC>
struct Shared {
  int abort;
  int has_nz;
  int nonzero;
  int scan_tot[kWalkWarps];
  int pf_ready, pf_nb, pf_eb;
  int n_split, n_fin;
  // the block's open run of chunks of a split column (run_kl < 0: none)
  int32_t run_kl, run_nch, run_chunk0, run_cnt;
  int64_t run_gi0;
  double run_g, run_h, run_w;
  // columns whose partial sums this block completed in the current batch
  int32_t fin_kl[kFinCap], fin_nch[kFinCap];
  int64_t fin_c0[kFinCap];
  double fin_w[kFinCap];
  int32_t split_j[kICap];
  Decision dec;
  double atab[kAlphaTab];
  float atab_f[kAlphaTab];
  double tot[kPartStride];
  double dparts[3];
  double dred[kWalkWarps];
  FxSlot fxs[kWalkWarps][kPartStride];
  int64_t plan_row[kMaxGrid + 1];  // the bundle's block plan of column items
  // phase A staging
  __align__(16) Item items[kICap];
  int32_t ioff[kICap + 1];  // slots of item j start at ioff[j] (a multiple of 4); its data at + (start & 3)
  __align__(16) int32_t row[kECap];
  __align__(16) float x[kECap];
  // the batch's coefficient pairs (phase A); the round's d of every entry (phase B)
  union {
    RecT<PREC> rec[kECap];
    typename std::conditional<PREC == 0, double, float>::type dv[kBCap];
  } u;
  GHT<PREC> g[kICap];
  GHT<PREC> h[kICap];
  // phase B staging: one round of the block's row-sorted entries
  int64_t b_cur;  // first entry staged
  int b_head;     // shared-memory index of entry b_cur
  int b_n;        // entries staged
  __align__(16) int32_t b_row[kBCap + 8];
  __align__(16) int32_t b_k[kBCap + 8];
  __align__(16) float b_val[kBCap + 8];
  int32_t rstart[kBCap + 2];
};

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16_zfill_stream(void* dst, const void* src, int bytes, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes), "l"(pol)
               : "memory");
}

// Inclusive block-wide scan of one int per thread.
template <class SH>
__device__ __forceinline__ int block_scan_incl(SH& sh, int v) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) sh.scan_tot[wib] = x;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < wib; ++w) off += sh.scan_tot[w];
  __syncthreads();
  return x + off;
}

// Column sums of one item: FP64 in FP64 mode, FP32 in mixed mode.
template <int PREC> struct ColAcc;
template <> struct ColAcc<0> {
  double g = 0.0, h = 0.0;
  __device__ __forceinline__ void add(float x, const RecT<0>& r) {
    const double xd = (double)x;
    g = fma(xd, r.cg, g);
    h = fma(xd * xd, r.ch, h);
  }
  __device__ __forceinline__ void reduce() {
    g = warp_sum(g);
    h = warp_sum(h);
  }
};
template <> struct ColAcc<1> {
  float g = 0.0f, h = 0.0f;
  __device__ __forceinline__ void add(float x, const RecT<1>& r) {
    g = fmaf(x, r.cg, g);
    h = fmaf(x * x, r.ch, h);
  }
  __device__ __forceinline__ void reduce() {
    g = warp_sum_f(g);
    h = warp_sum_f(h);
  }
};

// The smooth part's g, h from the column sums (times c, h <= 0 replaced by nu, plus l2 w_j and l2)
// and d (Eq. 5 with the penalty's l1); writes gk, hk, dk (and dkf) of position kl in parity half
// `par`.  Mixed mode works in FP32 and keeps d = -w exact, so that a coordinate set to zero is zero.
template <int PREC>
__device__ __forceinline__ double finalize(const WalkParams& p, int par, int32_t kl, GHT<PREC> g, GHT<PREC> h,
                                           double wj) {
  double d;
  if constexpr (PREC == 0) {
    g *= p.c;
    h *= p.c;
    if (h <= 0.0) h = p.nu;
    if (p.l2 != 0.0) {
      g += p.l2 * wj;
      h += p.l2;
    }
    d = newton_direction(g, h, wj, p.l1);
  } else {
    g *= p.c_f;
    h *= p.c_f;
    if (h <= 0.0f) h = p.nu_f;
    const float wf = (float)wj;
    if (p.l2 != 0.0) {
      g += p.l2_f * wf;
      h += p.l2_f;
    }
    d = newton_direction_f(g, h, wf, wj, p.l1_f);
  }
  const int64_t o = (int64_t)par * p.P_cap + kl;
  p.gk[o] = (double)g;
  p.hk[o] = (double)h;
  p.dk[o] = d;
  if constexpr (PREC == 1) p.dkf[o] = (float)d;
  if (!isfinite((double)g) || !isfinite((double)h) || !isfinite(d)) atomicOr(p.err, kErrNumeric);
  return d;
}

// ---------------------------------------------------------------- phase A staging
template <class SH>
__device__ __forceinline__ void stage_items_async(const WalkParams& p, SH& sh, int64_t i, int n) {
  for (int k = threadIdx.x; k < 2 * n; k += kWalkThreads)
    cp_async16(reinterpret_cast<char*>(&sh.items[k >> 1]) + 16 * (k & 1),
               reinterpret_cast<const char*>(p.items + i + (k >> 1)) + 16 * (k & 1));
  cp_async_commit();
}

// Slots of an item: its entries plus the alignment head (start & 3), rounded up to a multiple of 4,
// so that its 16-byte groups of X copy whole.
__device__ __forceinline__ int item_slots(const Item& it) { return (int)(((it.start & 3) + it.len + 3) & ~int64_t(3)); }

// With the n staged items visible: the batch is the longest prefix of them whose slots fit in kECap
// (at least one item: kChunk + 6 <= kECap).  Writes sh.ioff; returns the item and slot counts.
template <class SH>
__device__ __forceinline__ void plan_batch(SH& sh, int n, int& nb, int& eb) {
  const int tid = threadIdx.x;
  const int len = tid < n ? item_slots(sh.items[tid]) : 0;
  const int incl = block_scan_incl(sh, len);
  if (tid < n) sh.ioff[tid + 1] = incl;
  if (tid == 0) sh.ioff[0] = 0;
  nb = __syncthreads_count(tid < n && incl <= kECap);
  if (nb == 0) nb = 1;
  eb = sh.ioff[nb];
}

// Row indices and values of the batch's items: one warp per item, 16-byte groups (zero-filled past
// the end of the arrays), or 4-byte copies when the arrays are not 16-byte aligned.
template <class SH>
__device__ __forceinline__ void stage_entries_async(const WalkParams& p, SH& sh, int nb) {
  const uint64_t pol = l2_evict_first_policy();
  const int lane = threadIdx.x & 31;
  for (int j = threadIdx.x >> 5; j < nb; j += kWalkWarps) {
    const int64_t start = sh.items[j].start;
    const int o = sh.ioff[j];
    if (p.x_vec) {
      const int64_t g0 = start >> 2;
      const int ng = (sh.ioff[j + 1] - o) >> 2;
      for (int u = lane; u < ng; u += kWarp) {
        const int64_t e = (g0 + u) * 4;
        const int bytes = (int)min((int64_t)16, (p.nnz - e) * 4);
        if (bytes <= 0) continue;
        cp_async16_zfill_stream(&sh.row[o + 4 * u], p.row_idx + e, bytes, pol);
        cp_async16_zfill_stream(&sh.x[o + 4 * u], p.val + e, bytes, pol);
      }
    } else {
      const int len = sh.items[j].len, base = o + (int)(start & 3);
      for (int v = lane; v < len; v += kWarp) {
        cp_async4_stream(&sh.row[base + v], p.row_idx + start + v, pol);
        cp_async4_stream(&sh.x[base + v], p.val + start + v, pol);
      }
    }
  }
  cp_async_commit();
}

// ---------------------------------------------------------------- phase A: split columns
// Publishes the block's open run of a split column: its partial sums at the run's first item, and
// the run's chunk count added to the column's arrival counter.  The block whose addition completes
// the column lists it for finishing; a run that covers the whole column is finished at once.
template <int PREC>
__device__ __forceinline__ void close_run(const WalkParams& p, Shared<PREC>& sh, int par, uint32_t* col_cnt) {
  if (sh.run_kl < 0) return;
  if (sh.run_chunk0 == 0 && sh.run_cnt == sh.run_nch) {
    const double d = finalize<PREC>(p, par, sh.run_kl, (GHT<PREC>)sh.run_g, (GHT<PREC>)sh.run_h, sh.run_w);
    if (d != 0.0) sh.has_nz = 1;
  } else {
    double2* part = reinterpret_cast<double2*>(p.part);
    part[sh.run_gi0] = make_double2(sh.run_g, sh.run_h);
    const uint32_t old = atom_acqrel_add_u32(col_cnt + sh.run_kl, (uint32_t)sh.run_cnt);
    if (old + (uint32_t)sh.run_cnt == (uint32_t)sh.run_nch) {
      const int f = sh.n_fin++;
      sh.fin_kl[f] = sh.run_kl;
      sh.fin_nch[f] = sh.run_nch;
      sh.fin_c0[f] = sh.run_gi0 - sh.run_chunk0;
      sh.fin_w[f] = sh.run_w;
    }
  }
  sh.run_kl = -1;
}

// First index c in [0, n] with plan[c] > v (plan non-decreasing).
__device__ __forceinline__ int upper_bound_plan(const int64_t* plan, int n, int64_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (plan[mid] <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One warp finishes split column f of the finish list: the partial sums of its holders (blocks whose
// item ranges meet the column) in block order, then the direction.
template <int PREC>
__device__ __forceinline__ void finish_column(const WalkParams& p, Shared<PREC>& sh, int f, int par, uint32_t* col_cnt) {
  const int lane = threadIdx.x & 31;
  const int G = (int)gridDim.x;
  const int32_t kl = sh.fin_kl[f];
  const int64_t c0 = sh.fin_c0[f], c1 = c0 + sh.fin_nch[f];
  if (lane == 0) (void)ld_acquire_u32(col_cnt + kl);  // pairs with every holder's release
  __syncwarp();
  const int bf = upper_bound_plan(sh.plan_row, G + 1, c0) - 1;
  const int bl = upper_bound_plan(sh.plan_row, G + 1, c1 - 1) - 1;
  const double2* part = reinterpret_cast<const double2*>(p.part);
  double ag = 0.0, ah = 0.0;
  for (int b = bf + lane; b <= bl; b += kWarp) {
    const int64_t s0 = max(c0, sh.plan_row[b]), s1 = min(c1, sh.plan_row[b + 1]);
    if (s0 < s1) {
      const double2 v = __ldcg(part + s0);
      ag += v.x;
      ah += v.y;
    }
  }
  ag = warp_sum(ag);
  ah = warp_sum(ah);
  if (lane == 0) {
    const double d = finalize<PREC>(p, par, kl, (GHT<PREC>)ag, (GHT<PREC>)ah, sh.fin_w[f]);
    if (d != 0.0) sh.has_nz = 1;
    col_cnt[kl] = 0u;  // next used after a grid barrier
  }
}

// ---------------------------------------------------------------- phase A
template <int LOSS, int PREC>
__device__ void column_pass(const WalkParams& p, Shared<PREC>& sh, int par, int64_t lo, int64_t i0, int64_t i1) {
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  uint32_t* col_cnt = p.col_cnt;
  if (tid == 0) {
    sh.run_kl = -1;
    sh.n_fin = 0;
  }
  __syncthreads();
  for (int64_t i = i0; i < i1;) {
    int nb, eb;
    if (i == i0 && sh.pf_ready) {
      cp_async_wait_all();
      __syncthreads();
      nb = sh.pf_nb;
      eb = sh.pf_eb;
    } else {
      const int nload = (int)min((int64_t)kICap, i1 - i);
      stage_items_async(p, sh, i, nload);
      cp_async_wait_all();
      __syncthreads();
      plan_batch(sh, nload, nb, eb);
      stage_entries_async(p, sh, nb);
      cp_async_wait_all();
      __syncthreads();
    }
    (void)eb;
    // the entries' coefficient pairs, one warp per item
    for (int j = wib; j < nb; j += kWalkWarps) {
      const int a = sh.ioff[j] + (int)(sh.items[j].start & 3), b = a + sh.items[j].len;
      for (int v = a + lane; v < b; v += kWarp) {
        if constexpr (PREC == 0) cp_async16(&sh.u.rec[v], st_rec<0>(p.st, sh.row[v]));
        else cp_async8(&sh.u.rec[v], st_rec<1>(p.st, sh.row[v]));
      }
    }
    cp_async_commit();
    // the batch's chunks of split columns, in item order
    {
      const int is_split = (tid < nb && sh.items[tid].nch > 1) ? 1 : 0;
      const int at = block_scan_incl(sh, is_split) - is_split;
      if (is_split) sh.split_j[at] = tid;
      if (tid == kWalkThreads - 1) sh.n_split = at + is_split;
      if (tid == 0) sh.pf_ready = 0;
    }
    cp_async_wait_all();
    __syncthreads();
    // one warp per item: the column sums
    for (int j = wib; j < nb; j += kWalkWarps) {
      const int a = sh.ioff[j] + (int)(sh.items[j].start & 3), b = a + sh.items[j].len;
      ColAcc<PREC> acc;
      for (int v = a + lane; v < b; v += kWarp) acc.add(sh.x[v], sh.u.rec[v]);
      acc.reduce();
      if (lane == 0) {
        sh.g[j] = acc.g;
        sh.h[j] = acc.h;
      }
    }
    __syncthreads();
    // one thread per whole column: the direction; thread 0: the runs of split columns
    if (tid < nb) {
      const Item it = sh.items[tid];
      if (it.nch == 1) {
        const double d = finalize<PREC>(p, par, (int32_t)(it.pos - lo), sh.g[tid], sh.h[tid], it.w);
        if (d != 0.0) sh.has_nz = 1;
      }
    }
    if (tid == 0) {
      for (int s = 0; s < sh.n_split; ++s) {
        const int j = sh.split_j[s];
        const Item it = sh.items[j];
        const int32_t kl = (int32_t)(it.pos - lo);
        if (sh.run_kl >= 0 && sh.run_kl != kl) close_run(p, sh, par, col_cnt);
        if (sh.run_kl < 0) {
          sh.run_kl = kl;
          sh.run_nch = it.nch;
          sh.run_chunk0 = it.chunk;
          sh.run_cnt = 0;
          sh.run_gi0 = i + j;
          sh.run_g = 0.0;
          sh.run_h = 0.0;
          sh.run_w = it.w;
        }
        sh.run_g += (double)sh.g[j];
        sh.run_h += (double)sh.h[j];
        ++sh.run_cnt;
        if (it.chunk == it.nch - 1) close_run(p, sh, par, col_cnt);
      }
      if (i + nb >= i1) close_run(p, sh, par, col_cnt);  // the column continues in the next block
    }
    __syncthreads();
    for (int f = wib; f < sh.n_fin; f += kWalkWarps) finish_column(p, sh, f, par, col_cnt);
    __syncthreads();  // the staging area and the finish list are reused by the next batch
    if (tid == 0) sh.n_fin = 0;
    i += nb;
  }
}

// ---------------------------------------------------------------- phase B: per-sample terms
// Loss change of a sample at one step size, and its state after a step.
template <int LOSS, int PREC> struct Row;

// FP64 mode.  Logistic: Eq. 10 in cancellation-free form, log(p e^u + s) - [y = +1] u with
// p = E/(1+E), s = 1/(1+E): log1p(p expm1(u)) - [y = +1] u for E <= 1, log1p(s expm1(-u)) +
// [y = -1] u for E > 1, a log-sum-exp when |u| >= 700.  L2-SVM: Eq. 3 directly.
__device__ __forceinline__ double lr_change_lse(double E, int y, double u) {
  const double lp = log(E) - log1p(E), ls = -log1p(E);
  const double a = lp + u, b = ls;
  const double m = a > b ? a : b;
  return m + log1p(exp(-fabs(a - b))) - (y > 0 ? u : 0.0);
}

template <int LOSS> struct Row<LOSS, 0> {
  using DT = double;
  static __device__ __forceinline__ void term(Fx& acc, double mq, int y, double dl, RecT<1>, double a, float) {
    if constexpr (LOSS == 0) {
      const double u = a * dl;
      double l;
      if (fabs(u) < 700.0) {
        if (mq <= 1.0) l = log1p(mq / (1.0 + mq) * expm1(u)) - (y > 0 ? u : 0.0);
        else l = log1p(expm1(-u) / (1.0 + mq)) + (y < 0 ? u : 0.0);
      } else {
        l = lr_change_lse(mq, y, u);
      }
      fx_add_d(acc, l);
    } else {
      const double bn = mq - a * ((double)y * dl);
      fx_add_d(acc, (bn > 0.0 ? bn * bn : 0.0) - (mq > 0.0 ? mq * mq : 0.0));
    }
  }
  // Algorithm 4's update of the maintained quantity with step a
  static __device__ __forceinline__ double step(double mq, int y, double dl, double a, float) {
    if constexpr (LOSS == 0) return mq * exp(a * dl);
    else return mq - a * (double)y * dl;
  }
  // The first pass: the term at the full step and the state after it.  Logistic: one expm1 serves
  // both (e^u = 1 + m for E <= 1; e^u = 1 / (1 + m) with m = expm1(-u) for E > 1), and the
  // coefficient p or s comes from the sample's stored cg (-s for y = +1, p for y = -1; p = E s, and
  // s = 1 - p is exact for p >= 1/2) instead of a division.
  static __device__ __forceinline__ double term_step(Fx& acc, double mq, int y, double dl, double cg) {
    if constexpr (LOSS == 0) {
      const double u = dl;
      if (fabs(u) < 700.0) {
        double l, nq;
        if (mq <= 1.0) {
          const double pp = y > 0 ? mq * -cg : cg;
          const double m = expm1(u);
          l = log1p(pp * m) - (y > 0 ? u : 0.0);
          nq = fma(mq, m, mq);
        } else {
          const double ss = y > 0 ? -cg : 1.0 - cg;
          const double m = expm1(-u);
          l = log1p(m * ss) + (y < 0 ? u : 0.0);
          nq = mq / (1.0 + m);
        }
        fx_add_d(acc, l);
        return nq;
      }
      fx_add_d(acc, lr_change_lse(mq, y, u));
      return mq * exp(u);
    } else {
      term(acc, mq, y, dl, RecT<1>{0.0f, 0.0f}, 1.0, 1.0f);
      return step(mq, y, dl, 1.0, 1.0f);
    }
  }
};

// Mixed mode: the sample's loss change at u = alpha d^T x_i in FP32 as its first-order part cg u
// plus the remainder, one rounding; each sample's change is formed from the very u its state moves
// by, so the sum is the objective change of the step taken up to FP32 rounding of each term, with
// no cancellation between coordinates (a first-order part taken from the column sums, alpha g^T d,
// errs by about 2^-24 |d_j| sum_i |x_ij cg_i| per coordinate, which a bundle of large opposite d_j
// whose effects cancel in each x_i^T d turns into a spurious decrease).
template <int LOSS> struct Row<LOSS, 1> {
  using DT = float;
  static __device__ __forceinline__ void term(Fx& acc, double mq, int y, float dlf, RecT<1> rc, double a, float af) {
    const float u = af * dlf;
    if constexpr (LOSS == 0) {
      // p = E/(1+E) and s = 1/(1+E) from the FP32 coefficient pair: |cg| is s (y = +1) or p
      // (y = -1), ch = p s; the other one is 1 - |cg| when |cg| <= 1/2, else ch / |cg|
      const float known = fabsf(rc.cg);
      const float other = known <= 0.5f ? 1.0f - known : __fdividef(rc.ch, known);
      const float pp = y > 0 ? other : known, ss = y > 0 ? known : other;
      const bool use_p = pp <= ss;
      fx_add_f(acc, fmaf(rc.cg, u, lr_remainder(use_p ? pp : ss, use_p ? u : -u, fabsf(slot_df(mq).hi))));
    } else {
      fx_add_f(acc, fmaf(rc.cg, u, svm_remainder(slot_df(mq), y > 0 ? u : -u)));
    }
  }
  // the pair of z (logistic) or b (L2-SVM) plus the FP32 step alpha d^T x_i, on the FP32 pipe
  static __device__ __forceinline__ double step(double mq, int y, float dlf, double, float af) {
    const float s = af * dlf;
    return df_slot(df_add_f(slot_df(mq), LOSS == 0 ? s : (y > 0 ? -s : s)));
  }
};

// A pass over the block's samples at one step size.  Its mode (a template parameter) is kFirst:
// terms from the current state, then the full step's state written; kEval: terms from the kept
// state; kApply: the final state from the kept state.
struct RowCtx {
  double a;        // the step size of the terms (kFirst, kEval) or the accepted step (kApply)
  float af;
  bool accept;     // kApply: a step was accepted (else the kept state is restored)
};

// A sample's record as a pass reads it (one 32-byte access): maintained quantity, kept value,
// the coefficient words; the label from the sign of cg.
struct RowState {
  double mq;
  double bak;
  unsigned long long c0, c1;
  int y;
};

template <int PREC>
__device__ __forceinline__ RowState load_state(const WalkParams& p, int32_t r) {
  RowState st;
  const SampleRec* a = reinterpret_cast<const SampleRec*>(p.st) + r;
  asm volatile("ld.global.cg.v4.b64 {%0, %1, %2, %3}, [%4];"
               : "=d"(st.mq), "=d"(st.bak), "=l"(st.c0), "=l"(st.c1)
               : "l"(a));
  if constexpr (PREC == 0) st.y = (long long)st.c0 < 0 ? 1 : -1;
  else st.y = (int)(unsigned)st.c0 < 0 ? 1 : -1;
  return st;
}
__device__ __forceinline__ void store_state(const WalkParams& p, int32_t r, double mq, double bak, unsigned long long c0,
                                            unsigned long long c1) {
  SampleRec* a = reinterpret_cast<SampleRec*>(p.st) + r;
  asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(a), "d"(mq), "d"(bak), "l"(c0), "l"(c1) : "memory");
}
// the coefficient words of a RecT (the second word of a mixed record is left as it was)
__device__ __forceinline__ void rec_words(const RecT<0>& r, unsigned long long& c0, unsigned long long& c1) {
  c0 = (unsigned long long)__double_as_longlong(r.cg);
  c1 = (unsigned long long)__double_as_longlong(r.ch);
}
__device__ __forceinline__ void rec_words(const RecT<1>& r, unsigned long long& c0, unsigned long long&) {
  c0 = (unsigned long long)__float_as_uint(r.cg) | ((unsigned long long)__float_as_uint(r.ch) << 32);
}

// Line-search term and state writes of sample r with d^T x_i = dl (nonzero).
template <int LOSS, int PREC, int MODE>
__device__ __forceinline__ void row_work(const WalkParams& p, const RowCtx& c, int32_t r,
                                         typename Row<LOSS, PREC>::DT dl, RowState st, Fx& acc, unsigned& bad) {
  if constexpr (MODE == kFirst) {
    // the term at the full step alpha = 1 and the state after it, written now; the old value is
    // kept for the case that the line search rejects the full step
    double nq;
    if constexpr (PREC == 0) {
      nq = Row<LOSS, 0>::term_step(acc, st.mq, st.y, dl, __longlong_as_double((long long)st.c0));
    } else {
      RecT<1> rc;
      rc.cg = __uint_as_float((unsigned)st.c0);
      rc.ch = __uint_as_float((unsigned)(st.c0 >> 32));
      Row<LOSS, 1>::term(acc, st.mq, st.y, dl, rc, 1.0, 1.0f);
      nq = Row<LOSS, 1>::step(st.mq, st.y, dl, 1.0, 1.0f);
    }
    if (!slot_ok<LOSS, PREC>(nq)) bad = 1u;
    unsigned long long c0 = st.c0, c1 = st.c1;
    rec_words(slot_coef<LOSS, PREC>(nq, st.y), c0, c1);
    store_state(p, r, nq, st.mq, c0, c1);
  } else if constexpr (MODE == kEval) {
    // mixed: the record holds the full step's coefficients by now; the kept state's are recomputed
    RecT<1> rc{0.0f, 0.0f};
    if constexpr (PREC == 1) rc = RowCoef<LOSS, 1>::make(slot_df(st.bak), st.y);
    Row<LOSS, PREC>::term(acc, st.bak, st.y, dl, rc, c.a, c.af);
  } else {
    double nq = st.bak;
    if (c.accept) {
      nq = Row<LOSS, PREC>::step(st.bak, st.y, dl, c.a, c.af);
      if (!slot_ok<LOSS, PREC>(nq)) atomicOr(p.err, kErrRange);
    }
    unsigned long long c0 = st.c0, c1 = st.c1;
    rec_words(slot_coef<LOSS, PREC>(nq, st.y), c0, c1);
    store_state(p, r, nq, st.bak, c0, c1);
  }
}

// Copies the block's row-sorted entries [cur, min(e1, cur + room)) into the staging arrays.
template <int PREC>
__device__ __forceinline__ void stage_round_async(const WalkParams& p, Shared<PREC>& sh, int64_t cur, int64_t e1) {
  const int head = p.br_vec ? (int)(cur & 3) : 0;
  const int n = (int)min(e1 - cur, (int64_t)(kBCap - head));
  if (p.br_vec) {
    const int64_t g0 = (cur - head) >> 2;
    const int ng = (head + n + 3) >> 2;
    for (int u = threadIdx.x; u < ng; u += kWalkThreads) {
      const int64_t e = (g0 + u) * 4;
      const int bytes = (int)min((int64_t)16, (p.nnz - e) * 4);
      if (bytes <= 0) continue;
      cp_async16_zfill(&sh.b_row[4 * u], p.br_row + e, bytes);
      cp_async16_zfill(&sh.b_k[4 * u], p.br_k + e, bytes);
      cp_async16_zfill(&sh.b_val[4 * u], p.br_val + e, bytes);
    }
  } else {
    for (int v = threadIdx.x; v < n; v += kWalkThreads) {
      cp_async4(&sh.b_row[v], p.br_row + cur + v);
      cp_async4(&sh.b_k[v], p.br_k + cur + v);
      cp_async4(&sh.b_val[v], p.br_val + cur + v);
    }
  }
  cp_async_commit();
  if (threadIdx.x == 0) {
    sh.b_cur = cur;
    sh.b_head = head;
    sh.b_n = n;
  }
}

// A sample whose segment in this bundle is longer than a round: d^T x_i by the whole block straight
// from global memory (thread t sums entries t, t + 256, ... in order; lane trees; warps in order),
// then its work by thread 0.  Returns the end of the segment.
template <int LOSS, int PREC, int MODE>
__device__ __forceinline__ int64_t long_row(const WalkParams& p, Shared<PREC>& sh, int par, int64_t cur, int64_t e1,
                                            const RowCtx& c, Fx& acc, unsigned& bad) {
  using DT = typename Row<LOSS, PREC>::DT;
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int32_t r = sh.b_row[sh.b_head];
  __syncthreads();
  // the segment's end: the first entry of another row (or e1)
  int64_t end = e1;
  for (int64_t base = cur; base < e1; base += kWalkThreads) {
    const int64_t e = base + tid;
    const int diff = (e < e1 && __ldcg(p.br_row + e) != r) ? 1 : 0;
    const unsigned m = __ballot_sync(0xffffffffu, diff);
    if (lane == 0) sh.scan_tot[wib] = m ? (int)(__ffs(m) - 1) : -1;
    __syncthreads();
    int found = -1;
    for (int w = 0; w < kWalkWarps; ++w)
      if (sh.scan_tot[w] >= 0) {
        found = w * 32 + sh.scan_tot[w];
        break;
      }
    __syncthreads();
    if (found >= 0) {
      end = base + found;
      break;
    }
  }
  double part = 0.0;
  for (int64_t e = cur + tid; e < end; e += kWalkThreads) {
    const int k = __ldcg(p.br_k + e);
    const float xv = __ldcg(p.br_val + e);
    if constexpr (PREC == 0) {
      const double d = __ldcg(p.dk + (int64_t)par * p.P_cap + k);
      if (d != 0.0) part = __dadd_rn(part, __dmul_rn(d, (double)xv));
    } else {
      const float d = __ldcg(p.dkf + (int64_t)par * p.P_cap + k);
      if (d != 0.0f) part += (double)(d * xv);
    }
  }
  part = warp_sum(part);
  if (lane == 0) sh.dred[wib] = part;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kWalkWarps; ++w) s += sh.dred[w];
    const DT dl = (DT)s;
    if (dl != DT(0)) row_work<LOSS, PREC, MODE>(p, c, r, dl, load_state<PREC>(p, r), acc, bad);
  }
  __syncthreads();
  return end;
}

constexpr int kRowsPer = 3;  // samples whose state a thread loads at once

// Every sample the block owns in this bundle, once, in rounds of at most kBCap entries cut at row
// starts (the first round may already be staged: sh.b_cur == e0).  Per round: the row starts (a
// block scan), then every entry's d (Eq. 5) gathered into shared memory while each thread loads the
// state of its samples, then per sample d^T x_i in entry order and its work.
template <int LOSS, int PREC, int MODE>
__device__ __forceinline__ void rows_pass(const WalkParams& p, Shared<PREC>& sh, int par, int64_t e0, int64_t e1,
                                          const RowCtx& c, Fx& acc, unsigned& bad) {
  using DT = typename Row<LOSS, PREC>::DT;
  const int tid = threadIdx.x;
  int64_t cur = e0;
  bool staged = sh.b_cur == e0 && sh.b_n > 0;
  while (cur < e1) {
    if (!staged) {
      __syncthreads();  // the previous round's rows are done with the staging arrays
      stage_round_async(p, sh, cur, e1);
    }
    staged = false;
    cp_async_wait_all();
    __syncthreads();
    const int head = sh.b_head, n = sh.b_n;
    const bool complete = cur + n >= e1;
    // d of every staged entry (Eq. 5), gathered while the row starts are found
    {
      const int64_t o = (int64_t)par * p.P_cap;
      for (int v = tid; v < n; v += kWalkThreads) {
        if constexpr (PREC == 0) cp_async8(&sh.u.dv[v], p.dk + o + sh.b_k[head + v]);
        else cp_async4(&sh.u.dv[v], p.dkf + o + sh.b_k[head + v]);
      }
      cp_async_commit();
    }
    // row starts of the round: each thread flags a contiguous run of kPer entries
    constexpr int kPer = kBCap / kWalkThreads;
    int cnt = 0;
    int32_t prev = tid == 0 ? -1 : sh.b_row[head + tid * kPer - 1];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int v = tid * kPer + u;
      if (v < n) {
        const int32_t rv = sh.b_row[head + v];
        cnt += (v == 0 || rv != prev) ? 1 : 0;
        prev = rv;
      }
    }
    const int incl = block_scan_incl(sh, cnt);
    {
      int at = incl - cnt;
      prev = tid == 0 ? -1 : sh.b_row[head + tid * kPer - 1];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int v = tid * kPer + u;
        if (v < n) {
          const int32_t rv = sh.b_row[head + v];
          if (v == 0 || rv != prev) sh.rstart[at++] = v;
          prev = rv;
        }
      }
    }
    int Rt = 0;  // rows of the round: the sum of the warps' totals
    for (int w = 0; w < kWalkWarps; ++w) Rt += sh.scan_tot[w];
    __syncthreads();  // every thread has read the totals and written its row starts
    if (!complete && Rt == 1) {
      cur = long_row<LOSS, PREC, MODE>(p, sh, par, cur, e1, c, acc, bad);
      continue;
    }
    const int Ru = complete ? Rt : Rt - 1;  // the last row of an incomplete round may go on
    if (complete && tid == 0) sh.rstart[Rt] = n;
    __syncthreads();
    const int ne = sh.rstart[Ru];
    cp_async_wait_all();
    __syncthreads();
    // d^T x_i of each complete row, in entry order, kept in place of the row's first d; the rows
    // with a nonzero sum listed in row order (in b_k, idle once the d are gathered)
    int nzc = 0;
    for (int rr = tid; rr < Ru; rr += kWalkThreads) {
      const int a = sh.rstart[rr], b = sh.rstart[rr + 1];
      DT dl = DT(0);
      for (int v = a; v < b; ++v) {
        const DT d = sh.u.dv[v];
        if constexpr (PREC == 0) {
          if (d != 0.0) dl = __dadd_rn(dl, __dmul_rn(d, (double)sh.b_val[head + v]));
        } else {
          if (d != 0.0f) dl = fmaf(d, sh.b_val[head + v], dl);
        }
      }
      sh.u.dv[a] = dl;
      nzc += dl != DT(0) ? 1 : 0;
    }
    {
      const int incl2 = block_scan_incl(sh, nzc);
      int at = incl2 - nzc;
      for (int rr = tid; rr < Ru; rr += kWalkThreads)
        if (sh.u.dv[sh.rstart[rr]] != DT(0)) sh.b_k[at++] = rr;
      if (tid == 0) sh.b_cur = -1;  // the staged round no longer holds its positions: a later pass restages
    }
    int Rn = 0;
    for (int w = 0; w < kWalkWarps; ++w) Rn += sh.scan_tot[w];
    // rows touched by the bundle, a statistic (the first pass counts each once)
    if (MODE == kFirst && tid == 0 && Rn > 0) atomicAdd(p.counters + 4, (unsigned long long)Rn);
    __syncthreads();
    // the listed rows: every state load of a chunk in flight, then the work
    for (int base = 0; base < Rn; base += kRowsPer * kWalkThreads) {
      RowState st[kRowsPer];
      int32_t rrow[kRowsPer];
#pragma unroll
      for (int u = 0; u < kRowsPer; ++u) {
        const int i = base + tid + u * kWalkThreads;
        if (i < Rn) {
          rrow[u] = sh.b_row[head + sh.rstart[sh.b_k[i]]];
          st[u] = load_state<PREC>(p, rrow[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kRowsPer; ++u) {
        const int i = base + tid + u * kWalkThreads;
        if (i < Rn) row_work<LOSS, PREC, MODE>(p, c, rrow[u], sh.u.dv[sh.rstart[sh.b_k[i]]], st[u], acc, bad);
      }
    }
    cur += complete ? n : ne;
  }
  __syncthreads();
}

// Exact sums of one pass.  Fields: [0] g^T d, [1] d^T H d (diagonal), [2] the L1 change of the
// full step (the three parts of Delta, Eq. 7; first pass only), [3 + q] the penalty change at step
// alpha_q, [3 + kMaxK + q] the loss sum at alpha_q (Eq. 10), [kFBad] flag: a sample's speculative
// state left the usable range.  Per block: warp sums into shared memory, then one thread per field
// adds the block's sum to the pass's global accumulator (integer atomics).
template <int PREC>
__device__ __forceinline__ void warp_field(Shared<PREC>& sh, int f, Fx v) {
  v = fx_warp_sum(v);
  if ((threadIdx.x & 31) == 0) {
    FxSlot& s = sh.fxs[threadIdx.x >> 5][f];
    s.l0 = v.l0;
    s.l1 = v.l1;
    s.l2 = v.l2;
    s.fl = v.fl;
  }
}

// The block's sums of the fields in [f0, f1) over warps [0, nw) into the pass's accumulator.
template <int PREC>
__device__ __forceinline__ void block_fields_to_global(const WalkParams& p, Shared<PREC>& sh, int buf, int f, int nw) {
  Fx a;
  for (int w = 0; w < nw; ++w) {
    const FxSlot& s = sh.fxs[w][f];
    a.l0 += s.l0;
    a.l1 += s.l1;
    a.l2 += s.l2;
    a.fl |= s.fl;
  }
  fx_norm(a);
  fx_red_global(reinterpret_cast<long long*>(p.lsacc) + ((int64_t)buf * kPartStride + f) * kAccPad, a);
}

// Penalty change and Delta's terms of one position (FP64) into the thread's sums.
template <int PREC>
__device__ __forceinline__ void position_terms(const WalkParams& p, const Shared<PREC>& sh, double d, double g, double h,
                                               double wj, int q0, int K, bool first, double& gd, double& hdd,
                                               double& l1s, double* pen) {
  if (d == 0.0) return;
  if (first) {
    gd += g * d;
    hdd += h * d * d;
    l1s += p.l1 * (fabs(wj + d) - fabs(wj));
  }
#pragma unroll
  for (int q = 0; q < kMaxK; ++q) {
    if (q < K) {
      const double t = sh.atab[min(q0 + q, kAlphaTab - 1)] * d;
      double r = p.l1 * (fabs(wj + t) - fabs(wj));
      if (p.l2 != 0.0) r += 0.5 * p.l2 * ((wj + t) * (wj + t) - wj * wj);
      pen[q] += r;
    }
  }
}

// One line-search pass of the block: the loss sum of each step over the block's samples, Delta's
// parts (first pass) and the penalty change of each step over the block's positions; the block's
// sums added to accumulator buffer `buf`.  The positions' values are loaded before the samples are
// walked, so that their latency overlaps that work.
template <int LOSS, int PREC>
__device__ __forceinline__ void ls_pass(const WalkParams& p, Shared<PREC>& sh, int par, int64_t lo, int64_t k0,
                                        int64_t k1, int64_t e0, int64_t e1, int q0, int K, bool first, int buf,
                                        int64_t nx0, int nx_load) {
  const int tid = threadIdx.x, wib = tid >> 5;
  const int npos = (int)(k1 - k0);
  const int pos_warps = min(kWalkWarps, (npos + kWarp - 1) / kWarp);
  const int64_t o = (int64_t)par * p.P_cap;
  double d0 = 0.0, g0 = 0.0, h0 = 0.0, w0 = 0.0;
  if (tid < npos) {
    const int64_t kl = k0 + tid;
    d0 = __ldcg(p.dk + o + kl);
    g0 = __ldcg(p.gk + o + kl);
    h0 = __ldcg(p.hk + o + kl);
    w0 = p.w_pos[lo + kl];
  }
  // samples: one rows pass per step size (the first pass writes the full step's state on q = 0)
  unsigned bad = 0u;
  for (int q = 0; q < K; ++q) {
    RowCtx c;
    c.a = sh.atab[min(q0 + q, kAlphaTab - 1)];
    c.af = sh.atab_f[min(q0 + q, kAlphaTab - 1)];
    c.accept = false;
    Fx acc;
    if (first && q == 0) rows_pass<LOSS, PREC, kFirst>(p, sh, par, e0, e1, c, acc, bad);
    else rows_pass<LOSS, PREC, kEval>(p, sh, par, e0, e1, c, acc, bad);
    warp_field(sh, 3 + kMaxK + q, acc);
    // the next bundle's first batch of items, copied while the pass finishes (phase A's staging
    // area is idle here)
    if (q == 0 && nx_load > 0) stage_items_async(p, sh, nx0, nx_load);
  }
  // positions: FP64 per position, each thread's sums then added exactly
  if (wib < pos_warps) {
    double gd = 0.0, hdd = 0.0, l1s = 0.0, pen[kMaxK];
#pragma unroll
    for (int q = 0; q < kMaxK; ++q) pen[q] = 0.0;
    position_terms<PREC>(p, sh, d0, g0, h0, w0, q0, K, first, gd, hdd, l1s, pen);
    for (int64_t kl = k0 + tid + kWalkThreads; kl < k1; kl += kWalkThreads)
      position_terms<PREC>(p, sh, __ldcg(p.dk + o + kl), __ldcg(p.gk + o + kl), __ldcg(p.hk + o + kl),
                           p.w_pos[lo + kl], q0, K, first, gd, hdd, l1s, pen);
    // FP64 warp sums (a fixed tree), then each warp's sum added exactly
    auto field = [&](int f, double v) {
      v = warp_sum(v);
      Fx a;
      if ((tid & 31) == 0) {
        fx_add_d(a, v);
        FxSlot& sl = sh.fxs[wib][f];
        sl.l0 = a.l0;
        sl.l1 = a.l1;
        sl.l2 = a.l2;
        sl.fl = a.fl;
      }
    };
    if (first) {
      field(0, gd);
      field(1, hdd);
      field(2, l1s);
    }
#pragma unroll
    for (int q = 0; q < kMaxK; ++q)
      if (q < K) field(3 + q, pen[q]);
  }
  bad = __syncthreads_or(bad);
  // the block's sums to the pass's accumulators, one thread per field
  const int f = tid;
  if (f < 3 && first && pos_warps > 0) block_fields_to_global(p, sh, buf, f, pos_warps);
  else if (f >= 3 && f < 3 + K && pos_warps > 0) block_fields_to_global(p, sh, buf, f, pos_warps);
  else if (f >= 3 + kMaxK && f < 3 + kMaxK + K) block_fields_to_global(p, sh, buf, f, kWalkWarps);
  else if (f == kFBad && bad)
    asm volatile("red.global.or.b64 [%0], %1;" ::"l"(reinterpret_cast<long long*>(p.lsacc) +
                                                    ((int64_t)buf * kPartStride + kFBad) * kAccPad + 3),
                 "l"(1ll)
                 : "memory");
}

// After the pass's barrier: the grid's sums of the pass's fields into sh.tot (FP64, rounded once).
template <int PREC>
__device__ __forceinline__ void pass_totals(const WalkParams& p, Shared<PREC>& sh, int buf, int K, bool first) {
  const int f = threadIdx.x;
  if (f < kPartStride) {
    const bool used = (f < 3 && first) || (f >= 3 && f < 3 + K) || (f >= 3 + kMaxK && f < 3 + kMaxK + K) ||
                      (f == kFBad && first);
    if (used) {
      const long long* g = reinterpret_cast<const long long*>(p.lsacc) + ((int64_t)buf * kPartStride + f) * kAccPad;
      sh.tot[f] = f == kFBad ? (double)(__ldcg(g + 3) != 0) : fx_value(fx_load_global(g));
    }
  }
  __syncthreads();
}

// beta^q: the table for q < kAlphaTab, repeated multiplication beyond (the order in which Eq. 6's
// backtracking forms it)
template <int PREC>
__device__ __forceinline__ double alpha_of(const WalkParams& p, const Shared<PREC>& sh, int q) {
  if (q < kAlphaTab) return sh.atab[q];
  double a = sh.atab[kAlphaTab - 1];
  for (int i = kAlphaTab - 1; i < q; ++i) a *= p.beta;
  return a;
}

// ---------------------------------------------------------------- the walker
template <int LOSS, int PREC>
__global__ void __launch_bounds__(kWalkThreads, 2) walk_rows_kernel(WalkParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<PREC>& sh = *reinterpret_cast<Shared<PREC>*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int wib = tid >> 5;
  const int G = (int)gridDim.x;
  uint32_t bar = 0, n1 = 0, seen0 = 0, seen1 = 0, npass = 0;
  if (tid == 0) {
    sh.abort = 0;
    sh.has_nz = 0;
    sh.pf_ready = 0;
    sh.b_cur = -1;
    sh.b_n = 0;
    double a = 1.0;
    for (int q = 0; q < kAlphaTab; ++q) {
      sh.atab[q] = a;
      sh.atab_f[q] = (float)a;
      a *= p.beta;
    }
  }
  __syncthreads();

  for (int64_t t = p.t_begin; t < p.t_end; ++t) {
    const int64_t lo = t * (int64_t)p.P;
    const int64_t hi = min(p.npos, lo + (int64_t)p.P);
    const int32_t Pt = (int32_t)(hi - lo);
    const int par = (int)(t & 1);
    const int64_t* pl = p.plan + t * (int64_t)(G + 1);
    const int64_t e0 = p.br_plan[t * (int64_t)(G + 1) + blockIdx.x];
    const int64_t e1 = p.br_plan[t * (int64_t)(G + 1) + blockIdx.x + 1];

    // copies still in flight (the next bundle's first batch) land before new ones are issued
    cp_async_wait_all();
    __syncthreads();
    // the bundle's block plan (for finishing split columns) and the first round of this block's
    // row-sorted entries: both copied while the column pass runs
    for (int c = tid; c <= G; c += kWalkThreads) cp_async8(&sh.plan_row[c], pl + c);
    cp_async_commit();
    if (e1 > e0) stage_round_async(p, sh, e0, e1);
    else if (tid == 0) sh.b_cur = -1;

    // ---------------- A: column sums and directions
    column_pass<LOSS, PREC>(p, sh, par, lo, pl[blockIdx.x], pl[blockIdx.x + 1]);
    if (!grid_barrier_flag(p, n1, seen0, seen1, sh)) {
      cp_async_wait_all();
      return;
    }
    if (tid == 0) sh.has_nz = 0;  // read by the barrier above; next written in the next column pass
    const int64_t kpb = (Pt + G - 1) / G;  // bundle positions per block
    const int64_t k0 = min((int64_t)Pt, (int64_t)blockIdx.x * kpb), k1 = min((int64_t)Pt, k0 + kpb);
    if (!sh.nonzero) {
      if (blockIdx.x == 0 && tid == 0) {
        if (p.tr_q) p.tr_q[t] = 0;
        if (p.tr_alpha) p.tr_alpha[t] = 1.0;
        if (p.tr_Delta) p.tr_Delta[t] = 0.0;
        if (p.tr_dF) p.tr_dF[t] = 0.0;
        atomicAdd(p.counters + 5, 1ull);
        atomicAdd(p.counters + 6, (unsigned long long)Pt);
      }
      continue;  // nothing changed; the next bundle may start
    }

    // the next bundle's first batch of items, copied during the line search
    int64_t nx0 = 0, nx1 = 0;
    if (t + 1 < p.t_end) {
      nx0 = pl[(G + 1) + blockIdx.x];
      nx1 = pl[(G + 1) + blockIdx.x + 1];
    }
    const int nx_load = (int)min((int64_t)kICap, nx1 - nx0);

    // ---------------- B: line search passes
    int q0 = 0;
    bool first = true;
    Decision dec;
    for (;;) {
      const int K = first ? p.K1 : p.K;
      const int buf = (int)(npass % 3);
      ls_pass<LOSS, PREC>(p, sh, par, lo, k0, k1, e0, e1, q0, K, first, buf, first ? nx0 : 0, first ? nx_load : 0);
      // the next bundle's first batch: its nonzeros, once its items are in
      if (first && nx_load > 0) {
        cp_async_wait_all();
        __syncthreads();
        int nb, eb;
        plan_batch(sh, nx_load, nb, eb);
        stage_entries_async(p, sh, nb);
        if (tid == 0) {
          sh.pf_nb = nb;
          sh.pf_eb = eb;
          sh.pf_ready = 1;
        }
      }
      // barrier 2; then every block reads the same exact sums and takes the same decision.  The
      // accumulators rotate over three buffers by pass: after the barrier of pass k, block 0 clears
      // the buffer of pass k + 2 (last read after the barrier of pass k - 1, before this barrier;
      // next added to in pass k + 2, after the barrier of pass k + 1, which block 0 reaches only
      // after clearing it).
      if (!grid_barrier(p, bar, sh)) {
        cp_async_wait_all();
        return;
      }
      pass_totals<PREC>(p, sh, buf, K, first);
      if (blockIdx.x == 0 && tid < kPartStride) {
        long long* z = reinterpret_cast<long long*>(p.lsacc) + ((int64_t)((npass + 2) % 3) * kPartStride + tid) * kAccPad;
        z[0] = 0;
        z[1] = 0;
        z[2] = 0;
        z[3] = 0;
      }
      // the decision (Eq. 6): lane q of warp 0 tests step size alpha_{q0+q}, the first passing one wins
      if (wib == 0) {
        const double* tot = sh.tot;
        if (first && lane == 0) {
          sh.dparts[0] = tot[0];  // Delta's parts, kept for later passes
          sh.dparts[1] = tot[1];
          sh.dparts[2] = tot[2];
        }
        __syncwarp();
        const double gd = sh.dparts[0], hdd = sh.dparts[1], l1 = sh.dparts[2];
        double Delta = gd + p.gamma * hdd + l1;
        // Delta <= (gamma - 1) d^T H d <= 0 (Eq. 7 with Eq. 5's d); mixed mode's FP32 g can leave a
        // small positive rounding residue, which would let a step that raises F pass
        if (PREC == 1 && Delta > 0.0) Delta = 0.0;
        const double a = alpha_of(p, sh, q0 + (lane < K ? lane : 0));
        double dF = 0.0;
        bool pass = false;
        if (lane < K && q0 + lane < p.q_max) {
          dF = p.c * tot[3 + kMaxK + lane] + tot[3 + lane];
          // Delta and the change are finite in exact arithmetic (Delta <= 0): a sum that overflowed
          // (a huge direction or trial step) fails the test instead of passing as inf <= inf
          pass = isfinite(Delta) && isfinite(dF) && dF <= p.sigma * a * Delta;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, pass);
        const int qa = m ? __ffs(m) - 1 : 0;
        const double dFa = __shfl_sync(0xffffffffu, dF, qa);
        const double aa = __shfl_sync(0xffffffffu, a, qa);
        if (lane == 0) {
          Decision dd;
          dd.Delta = Delta;
          if (m) {
            dd.state = kDecAccept;
            dd.q = q0 + qa;
            dd.alpha = aa;
            dd.alpha_f = (float)aa;
            dd.dF = dFa;
          } else if (q0 + K < p.q_max) {
            dd.state = kDecContinue;
            dd.q = q0 + K;
            dd.alpha = 0.0;
            dd.alpha_f = 0.0f;
            dd.dF = 0.0;
          } else {
            dd.state = kDecCap;
            dd.q = p.q_max;
            dd.alpha = 0.0;
            dd.alpha_f = 0.0f;
            dd.dF = 0.0;
          }
          if (blockIdx.x == 0) {
            atomicAdd(p.counters + 2, 1ull);
            if (dd.state != kDecContinue) {
              atomicAdd(p.counters + 0, (unsigned long long)(dd.state == kDecAccept ? dd.q + 1 : p.q_max));
              if (dd.state == kDecCap) atomicAdd(p.counters + 1, 1ull);
              atomicAdd(p.counters + 5, 1ull);
              atomicAdd(p.counters + 6, (unsigned long long)Pt);
              atomicAdd(p.counters + 7, 1ull);
              if (p.tr_q) p.tr_q[t] = dd.q;
              if (p.tr_alpha) p.tr_alpha[t] = dd.alpha;
              if (p.tr_Delta) p.tr_Delta[t] = Delta;
              if (p.tr_dF) p.tr_dF[t] = dd.dF;
            }
            // the full step was taken with some sample outside the usable range
            if (first && dd.state == kDecAccept && dd.q == 0 && tot[kFBad] != 0.0) atomicOr(p.err, kErrRange);
          }
          sh.dec = dd;
        }
      }
      __syncthreads();
      ++npass;
      dec = sh.dec;
      const bool was_first = first;
      first = false;
      if (dec.state == kDecContinue) {
        q0 = dec.q;
        continue;
      }
      // ---------------- C: w_B; the samples' state unless the full step's is already written
      const bool accept = dec.state == kDecAccept;
      if (accept) {
        const int64_t o = (int64_t)par * p.P_cap;
        for (int64_t kl = k0 + tid; kl < k1; kl += kWalkThreads) {
          const double d = p.dk[o + kl];
          if (d != 0.0) p.w_pos[lo + kl] += dec.alpha * d;
        }
      }
      if (!(was_first && accept && dec.q == 0)) {
        RowCtx ca;
        ca.a = dec.alpha;
        ca.af = dec.alpha_f;
        ca.accept = accept;
        Fx none;
        unsigned nb = 0u;
        rows_pass<LOSS, PREC, kApply>(p, sh, par, e0, e1, ca, none, nb);
        if (!grid_barrier(p, bar, sh)) {
          cp_async_wait_all();
          return;
        }
      }
      break;
    }
  }
  cp_async_wait_all();
}

template __global__ void walk_rows_kernel<0, 0>(WalkParams);
template __global__ void walk_rows_kernel<0, 1>(WalkParams);
template __global__ void walk_rows_kernel<1, 0>(WalkParams);
template __global__ void walk_rows_kernel<1, 1>(WalkParams);

namespace {
const void* walk_fn(int loss, int prec) {
  if (loss == 0 && prec == 0) return (const void*)walk_rows_kernel<0, 0>;
  if (loss == 0) return (const void*)walk_rows_kernel<0, 1>;
  if (prec == 0) return (const void*)walk_rows_kernel<1, 0>;
  return (const void*)walk_rows_kernel<1, 1>;
}
size_t walk_smem(int prec) { return prec == 0 ? sizeof(Shared<0>) : sizeof(Shared<1>); }
}  // namespace

}  // namespace rows

cudaError_t walk_rows_configure(int loss, int prec) {
  return cudaFuncSetAttribute(rows::walk_fn(loss, prec), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rows::walk_smem(prec));
}

int walk_rows_max_grid() { return rows::kMaxGrid; }

// Host launcher (cooperative launch: all blocks are co-resident, which the barriers need).  While
// the stream is captured into a graph, the cooperative launch goes through cudaLaunchKernelEx with
// the cooperative attribute, which graph kernel nodes carry.
cudaError_t launch_walk_rows(int loss, int prec, const WalkParams& p, int grid, cudaStream_t s, bool capturing) {
  if (grid > rows::kMaxGrid) return cudaErrorInvalidValue;
  void* args[] = {(void*)&p};
  const void* fn = rows::walk_fn(loss, prec);
  const size_t smem = rows::walk_smem(prec);
  if (grid > 1 && capturing) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kWalkThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
  }
  if (grid > 1) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kWalkThreads), args, smem, s);
  return cudaLaunchKernel(fn, dim3(1), dim3(kWalkThreads), args, smem, s);
}

cudaError_t walk_rows_max_blocks_per_sm(int loss, int prec, int* out) {
  cudaError_t e = walk_rows_configure(loss, prec);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, rows::walk_fn(loss, prec), kWalkThreads,
                                                       rows::walk_smem(prec));
}

}  // namespace pcdn
