// Bundle walker: one persistent launch steps a run of bundles of one outer iteration
// (Algorithm 3's inner loop with Algorithm 4), all thread blocks in lockstep.
//
// Per bundle t (positions [tP, min((t+1)P, npos)) of the partition's feature order):
//   A  column pass.  The bundle's work items (a column, or a chunk of at most kChunk nonzeros of a
//      long column) are split over the blocks in contiguous runs of balanced nonzero count (the
//      plan).  A block stages a batch of items: item records and w_j (one wave of loads), then the
//      batch's row indices and values and, for each, the row's coefficient pair (two waves, every
//      load of a wave in flight at once), all into shared memory.  One warp per item reduces
//      g_j, h_j (Eq. 11 / generalised Hessian) from shared memory; one thread per item then forms
//      d_j (Eq. 5); one warp per item scatters d_j x_ij into delta (red.add.f64) from the staged
//      copy and sets the row's touched bit.  Chunks of one column combine through a per-column
//      arrival counter: the last chunk in computes d_j and publishes it; the other chunks scatter
//      once it is published.
//   -- barrier 1 (its counter also carries "some block has a nonzero direction")
//   B  line search: every warp walks a fixed range of the touched-row bitmap, lists the touched
//      rows and sums the loss change of each for K step sizes beta^q (Eq. 10); a block also sums
//      Delta's parts (Eq. 7) and the L1 change of each step over a fixed slice of the bundle.
//      Partial sums per block.
//   -- barrier 2; then every block reduces all partials in block order and takes the same
//      decision: accept / next step sizes / cap (Eq. 6)
//   C  update: w_B += alpha d; each warp updates the maintained quantity and coefficients of
//      the rows it evaluated (Algorithm 4), clears delta and the bitmap.
//   -- barrier 3
// A bundle whose directions are all zero ends after barrier 1.
//
// Precision.  FP64 mode sums in FP64 throughout.  Mixed mode does its per-nonzero and per-row
// arithmetic in FP32 and carries every sum that feeds the Armijo test (Delta's parts, the L1
// change of each step, the line-search remainders) as double-float pairs: about 48 significant
// bits on the FP32 pipe, because GB300's FP64 rate is a small fraction of its FP32 rate.
//
// Every wait between blocks is a bounded spin; at the bound the block records kErrTimeout
// and the launch ends (the host reports PCDN_ETIMEOUT).  With one block the barriers are
// __syncthreads() alone.

#include "pcdn_internal.cuh"

namespace pcdn {

// Phases B and C: a warp's listed touched rows and their staged values.  Mixed mode also stages
// the rows' FP32 coefficient pairs, from which its logistic line search takes p and s.
template <int PREC>
struct RowStage {
  double mq[kWarpRowCap];
  DeltaT<PREC> dl[kWarpRowCap];
  RecT<1> rc[PREC == 1 ? kWarpRowCap : 1];
  int32_t yw[kWarpRowCap];  // the aligned 4-byte word of y holding the row's label
  int32_t row[kWarpRowCap];
};

// One touched row's values as phases B and C see them.
template <int PREC>
struct RowVals {
  DeltaT<PREC> dl;  // d^T x_i
  double mq;        // maintained quantity (E = e^{w^T x_i}, or b = 1 - y w^T x_i)
  RecT<1> rc;       // mixed mode: the FP32 coefficient pair
  int y;
};

// Per-column g and h: FP64 in FP64 mode, FP32 in mixed mode (whose column sums are FP32).
template <int PREC> using GHT = typename std::conditional<PREC == 0, double, float>::type;

// A column's terms of Delta (Eq. 7): g d, h d^2, |w + d| - |w| (zero when d = 0).
template <int PREC>
struct ColTerms {
  double gd, hdd, l1;  // FP64 in both modes (one product per coordinate)
};

// Phase A scratch that phases B and C reuse for their row lists.
template <int PREC>
struct StageA {
  GHT<PREC> g[kICap];
  GHT<PREC> h[kICap];
  double d[kICap];
  RecT<PREC> rec[kECap];
};

constexpr int kAlphaTab = 64;

template <int PREC>
struct SharedWalk {
  int abort;
  int has_nz;
  int nonzero;
  int64_t dko;  // this bundle's half of gk, hk, dk (bundle parity times P_cap)
  int spec_bad;  // a warp's speculative state left the usable range (this bundle)
  int nospec;    // warps of this block whose rows did not fit one staging round
  int all_spec;  // every warp of the grid wrote the full step's state in the first pass
  int n_split;
  int split_ok;
  double split_d;
  int64_t split_items[kSplitCap];
  // the listed split chunks: column position, chunk count, chunk index, w_j, length, start, column
  // index among the block's split columns; and each column's d
  int32_t s_kl[kSplitCap], s_nch[kSplitCap], s_chunk[kSplitCap], s_len[kSplitCap], s_col[kSplitCap];
  double s_w[kSplitCap];
  int64_t s_start[kSplitCap];
  double s_d[kSplitCap];
  ColTerms<PREC> s_terms[kSplitCap];
  double apart[3];  // the block's phase-A sums of Delta's terms (Acc slots): g d, h d^2, |w + d| - |w|
  int scan_tot[kWalkWarps];
  Decision dec;
  double tot[kPartStride];
  double red[kWalkWarps][kPartStride];
  // the batch of work items and their nonzeros; the next bundle's first batch is copied in during
  // phases B and C (pf_ready), since X does not change
  int pf_ready, pf_nb, pf_eb;
  double atab[kAlphaTab];  // beta^q as the running product 1, beta, beta*beta, ... (q < kAlphaTab)
  float atab_f[kAlphaTab];  // the same in FP32 (converted once: conversions run on the FP64 pipe)
  int halving;              // beta == 1/2
  int nrows[kWalkWarps];
  __align__(16) Item items[kICap];  // 16-byte halves are copied asynchronously
  int32_t ioff[kICap + 1];
  int32_t row[kECap];
  float x[kECap];
  union {
    StageA<PREC> a;
    RowStage<PREC> rs[kWalkWarps];
  } u;
};

// A partial sum slot: FP64 mode stores a double, mixed mode a double-float pair in the same 8 bytes.
template <int PREC> struct Acc;
template <> struct Acc<0> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add_t(double x) { v += x; }
  __device__ __forceinline__ void add_acc(const Acc& o) { v += o.v; }
  __device__ __forceinline__ void warp_reduce() { v = warp_sum(v); }
  // sum over aligned groups of T lanes (T a power of two, at most 32)
  __device__ __forceinline__ void group_reduce(int T) {
    for (int o = T >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __device__ __forceinline__ double store() const { return v; }
  __device__ __forceinline__ static Acc load(double s) { Acc a; a.v = s; return a; }
  __device__ __forceinline__ double value() const { return v; }
};
template <> struct Acc<1> {
  dfloat v = {0.0f, 0.0f};
  __device__ __forceinline__ void add(double x) { v = df_add(v, df_make(x)); }
  __device__ __forceinline__ void add_t(float x) { v = df_add_f(v, x); }
  __device__ __forceinline__ void add_acc(const Acc& o) { v = df_add(v, o.v); }
  __device__ __forceinline__ void warp_reduce() { v = df_warp_sum(v); }
  __device__ __forceinline__ void group_reduce(int T) {
    for (int o = T >> 1; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  }
  __device__ __forceinline__ double store() const {
    double s;
    float2 f = make_float2(v.hi, v.lo);
    memcpy(&s, &f, sizeof(s));
    return s;
  }
  __device__ __forceinline__ static Acc load(double s) {
    float2 f;
    memcpy(&f, &s, sizeof(f));
    Acc a;
    a.v.hi = f.x;
    a.v.lo = f.y;
    return a;
  }
  __device__ __forceinline__ double value() const { return df_value(v); }
};

// ---------------------------------------------------------------- phase A helpers
template <int PREC>
struct ColAcc;
template <> struct ColAcc<0> {
  double g = 0.0, h = 0.0;
  __device__ __forceinline__ void add(float x, const RecT<0>& r) {
    const double xd = (double)x;
    g = fma(xd, r.cg, g);
    h = fma(xd * xd, r.ch, h);
  }
  __device__ __forceinline__ void reduce(double& go, double& ho) const {
    go = warp_sum(g);
    ho = warp_sum(h);
  }
};
template <> struct ColAcc<1> {
  float g = 0.0f, h = 0.0f;
  __device__ __forceinline__ void add(float x, const RecT<1>& r) {
    g = fmaf(x, r.cg, g);
    h = fmaf(x * x, r.ch, h);
  }
  __device__ __forceinline__ void reduce(float& go, float& ho) const {
    go = warp_sum_f(g);
    ho = warp_sum_f(h);
  }
};

// delta_r += v and mark row r (r < 0: nothing).  v = d_j x_ij in DeltaT<PREC>: the caller converts
// d_j once per column (dv) and forms dv * x.
template <int PREC>
__device__ __forceinline__ void scatter_one(const WalkParams& p, int32_t r, DeltaT<PREC> v) {
  if (r >= 0 && v != DeltaT<PREC>(0)) {
    red_add(static_cast<DeltaT<PREC>*>(p.delta) + r, v);
    red_or_u32(p.touched + (r >> 5), 1u << (r & 31));
  }
}

// g, h (sums without the factor c) -> the smooth part's g, h (c times the loss's, h <= 0 replaced
// by nu, plus l2 w_j and l2) and d (Eq. 5 with the penalty's l1).
__device__ __forceinline__ double column_direction(const WalkParams& p, double& g, double& h, double wj) {
  g *= p.c;
  h *= p.c;
  if (h <= 0.0) h = p.nu;
  if (p.l2 != 0.0) {
    g += p.l2 * wj;
    h += p.l2;
  }
  return newton_direction(g, h, wj, p.l1);
}

// A column's direction (Eq. 5) from its sums g, h (without the factor c; h <= 0 replaced by nu)
// and its terms of Delta (Eq. 7, their L1 part also the L1 change of the full step alpha = 1);
// with `write`, gk, hk, dk of position kl too.  FP64 mode works in FP64.  Mixed mode works in FP32
// but for |w + d| - |w| (FP64, to keep its cancellation exact) and keeps d = -w exact, so that a
// coordinate set to zero is zero: FP64 instructions are costly on this part.
template <int PREC>
__device__ __forceinline__ double finalize(const WalkParams& p, int64_t kl, GHT<PREC> g, GHT<PREC> h, double wj, bool write,
                                           ColTerms<PREC>& t) {
  double d;
  if constexpr (PREC == 0) {
    d = column_direction(p, g, h, wj);
    t.gd = g * d;
    t.hdd = h * d * d;
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
    t.gd = (double)g * d;
    t.hdd = (double)h * d * d;
  }
  t.l1 = d != 0.0 ? p.l1 * (fabs(wj + d) - fabs(wj)) : 0.0;
  if (write) {
    p.gk[kl] = (double)g;
    p.hk[kl] = (double)h;
    p.dk[kl] = d;
    if (!isfinite(g) || !isfinite(h) || !isfinite(d)) atomicOr(p.err, kErrNumeric);
  }
  return d;
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

// ---------------------------------------------------------------- split columns
// A column longer than kChunk is cut into chunks whose partial sums (g, h) go to part[2 gi],
// part[2 gi + 1]; col_cnt counts the chunks that published.

// Waits (one thread) until all nch chunks of a column have published; false on timeout or another
// block's error.
__device__ __forceinline__ bool split_wait(const WalkParams& p, const uint32_t* cnt, int nch) {
  Waiter wt;
  while (ld_acquire_u32(cnt) != (uint32_t)nch) {
    if (wt.poll(p)) return false;
  }
  return true;
}

// split_wait by lane 0 of a whole (converged) warp; every lane gets the result.
__device__ __forceinline__ bool split_wait_warp(const WalkParams& p, const uint32_t* cnt, int nch) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = split_wait(p, cnt, nch) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Canonical sum of the nch <= kWarpChunks chunk partials of a column, by one warp: lane l sums
// chunks l, l + 32, ... in order (all loads in flight at once), then the lane tree.
__device__ __forceinline__ void split_combine_warp(const double* part, int nch, double& g, double& h) {
  const int lane = threadIdx.x & 31;
  double2 v[kWarpChunks / kWarp];
#pragma unroll
  for (int u = 0; u < kWarpChunks / kWarp; ++u) {
    const int c = u * kWarp + lane;
    v[u] = c < nch ? __ldcg(reinterpret_cast<const double2*>(part) + c) : make_double2(0.0, 0.0);
  }
  g = v[0].x;
  h = v[0].y;
  const int nu = (nch + kWarp - 1) / kWarp;  // FP64 adds are costly on this part: only loaded rounds
#pragma unroll
  for (int u = 1; u < kWarpChunks / kWarp; ++u) {
    if (u < nu) {
      g += v[u].x;
      h += v[u].y;
    }
  }
  g = warp_sum(g);
  h = warp_sum(h);
}

// The same sum, polling the partial slots themselves instead of the column's counter: before each
// walker launch the slots are filled with an all-ones pattern (a NaN payload that no arithmetic
// produces), so a slot is published once its two words differ from it, and the warp has every
// chunk's sums in one round trip when they are ready.  The order of the sum is split_combine_warp's.
// false when the wait gave up (or another block recorded an error).
__device__ __forceinline__ bool split_poll_combine_warp(const WalkParams& p, const double* part, int nch, double& g,
                                                        double& h) {
  const int lane = threadIdx.x & 31;
  double2 v[kWarpChunks / kWarp];
  Waiter wt;
  for (;;) {
    bool ready = true;
#pragma unroll
    for (int u = 0; u < kWarpChunks / kWarp; ++u) {
      const int c = u * kWarp + lane;
      v[u] = c < nch ? __ldcv(reinterpret_cast<const double2*>(part) + c) : make_double2(0.0, 0.0);
      ready = ready && __double_as_longlong(v[u].x) != -1ll && __double_as_longlong(v[u].y) != -1ll;
    }
    if (__all_sync(0xffffffffu, ready)) break;
    int stop = 0;
    if (lane == 0) stop = wt.poll(p);
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
  }
  g = v[0].x;
  h = v[0].y;
  const int nu = (nch + kWarp - 1) / kWarp;
#pragma unroll
  for (int u = 1; u < kWarpChunks / kWarp; ++u) {
    if (u < nu) {
      g += v[u].x;
      h += v[u].y;
    }
  }
  g = warp_sum(g);
  h = warp_sum(h);
  return true;
}

// Canonical sum for nch > kWarpChunks, by the whole block: thread s sums chunks s, s + 256, ...,
// then each warp's lane tree, then the warps in order (result in thread 0).
template <class SH>
__device__ __forceinline__ void split_combine_block(const double* part, int nch, SH& sh, double& g, double& h) {
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  double gs = 0.0, hs = 0.0;
  for (int base = 0; base < nch; base += 8 * kWalkThreads) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = base + u * kWalkThreads + tid;
      v[u] = c < nch ? __ldcg(reinterpret_cast<const double2*>(part) + c) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (base + u * kWalkThreads < nch) {
        gs += v[u].x;
        hs += v[u].y;
      }
    }
  }
  gs = warp_sum(gs);
  hs = warp_sum(hs);
  if (lane == 0) {
    sh.red[wib][0] = gs;
    sh.red[wib][1] = hs;
  }
  __syncthreads();
  g = h = 0.0;
  if (tid == 0) {
    for (int wv = 0; wv < kWalkWarps; ++wv) {
      g += sh.red[wv][0];
      h += sh.red[wv][1];
    }
  }
}

// d of a combined split column (FP64 sums) and, for the holder of chunk 0, its terms of Delta (zero
// for the other holders, so that each column counts once); the holder of chunk 0 also writes gk,
// hk, dk.
template <int PREC>
__device__ __forceinline__ double split_finalize(const WalkParams& p, int64_t kl, bool chunk0, double g, double h, double wj,
                                                 ColTerms<PREC>& t) {
  const double d = finalize<PREC>(p, kl, (GHT<PREC>)g, (GHT<PREC>)h, wj, chunk0, t);
  if (!chunk0) t = ColTerms<PREC>{0, 0, 0};
  return d;
}

// Scatter d x_ij of a chunk reloaded from X, the whole block (eight loads in flight per thread).
template <int PREC>
__device__ __forceinline__ void scatter_chunk_global(const WalkParams& p, int64_t start, int len, double d) {
  const DeltaT<PREC> dv = (DeltaT<PREC>)d;
  int32_t rr[kChunk / kWalkThreads];
  float xx[kChunk / kWalkThreads];
#pragma unroll
  for (int u = 0; u < kChunk / kWalkThreads; ++u) {
    const int v = threadIdx.x + u * kWalkThreads;
    rr[u] = -1;
    xx[u] = 0.0f;
    if (v < len) {
      rr[u] = ld_stream_i32(p.row_idx + start + v);
      xx[u] = ld_stream_f32(p.val + start + v);
    }
  }
#pragma unroll
  for (int u = 0; u < kChunk / kWalkThreads; ++u)
    scatter_one<PREC>(p, rr[u], rr[u] >= 0 ? dv * (DeltaT<PREC>)xx[u] : DeltaT<PREC>(0));
}

// Asynchronous copy of items [i, i + n) (n <= kICap) into sh.items, two 16-byte halves each.
template <class SH>
__device__ __forceinline__ void stage_items_async(const WalkParams& p, SH& sh, int64_t i, int n) {
  for (int k = threadIdx.x; k < 2 * n; k += kWalkThreads)
    cp_async16(reinterpret_cast<char*>(&sh.items[k >> 1]) + 16 * (k & 1),
               reinterpret_cast<const char*>(p.items + i + (k >> 1)) + 16 * (k & 1));
  cp_async_commit();
}

// With the n staged items visible: the batch is the longest prefix of them whose nonzeros fit in
// kECap (at least one item; kChunk <= kECap).  Writes sh.ioff; returns the item and nonzero counts.
template <class SH>
__device__ __forceinline__ void plan_batch(SH& sh, int n, int& nb, int& eb) {
  const int tid = threadIdx.x;
  const int len = tid < n ? sh.items[tid].len : 0;
  const int incl = block_scan_incl(sh, len);
  if (tid < n) sh.ioff[tid + 1] = incl;
  if (tid == 0) sh.ioff[0] = 0;
  nb = __syncthreads_count(tid < n && incl <= kECap);
  if (nb == 0) nb = 1;
  eb = sh.ioff[nb];
}

// Asynchronous copy of the batch's row indices and values into sh.row, sh.x: one warp per item,
// coalesced over the lanes.
template <class SH>
__device__ __forceinline__ void stage_entries_async(const WalkParams& p, SH& sh, int nb) {
  const uint64_t pol = l2_evict_first_policy();
  const int lane = threadIdx.x & 31;
  for (int j = threadIdx.x >> 5; j < nb; j += kWalkWarps) {
    const int64_t start = sh.items[j].start;
    const int o = sh.ioff[j], len = sh.ioff[j + 1] - o;
    for (int v = lane; v < len; v += kWarp) {
      cp_async4_stream(&sh.row[o + v], p.row_idx + start + v, pol);
      cp_async4_stream(&sh.x[o + v], p.val + start + v, pol);
    }
  }
  cp_async_commit();
}

// Phase A for this block: items [i0, i1) of the bundle whose positions start at lo.
template <int LOSS, int PREC>
__device__ void column_pass(const WalkParams& p, SharedWalk<PREC>& sh, int64_t lo, int64_t i0, int64_t i1,
                            uint32_t* col_cnt) {
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  StageA<PREC>& st = sh.u.a;
  if (tid == 0) {
    sh.n_split = 0;
    sh.apart[0] = sh.apart[1] = sh.apart[2] = Acc<PREC>().store();
  }
  __syncthreads();
  int64_t last_i = i0;  // the batch still staged in shared memory
  int last_nb = 0;
  for (int64_t i = i0; i < i1;) {
    // items and nonzeros of the batch: prefetched for the first batch, else copied now
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
    // the rows' coefficient pairs
    for (int v = tid; v < eb; v += kWalkThreads) {
      if constexpr (PREC == 0) cp_async16(&st.rec[v], st_rec<0>(p.st, sh.row[v]));
      else cp_async8(&st.rec[v], st_rec<1>(p.st, sh.row[v]));
    }
    cp_async_commit();
    // chunks of split columns processed by this batch, listed in item order for the deferred
    // scatter (n_split counts them all, also beyond kSplitCap)
    {
      const int is_split = (tid < nb && sh.items[tid].nch > 1) ? 1 : 0;
      const int base = sh.n_split;
      const int at = base + block_scan_incl(sh, is_split) - is_split;
      if (is_split && at < kSplitCap) sh.split_items[at] = i + tid;
      if (tid == kWalkThreads - 1) sh.n_split = at + is_split;  // every thread read it before the scan's barriers
      if (tid == 0) sh.pf_ready = 0;                           // read before the scan's barriers too
    }
    cp_async_wait_all();
    __syncthreads();
    // one warp per item: the reduction; chunks of split columns combine here
    for (int j = wib; j < nb; j += kWalkWarps) {
      const Item it = sh.items[j];
      const int a = sh.ioff[j], b = sh.ioff[j + 1];
      ColAcc<PREC> acc;
      for (int v = a + lane; v < b; v += kWarp) acc.add(sh.x[v], st.rec[v]);
      GHT<PREC> g, h;
      acc.reduce(g, h);
      if (it.nch == 1) {
        if (lane == 0) {
          st.g[j] = g;
          st.h[j] = h;
        }
        continue;
      }
      // a chunk of a split column: publish its partial sums; the column is combined after the
      // batches by every block that holds one of its chunks
      if (lane == 0) {
        const int64_t gi = i + j;  // global item index
        p.part[2 * gi] = (double)g;
        p.part[2 * gi + 1] = (double)h;
        red_release_add_u32(col_cnt + (int32_t)(it.pos - lo), 1u);
      }
    }
    __syncthreads();
    // one thread per item: the direction (Eq. 5) and the column's terms of Delta, summed per warp
    {
      ColTerms<PREC> ct{0, 0, 0};
      if (tid < nb) {
        const Item it = sh.items[tid];
        double d = 0.0;
        if (it.nch == 1) {
          d = finalize<PREC>(p, sh.dko + (it.pos - lo), st.g[tid], st.h[tid], it.w, true, ct);
          if (d != 0.0) sh.has_nz = 1;
        }
        st.d[tid] = d;
      }
      if (wib * kWarp < nb) {
        Acc<PREC> a0, a1, a2;
        a0.add(ct.gd);
        a1.add(ct.hdd);
        a2.add(ct.l1);
        a0.warp_reduce();
        a1.warp_reduce();
        a2.warp_reduce();
        if (lane == 0) {
          sh.red[wib][0] = a0.store();
          sh.red[wib][1] = a1.store();
          sh.red[wib][2] = a2.store();
        }
      }
    }
    __syncthreads();
    if (tid == 0) {  // the block's sums, batches and warps in order
      Acc<PREC> a0 = Acc<PREC>::load(sh.apart[0]), a1 = Acc<PREC>::load(sh.apart[1]), a2 = Acc<PREC>::load(sh.apart[2]);
      for (int wv = 0; wv * kWarp < nb; ++wv) {
        a0.add_acc(Acc<PREC>::load(sh.red[wv][0]));
        a1.add_acc(Acc<PREC>::load(sh.red[wv][1]));
        a2.add_acc(Acc<PREC>::load(sh.red[wv][2]));
      }
      sh.apart[0] = a0.store();
      sh.apart[1] = a1.store();
      sh.apart[2] = a2.store();
    }
    // one warp per item: scatter from the staged copy
    for (int j = wib; j < nb; j += kWalkWarps) {
      const double d = st.d[j];
      if (d == 0.0) continue;
      const DeltaT<PREC> dv = (DeltaT<PREC>)d;
      const int b = sh.ioff[j + 1];
      for (int v = sh.ioff[j] + lane; v < b; v += kWarp) scatter_one<PREC>(p, sh.row[v], dv * (DeltaT<PREC>)sh.x[v]);
    }
    __syncthreads();  // the staging area is reused by the next batch
    last_i = i;
    last_nb = nb;
    i += nb;
  }
  // Chunks of split columns.  Once all chunks of a column have published their sums, each block
  // holding one of them combines the column itself (split_combine: an order fixed by the chunk count
  // alone, so every holder gets the same bits; the holder of chunk 0 writes gk, hk, dk), then
  // scatters its chunks, from the staged copy when the chunk is in the last batch, else reloaded.
  __syncthreads();
  const int ns = sh.n_split;
  if (ns == 0) return;
  if (ns <= kSplitCap) {
    // the listed chunks (item order): their columns, one warp per column of at most kWarpChunks
    // chunks, then the block for each larger one
    if (tid < ns) {
      // the chunk's record: still staged when it belongs to the last batch (a block's whole share,
      // usually), else from global memory
      const int64_t gi = sh.split_items[tid];
      const Item it = (gi >= last_i && gi < last_i + last_nb) ? sh.items[gi - last_i] : p.items[gi];
      sh.s_kl[tid] = (int32_t)(it.pos - lo);
      sh.s_nch[tid] = it.nch;
      sh.s_chunk[tid] = it.chunk;
      sh.s_w[tid] = it.w;
      sh.s_len[tid] = it.len;
      sh.s_start[tid] = it.start;
    }
    if (tid == 0) sh.split_ok = 1;
    __syncthreads();
    if (tid < ns) {  // column index of each listed chunk: the number of column starts before it
      int c = 0;
      for (int k = 1; k <= tid; ++k) c += sh.s_kl[k] != sh.s_kl[k - 1];
      sh.s_col[tid] = c;
    }
    __syncthreads();
    for (int k = wib; k < ns; k += kWalkWarps) {  // a column start per warp, small columns
      const bool start = k == 0 || sh.s_kl[k] != sh.s_kl[k - 1];
      if (!start || sh.s_nch[k] > kWarpChunks) continue;
      double g, h;
      if (!split_poll_combine_warp(p, p.part + 2 * (sh.split_items[k] - sh.s_chunk[k]), sh.s_nch[k], g, h)) {
        if (lane == 0) sh.split_ok = 0;
        continue;
      }
      if (lane == 0) {
        const double dj = split_finalize<PREC>(p, sh.dko + sh.s_kl[k], sh.s_chunk[k] == 0, g, h, sh.s_w[k], sh.s_terms[sh.s_col[k]]);
        if (dj != 0.0) sh.has_nz = 1;
        sh.s_d[sh.s_col[k]] = dj;
      }
    }
    for (int k = 0; k < ns; ++k) {  // large columns, the whole block each
      const bool start = k == 0 || sh.s_kl[k] != sh.s_kl[k - 1];
      if (!start || sh.s_nch[k] <= kWarpChunks) continue;
      __syncthreads();
      if (tid == 0 && !split_wait(p, col_cnt + sh.s_kl[k], sh.s_nch[k])) sh.split_ok = 0;
      __syncthreads();
      if (!sh.split_ok) break;
      double g, h;
      split_combine_block(p.part + 2 * (sh.split_items[k] - sh.s_chunk[k]), sh.s_nch[k], sh, g, h);
      if (tid == 0) {
        const double dj = split_finalize<PREC>(p, sh.dko + sh.s_kl[k], sh.s_chunk[k] == 0, g, h, sh.s_w[k], sh.s_terms[sh.s_col[k]]);
        if (dj != 0.0) sh.has_nz = 1;
        sh.s_d[sh.s_col[k]] = dj;
      }
    }
    __syncthreads();
    if (!sh.split_ok) return;
    if (tid == 0) {  // the split columns' terms of Delta, in column order (held chunk 0 only)
      Acc<PREC> a0 = Acc<PREC>::load(sh.apart[0]), a1 = Acc<PREC>::load(sh.apart[1]), a2 = Acc<PREC>::load(sh.apart[2]);
      const int ncol = sh.s_col[ns - 1] + 1;
      for (int c = 0; c < ncol; ++c) {
        a0.add(sh.s_terms[c].gd);
        a1.add(sh.s_terms[c].hdd);
        a2.add(sh.s_terms[c].l1);
      }
      sh.apart[0] = a0.store();
      sh.apart[1] = a1.store();
      sh.apart[2] = a2.store();
    }
    // scatter every listed chunk, no barriers in between
    for (int k = 0; k < ns; ++k) {
      const double d = sh.s_d[sh.s_col[k]];
      if (d == 0.0) continue;
      const int64_t gi = sh.split_items[k];
      if (gi >= last_i && gi < last_i + last_nb) {
        const int j = (int)(gi - last_i);
        const int b = sh.ioff[j + 1];
        const DeltaT<PREC> dv = (DeltaT<PREC>)d;
        for (int v = sh.ioff[j] + tid; v < b; v += kWalkThreads) scatter_one<PREC>(p, sh.row[v], dv * (DeltaT<PREC>)sh.x[v]);
      } else {
        scatter_chunk_global<PREC>(p, sh.s_start[k], sh.s_len[k], d);
      }
    }
    return;
  }
  // more split chunks than listed: every split chunk of [i0, i1) in item order, one at a time
  int32_t kl_prev = -1;
  double d = 0.0;
  for (int64_t gi = i0; gi < i1; ++gi) {
    const Item it = p.items[gi];
    if (it.nch == 1) continue;
    const int32_t kl = (int32_t)(it.pos - lo);
    if (kl != kl_prev) {
      __syncthreads();
      if (tid == 0) sh.split_ok = split_wait(p, col_cnt + kl, it.nch) ? 1 : 0;
      __syncthreads();
      if (!sh.split_ok) return;
      double g, h;
      if (it.nch <= kWarpChunks) {
        if (wib == 0) split_combine_warp(p.part + 2 * (gi - it.chunk), it.nch, g, h);
      } else {
        split_combine_block(p.part + 2 * (gi - it.chunk), it.nch, sh, g, h);
      }
      if (tid == 0) {
        ColTerms<PREC> ct;
        const double dj = split_finalize<PREC>(p, sh.dko + kl, it.chunk == 0, g, h, it.w, ct);
        if (dj != 0.0) sh.has_nz = 1;
        sh.split_d = dj;
        if (it.chunk == 0) {
          Acc<PREC> a0 = Acc<PREC>::load(sh.apart[0]), a1 = Acc<PREC>::load(sh.apart[1]), a2 = Acc<PREC>::load(sh.apart[2]);
          a0.add(ct.gd);
          a1.add(ct.hdd);
          a2.add(ct.l1);
          sh.apart[0] = a0.store();
          sh.apart[1] = a1.store();
          sh.apart[2] = a2.store();
        }
      }
      __syncthreads();
      d = sh.split_d;
      kl_prev = kl;
    }
    if (d != 0.0) scatter_chunk_global<PREC>(p, it.start, it.len, d);
  }
}

// ---------------------------------------------------------------- phase B: per-row line-search terms
template <int LOSS, int PREC>
struct LsAcc;

// FP64: direct loss change per row.  Logistic: Eq. 10 in cancellation-free form, log(p e^u + s) -
// [y = +1] u with p = E/(1+E), s = 1/(1+E): log1p(p expm1(u)) - [y = +1] u for E <= 1,
// log1p(s expm1(-u)) + [y = -1] u for E > 1, a log-sum-exp when |u| >= 700.  L2-SVM: Eq. 3.
__device__ __forceinline__ double lr_change_lse(double E, int y, double u) {
  const double lp = log(E) - log1p(E), ls = -log1p(E);
  const double a = lp + u, b = ls;
  const double m = a > b ? a : b;
  return m + log1p(exp(-fabs(a - b))) - (y > 0 ? u : 0.0);
}

template <int LOSS>
struct LsAcc<LOSS, 0> {
  double s[kMaxK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < kMaxK; ++q) s[q] = 0.0;
  }
  __device__ __forceinline__ void row(const RowVals<0>& rv, const double* alpha, const float*, int K, bool halving) {
    const double dl = rv.dl, mq = rv.mq;
    const int y = rv.y;
    if constexpr (LOSS == 0) {
      // form A (E <= 1): coefficient p, expm1(+u), label term -[y=+1] u
      // form B (E > 1):  coefficient s, expm1(-u), label term +[y=-1] u
      const bool fa = mq <= 1.0;
      const double coef = fa ? mq / (1.0 + mq) : 1.0 / (1.0 + mq);
      const double sg = fa ? 1.0 : -1.0;
      if (halving) {
        // alpha_q = 2 alpha_{q+1}: expm1(2v) = m (m + 2) with m = expm1(v)
        double m = expm1(sg * alpha[K - 1] * dl);
#pragma unroll
        for (int q = kMaxK - 1; q >= 0; --q) {
          if (q < K) {
            const double u = alpha[q] * dl;
            double l;
            if (fabs(u) < 700.0) l = fa ? log1p(coef * m) - (y > 0 ? u : 0.0) : log1p(m * coef) + (y < 0 ? u : 0.0);
            else l = lr_change_lse(mq, y, u);
            s[q] += l;
            m = m * (m + 2.0);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          if (q < K) {
            const double u = alpha[q] * dl;
            double l;
            if (fabs(u) < 700.0) l = fa ? log1p(coef * expm1(u)) - (y > 0 ? u : 0.0) : log1p(expm1(-u) * coef) + (y < 0 ? u : 0.0);
            else l = lr_change_lse(mq, y, u);
            s[q] += l;
          }
        }
      }
    } else {
      const double b2 = mq > 0.0 ? mq * mq : 0.0;
      const double v = (double)y * dl;
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) {
        if (q < K) {
          const double bn = mq - alpha[q] * v;
          s[q] += (bn > 0.0 ? bn * bn : 0.0) - b2;
        }
      }
    }
  }
  __device__ __forceinline__ Acc<0> get(int q) const { Acc<0> a; a.v = s[q]; return a; }
};

// Mixed: each row's loss change in FP32, its first-order part cg u plus the remainder at the very
// u = alpha d^T x_i its state moves by (one rounding), compensated FP32 sums per lane.  Summing the
// first-order part per row rather than as alpha g^T d from the column sums keeps the FP32 error of
// each coordinate's g_j away from large opposite d_j whose effects cancel within each x_i^T d.
template <int LOSS>
struct LsAcc<LOSS, 1> {
  float s[kMaxK], cmp[kMaxK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < kMaxK; ++q) { s[q] = 0.0f; cmp[q] = 0.0f; }
  }
  __device__ __forceinline__ void row(const RowVals<1>& rv, const double* alpha, const float* alpha_f, int K, bool) {
    const float dlf = rv.dl;
    if constexpr (LOSS == 0) {
      // p = E/(1+E) and s = 1/(1+E) from the row's FP32 coefficient pair: |cg| is s (y = +1) or p
      // (y = -1) as computed from E, ch = p s; the other one is 1 - |cg| when |cg| <= 1/2 (then
      // it is the larger, so 1 - |cg| is accurate), else ch / |cg|.
      const float known = fabsf(rv.rc.cg);
      const float other = known <= 0.5f ? 1.0f - known : rv.rc.ch / known;
      const float pp = rv.y > 0 ? other : known, ss = rv.y > 0 ? known : other;
      const bool use_p = pp <= ss;
      const float a = use_p ? pp : ss, az = fabsf(slot_df(rv.mq).hi);
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) {
        if (q < K) {
          const float u = alpha_f[q] * dlf;
          kahan_add(s[q], cmp[q], fmaf(rv.rc.cg, u, lr_remainder(a, use_p ? u : -u, az)));
        }
      }
    } else {
      // the L2-SVM's coefficient from b (its records are not staged): -2 y max(b, 0)
      const dfloat b = slot_df(rv.mq);
      const float cg = RowCoef<1, 1>::make(b, rv.y).cg;
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) {
        if (q < K) {
          const float u = alpha_f[q] * dlf;
          kahan_add(s[q], cmp[q], fmaf(cg, u, svm_remainder(b, rv.y > 0 ? u : -u)));
        }
      }
    }
  }
  __device__ __forceinline__ Acc<1> get(int q) const {
    Acc<1> a;
    a.v.hi = s[q];
    a.v.lo = -cmp[q];
    a.v = df_add(a.v, dfloat{0.0f, 0.0f});
    return a;
  }
};

// Update of one touched row after acceptance with step alpha (Algorithm 4).
template <int LOSS, int PREC>
__device__ __forceinline__ void row_update(const WalkParams& p, int32_t r, const RowVals<PREC>& rv, double alpha,
                                           float alpha_f) {
  double mq = rv.mq;
  if constexpr (PREC == 0) {
    if constexpr (LOSS == 0) mq = mq * exp(alpha * rv.dl);
    else mq = mq - alpha * (double)rv.y * rv.dl;
  } else {
    // the pair of z (logistic) or b (L2-SVM) plus the FP32 step alpha d^T x_i
    const float step = alpha_f * rv.dl;
    mq = df_slot(df_add_f(slot_df(mq), LOSS == 0 ? step : (rv.y > 0 ? -step : step)));
  }
  if (!slot_ok<LOSS, PREC>(mq)) atomicOr(p.err, kErrRange);
  *st_mq(p.st, r) = mq;
  *st_rec<PREC>(p.st, r) = slot_coef<LOSS, PREC>(mq, rv.y);
}

// The full step's (alpha = 1) state of a touched row, written during the first line-search pass
// (the old values stay staged in shared memory for the case that the step is rejected).  A state
// outside the usable range is reported in `bad`, and an error only if the full step is taken.
template <int LOSS, int PREC>
__device__ __forceinline__ void spec_update(const WalkParams& p, int32_t r, const RowVals<PREC>& rv, int& bad) {
  double mq = rv.mq;
  if constexpr (PREC == 0) {
    if constexpr (LOSS == 0) mq = mq * exp(1.0 * rv.dl);
    else mq = mq - 1.0 * (double)rv.y * rv.dl;
  } else {
    mq = df_slot(df_add_f(slot_df(mq), LOSS == 0 ? rv.dl : (rv.y > 0 ? -rv.dl : rv.dl)));
  }
  if (!slot_ok<LOSS, PREC>(mq)) bad = 1;
  *st_mq(p.st, r) = mq;
  *st_rec<PREC>(p.st, r) = slot_coef<LOSS, PREC>(mq, rv.y);
  static_cast<DeltaT<PREC>*>(p.delta)[r] = DeltaT<PREC>(0);
}

// The old state of a row written back (the full step, written speculatively, was not taken).
template <int LOSS, int PREC>
__device__ __forceinline__ void spec_restore(const WalkParams& p, int32_t r, const RowVals<PREC>& rv) {
  *st_mq(p.st, r) = rv.mq;
  *st_rec<PREC>(p.st, r) = slot_coef<LOSS, PREC>(rv.mq, rv.y);
}

// ---------------------------------------------------------------- phases B and C: the touched rows
// Warp w of the grid owns the bitmap words [w0, w1) (equal contiguous shares).  It lists its touched
// rows (lane l reads word l of each group of 32), copies each listed row's delta, maintained
// quantity and label word into its own shared-memory area kWarpRowCap rows at a time (cp.async,
// all copies of a round in flight at once) and evaluates the rows one lane per row; no block
// barriers.  When the warp's rows fit one group and one round (the usual case) the copies stay
// for the later line-search passes and for phase C.
struct WarpRows {
  int32_t w0, w1;  // n_samples < 2^31: at most 2^26 words
  int n;           // rows listed (cached)
  bool cached;
  bool spec;       // the rows fit one staging round: the first pass writes the full step's state
  uint32_t word;   // this lane's bitmap word (cached)
};

__device__ __forceinline__ WarpRows warp_rows_range(const WalkParams& p) {
  const int64_t W = (int64_t)gridDim.x * kWalkWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWalkWarps + (threadIdx.x >> 5);
  const int64_t per = (p.nwords + W - 1) / W;
  WarpRows wr;
  wr.w0 = (int32_t)min(p.nwords, gw * per);
  wr.w1 = (int32_t)min(p.nwords, (int64_t)wr.w0 + per);
  wr.n = 0;
  // a warp past the last bitmap word has no rows: nothing to stage, nothing to restore
  wr.cached = wr.w1 <= wr.w0;
  wr.spec = wr.w1 <= wr.w0;
  wr.word = 0u;
  return wr;
}

// Counts the touched rows of words [base, min(base + 32, w1)); returns the count (every lane);
// `word` is this lane's word, `off` the rows of the lanes before it.
__device__ __forceinline__ int scan_group(const WalkParams& p, int32_t base, int32_t w1, uint32_t& word, int& off) {
  const int lane = threadIdx.x & 31;
  const int32_t wi = base + lane;
  word = wi < w1 ? p.touched[wi] : 0u;
  const int cnt = __popc(word);
  int x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  off = x - cnt;
  return __shfl_sync(0xffffffffu, x, 31);
}

// Lists the group's rows with index in [i0, i0 + kWarpRowCap) (row order) into rs.row[index - i0].
template <int PREC>
__device__ __forceinline__ void list_window(RowStage<PREC>& rs, int32_t base, uint32_t word, int off, int i0) {
  if (off < i0 + kWarpRowCap && off + __popc(word) > i0) {
    const int32_t wi = base + (threadIdx.x & 31);
    uint32_t bits = word;
    int k = off;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      if (k >= i0 && k < i0 + kWarpRowCap) rs.row[k - i0] = wi * 32 + b;
      ++k;
    }
  }
  __syncwarp();
}

// Copies delta, maintained quantity, label word (and in mixed mode the coefficient pair) of listed
// rows [0, cnt) into the warp's staging arrays and waits for them.
template <int LOSS, int PREC>
__device__ __forceinline__ void stage_rows(const WalkParams& p, RowStage<PREC>& rs, int cnt) {
  for (int i = threadIdx.x & 31; i < cnt; i += kWarp) {
    const int32_t r = rs.row[i];
    if constexpr (PREC == 0) cp_async8(&rs.dl[i], static_cast<const double*>(p.delta) + r);
    else cp_async4(&rs.dl[i], static_cast<const float*>(p.delta) + r);
    cp_async8(&rs.mq[i], st_mq(p.st, r));
    if constexpr (PREC == 1 && LOSS == 0) cp_async8(&rs.rc[i], st_rec<1>(p.st, r));
    cp_async4(&rs.yw[i], p.y + (r & ~3));
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncwarp();
}

// fn(row, values) for staged rows [0, cnt).
template <int LOSS, int PREC, class Fn>
__device__ __forceinline__ void for_staged_rows(const RowStage<PREC>& rs, int cnt, Fn&& fn) {
  for (int i = threadIdx.x & 31; i < cnt; i += kWarp) {
    const int32_t r = rs.row[i];
    RowVals<PREC> v;
    v.dl = rs.dl[i];
    v.mq = rs.mq[i];
    if constexpr (PREC == 1 && LOSS == 0) v.rc = rs.rc[i];
    v.y = (int)(int8_t)(rs.yw[i] >> (8 * (r & 3)));
    fn(r, v);
  }
}

// Every touched row of the warp once (a line-search pass or phase C).  The first call of a bundle
// decides whether the staged rows stay (wr.cached); phase C (clear = true) also clears the words.
template <int LOSS, int PREC, class Fn>
__device__ __forceinline__ void warp_rows(const WalkParams& p, RowStage<PREC>& rs, WarpRows& wr, bool clear, Fn&& fn) {
  const int lane = threadIdx.x & 31;
  if (wr.cached) {
    for_staged_rows<LOSS, PREC>(rs, wr.n, fn);
    if (clear && wr.word != 0u) p.touched[wr.w0 + lane] = 0u;
    return;
  }
  const bool single = wr.w1 - wr.w0 <= kWarp;
  for (int32_t base = wr.w0; base < wr.w1; base += kWarp) {
    uint32_t word;
    int off;
    const int n = scan_group(p, base, wr.w1, word, off);
    if (!clear) wr.spec = single && n <= kWarpRowCap;  // decided before the rows are visited
    for (int i0 = 0; i0 < n; i0 += kWarpRowCap) {
      const int cnt = min(kWarpRowCap, n - i0);
      list_window(rs, base, word, off, i0);
      stage_rows<LOSS, PREC>(p, rs, cnt);
      for_staged_rows<LOSS, PREC>(rs, cnt, fn);
      __syncwarp();  // the next round overwrites the list and staging arrays
    }
    if (clear && word != 0u) p.touched[base + lane] = 0u;
    if (single && n <= kWarpRowCap && !clear) {
      wr.cached = true;
      wr.n = n;
      wr.word = word;
    }
  }
}

// ---------------------------------------------------------------- the walker
template <int LOSS, int PREC>
__global__ void __launch_bounds__(kWalkThreads, 2) walk_kernel(WalkParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SharedWalk<PREC>& sh = *reinterpret_cast<SharedWalk<PREC>*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int wib = tid >> 5;
  const int G = (int)gridDim.x;
  uint32_t bar = 0, n1 = 0, seen0 = 0, seen1 = 0, npass = 0;
  if (tid == 0) {
    sh.abort = 0;
    sh.has_nz = 0;
    sh.pf_ready = 0;
    sh.spec_bad = 0;
    sh.nospec = 0;
    sh.halving = p.beta == 0.5;
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
    const int64_t dko = (t & 1) * p.P_cap;  // this bundle's half of gk, hk, dk

    // the next bundle's item range (its first batch is copied in during phases B and C)
    int64_t nx0 = 0, nx1 = 0;
    if (t + 1 < p.t_end) {
      const int64_t* pn = p.plan + (t + 1) * (int64_t)(G + 1) + blockIdx.x;
      nx0 = pn[0];
      nx1 = pn[1];
    }

    // ---------------- A: column reductions, directions, scatter
    if (tid == 0) sh.dko = (t & 1) * p.P_cap;  // read after column_pass's first barrier
    {
      const int64_t* pl = p.plan + t * (int64_t)(G + 1) + blockIdx.x;
      column_pass<LOSS, PREC>(p, sh, lo, pl[0], pl[1], p.col_cnt + (t & 1) * (int64_t)p.P);
    }
    if (!grid_barrier_flag(p, n1, seen0, seen1, sh)) return;  // no copies in flight: the column pass waited
    if (tid == 0) sh.has_nz = 0;  // read by the barrier above; next written in the next column pass
    const int64_t kpb = (Pt + G - 1) / G;  // bundle positions per block
    const int64_t k0 = min((int64_t)Pt, (int64_t)blockIdx.x * kpb), k1 = min((int64_t)Pt, k0 + kpb);
    // chunk counts of this bundle's split columns, last read before barrier 1; the next bundle
    // counts in the other half, and the one after it only after the next barrier 1
    for (int64_t kl = k0 + tid; kl < k1; kl += kWalkThreads) p.col_cnt[(t & 1) * (int64_t)p.P + kl] = 0u;
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

    // the next bundle's first batch: its items now, its nonzeros inside barrier 3
    const int nx_load = (int)min((int64_t)kICap, nx1 - nx0);
    if (nx_load > 0) stage_items_async(p, sh, nx0, nx_load);

    // ---------------- B: line search passes
    int q0 = 0;
    Decision dec;
    // warps that sum the bundle-position terms (about 128 positions each)
    const int pos_warps = (int)min((int64_t)kWalkWarps, max((int64_t)1, (k1 - k0 + 127) / 128));
    WarpRows wr = warp_rows_range(p);
    RowStage<PREC>& rs = sh.u.rs[wib];
    for (;;) {
      // step sizes of this pass: K1 on the first pass, K on later ones
      const int K = q0 == 0 ? p.K1 : p.K;
      double alpha[kMaxK];
      float alpha_f[kMaxK];
      if (q0 + kMaxK <= kAlphaTab) {
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          alpha[q] = sh.atab[q0 + q];
          alpha_f[q] = sh.atab_f[q0 + q];
        }
      } else {
        double a = 1.0;
        for (int q = 0; q < q0; ++q) a *= p.beta;
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          alpha[q] = a;
          alpha_f[q] = (float)a;
          a *= p.beta;
        }
      }
      const bool halving = sh.halving != 0;
      LsAcc<LOSS, PREC> acc;
      acc.zero();
      int nrows = 0;
      int bad = 0;
      const bool spec_pass = q0 == 0;
      warp_rows<LOSS, PREC>(p, rs, wr, false, [&](int32_t r, const RowVals<PREC>& v) {
        acc.row(v, alpha, alpha_f, K, halving);
        ++nrows;
        if (spec_pass && wr.spec) spec_update<LOSS, PREC>(p, r, v, bad);
      });
      if (spec_pass) {
        // speculating warps clear their bitmap words now (their rows stay staged); the others count
        if (wr.spec && wr.word != 0u) p.touched[wr.w0 + lane] = 0u;
        bad = __any_sync(0xffffffffu, bad != 0) ? 1 : 0;
        if (lane == 0) {
          if (bad) atomicOr(&sh.spec_bad, 1);
          if (!wr.spec) atomicAdd(&sh.nospec, 1);
        }
      }
      // line-search sums of this warp
      {
        nrows = warp_sum_int(nrows);
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          if (q < K) {
            Acc<PREC> a = acc.get(q);
            a.warp_reduce();
            if (lane == 0) sh.red[wib][3 + kMaxK + q] = a.store();
          }
        }
      }
      // the penalty's change for each step over a slice of the bundle's positions; Delta's terms (and
      // the L1 change of the full step, when it is the only one and there is no L2 term) come from
      // the column pass
      const bool full_only = q0 == 0 && K == 1 && p.l2 == 0.0;
      if (!full_only && wib < pos_warps) {
        Acc<PREC> pq[kMaxK];
        for (int64_t kl = k0 + wib * 32 + lane; kl < k1; kl += 32 * pos_warps) {
          const double d = p.dk[dko + kl];
          if (d == 0.0) continue;
          const double wj = p.w_pos[lo + kl];
          if constexpr (PREC == 0) {
#pragma unroll
            for (int q = 0; q < kMaxK; ++q) {
              if (q < K) {
                const double t = alpha[q] * d;
                double r = p.l1 * (fabs(wj + t) - fabs(wj));
                if (p.l2 != 0.0) r += 0.5 * p.l2 * ((wj + t) * (wj + t) - wj * wj);
                pq[q].add(r);
              }
            }
          } else {
            // l1 (|w + a d| - |w|) in double-float arithmetic (a is a power of two when beta = 1/2),
            // plus the L2 change (l2/2) ((w + a d)^2 - w^2)
            const dfloat wd = df_make(wj), dd = df_make(d), aw = df_neg(df_abs(wd));
#pragma unroll
            for (int q = 0; q < kMaxK; ++q) {
              if (q < K) {
                dfloat r = df_add(df_abs(df_add(wd, df_scale(dd, alpha_f[q]))), aw);
                if (p.l1 != 1.0) r = df_scale(r, p.l1_f);
                if (p.l2 != 0.0) {
                  const double t = alpha[q] * d;
                  r = df_add(r, df_make(0.5 * p.l2 * ((wj + t) * (wj + t) - wj * wj)));
                }
                pq[q].v = df_add(pq[q].v, r);
              }
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          if (q < K) {
            pq[q].warp_reduce();
            if (lane == 0) sh.red[wib][3 + q] = pq[q].store();
          }
        }
      }
      if (lane == 0) sh.nrows[wib] = nrows;
      __syncthreads();
      // block total of each field, warps in order, added (FP64) to the grid's accumulator of the field
      if (tid == kWarp && q0 == 0) {  // rows touched by this bundle, a statistic (warp 1)
        int s = 0;
        for (int wv = 0; wv < kWalkWarps; ++wv) s += sh.nrows[wv];
        atomicAdd(p.counters + 4, (unsigned long long)s);
      }
      // one block: its sums are the totals, kept in shared memory (no accumulator round trip)
      if (q0 == 0 && tid == 3 + 2 * kMaxK) {
        if (G == 1) sh.tot[tid] = sh.spec_bad ? 1.0 : 0.0;
        else if (sh.spec_bad) red_add_f64(p.lsacc + ((npass % 3) * kPartStride + 3 + 2 * kMaxK) * kAccPad, 1.0);
      }
      if (q0 == 0 && tid == 4 + 2 * kMaxK) {
        if (G == 1) sh.tot[tid] = (double)sh.nospec;
        else if (sh.nospec)
          red_add_f64(p.lsacc + ((npass % 3) * kPartStride + 4 + 2 * kMaxK) * kAccPad, (double)sh.nospec);
      }
      if (tid < 3 + 2 * kMaxK) {
        const int f = tid;
        {
          double out;
          Acc<PREC> s;
          const bool posf = f < 3 + kMaxK;
          const int nw = posf ? pos_warps : kWalkWarps;
          if ((f >= 3 && f < 3 + kMaxK && f - 3 >= K) || (f >= 3 + kMaxK && f - 3 - kMaxK >= K)) {
            out = s.store();
          } else if (f < 3) {
            out = sh.apart[f];
          } else if (f == 3 && full_only) {
            out = sh.apart[2];
          } else {
            for (int wv = 0; wv < nw; ++wv) s.add_acc(Acc<PREC>::load(sh.red[wv][f]));
            out = s.store();
          }
          const double v = Acc<PREC>::load(out).value();
          if (G == 1) sh.tot[f] = v;  // = 0 + v, what the accumulator would hold
          else red_add_f64(p.lsacc + ((npass % 3) * kPartStride + f) * kAccPad, v);
        }
      }
      const int qbase = q0;
      // the next bundle's first batch of nonzeros, copied while barrier 2 and the decision run (X and
      // the plan are read-only; the item and nonzero arrays are idle until the next column pass)
      if (q0 == 0 && nx_load > 0) {
        cp_async_wait_all();  // its items
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
      // barrier 2; then every block reads the accumulated sums and takes the same decision.  The
      // accumulators rotate over three buffers by pass: after barrier 2 of pass k, block 0 clears the
      // buffer of pass k + 2 (last read in pass k - 1, before this barrier; next added to after
      // barrier 2 of pass k + 1, which block 0 reaches only after clearing it).
      if (!grid_barrier(p, bar, sh)) {
        cp_async_wait_all();  // the next bundle's item copies
        return;
      }
      {
        if (tid < kPartStride) {
          const int f = tid;
          const bool used = f < 3 + K || (f >= 3 + kMaxK && f < 3 + kMaxK + K) || (qbase == 0 && f >= 3 + 2 * kMaxK);
          if (G > 1) {
            if (used) sh.tot[f] = __ldcg(p.lsacc + ((npass % 3) * kPartStride + f) * kAccPad);
            if (blockIdx.x == 0) p.lsacc[(((npass + 2) % 3) * kPartStride + f) * kAccPad] = 0.0;
          }
        }
        __syncthreads();
        // the decision (Eq. 6): lane q of warp 0 tests step size alpha_q, the first passing one wins
        if (wib == 0) {
          const double* tot = sh.tot;
          const double gd = tot[0], hdd = tot[1], l1 = tot[2];
          double Delta = gd + p.gamma * hdd + l1;
          // Delta <= (gamma - 1) d^T H d <= 0 (Eq. 7 with Eq. 5's d); mixed mode's FP32 g can leave
          // a small positive rounding residue, which would let a step that raises F pass
          if (PREC == 1 && Delta > 0.0) Delta = 0.0;
          double a = alpha[0];
#pragma unroll
          for (int q = 1; q < kMaxK; ++q)
            if (lane == q) a = alpha[q];
          double dF = 0.0;
          bool pass = false;
          if (lane < K && qbase + lane < p.q_max) {
            dF = p.c * tot[3 + kMaxK + lane] + tot[3 + lane];
            // Delta and the change are finite in exact arithmetic (Delta <= 0): a sum that overflowed
            // (a huge direction or trial step) fails the test instead of passing as inf <= inf
            pass = isfinite(Delta) && isfinite(dF) && dF <= p.sigma * a * Delta;
          }
          const uint32_t m = __ballot_sync(0xffffffffu, pass);
          const int qa = m ? __ffs(m) - 1 : 0;
          const double dFa = __shfl_sync(0xffffffffu, dF, qa);
          const double aa = __shfl_sync(0xffffffffu, a, qa);
          float af = alpha_f[0];
#pragma unroll
          for (int q = 1; q < kMaxK; ++q)
            if (qa == q) af = alpha_f[q];
          if (lane == 0) {
            Decision dd;
            dd.Delta = Delta;
            if (m) {
              dd.state = kDecAccept;
              dd.q = qbase + qa;
              dd.alpha = aa;
              dd.alpha_f = af;
              dd.dF = dFa;
            } else if (qbase + K < p.q_max) {
              dd.state = kDecContinue;
              dd.q = qbase + K;
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
            if (qbase == 0) sh.all_spec = tot[4 + 2 * kMaxK] == 0.0;
            if (blockIdx.x == 0) {
              // the full step was taken with some sample's speculative state outside the usable range
              if (qbase == 0 && dd.state == kDecAccept && dd.q == 0 && tot[3 + 2 * kMaxK] != 0.0)
                atomicOr(p.err, kErrRange);
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
            }
            sh.dec = dd;
          }
        }
        __syncthreads();
      }
      ++npass;
      dec = sh.dec;
      if (dec.state != kDecContinue) break;
      q0 = dec.q;
    }

    // ---------------- C: update w_B; the touched rows unless the full step's state is in place
    const double a = dec.alpha;
    const bool accept = dec.state == kDecAccept;
    if (accept) {
      for (int64_t kl = k0 + tid; kl < k1; kl += kWalkThreads) {
        const double d = p.dk[dko + kl];
        if (d != 0.0) p.w_pos[lo + kl] += a * d;
      }
    }
    const bool full_step = accept && dec.q == 0;
    if (full_step && sh.all_spec) {
      // every warp wrote the full step's state and cleared its scratch during the line search:
      // the next bundle may start without a third barrier (its column pass reads the new states
      // after barrier 2; gk, hk, dk alternate halves by bundle; its first batch is in flight)
      if (tid == 0) {
        sh.spec_bad = 0;
        sh.nospec = 0;
      }
      __syncthreads();
      continue;
    }
    const float a_f = dec.alpha_f;
    const bool spec_rows = wr.spec;  // this warp's rows hold the full step's state
    warp_rows<LOSS, PREC>(p, rs, wr, true, [&](int32_t r, const RowVals<PREC>& v) {
      if (spec_rows) {
        if (full_step) return;
        if (accept) row_update<LOSS, PREC>(p, r, v, a, a_f);
        else spec_restore<LOSS, PREC>(p, r, v);
        return;
      }
      if (accept) row_update<LOSS, PREC>(p, r, v, a, a_f);
      static_cast<DeltaT<PREC>*>(p.delta)[r] = DeltaT<PREC>(0);
    });
    if (tid == 0) {
      sh.spec_bad = 0;
      sh.nospec = 0;
    }
    // barrier 3 (the next bundle's first batch was issued before barrier 2)
    grid_arrive(p);
    if (!grid_wait(p, bar, sh)) {
      cp_async_wait_all();  // the next bundle's nonzero copies
      return;
    }
  }
}

template __global__ void walk_kernel<0, 0>(WalkParams);
template __global__ void walk_kernel<0, 1>(WalkParams);
template __global__ void walk_kernel<1, 0>(WalkParams);
template __global__ void walk_kernel<1, 1>(WalkParams);

namespace {
const void* walk_fn(int loss, int prec) {
  if (loss == 0 && prec == 0) return (const void*)walk_kernel<0, 0>;
  if (loss == 0) return (const void*)walk_kernel<0, 1>;
  if (prec == 0) return (const void*)walk_kernel<1, 0>;
  return (const void*)walk_kernel<1, 1>;
}
size_t walk_smem(int prec) { return prec == 0 ? sizeof(SharedWalk<0>) : sizeof(SharedWalk<1>); }
}  // namespace

cudaError_t walk_configure(int loss, int prec) {
  return cudaFuncSetAttribute(walk_fn(loss, prec), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)walk_smem(prec));
}

// Host launcher (cooperative launch: all blocks are co-resident, which the barriers need).  While
// the stream is captured into a graph, the cooperative launch goes through cudaLaunchKernelEx with
// the cooperative attribute, which graph kernel nodes carry.
cudaError_t launch_walk(int loss, int prec, const WalkParams& p, int grid, cudaStream_t s, bool capturing) {
  void* args[] = {(void*)&p};
  const void* fn = walk_fn(loss, prec);
  const size_t smem = walk_smem(prec);
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

cudaError_t walk_max_blocks_per_sm(int loss, int prec, int* out) {
  cudaError_t e = walk_configure(loss, prec);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, walk_fn(loss, prec), kWalkThreads, walk_smem(prec));
}

}  // namespace pcdn
