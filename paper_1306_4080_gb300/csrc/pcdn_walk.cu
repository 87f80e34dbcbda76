// Bundle walker: one persistent launch steps a run of bundles of one outer iteration
// (Algorithm 3's inner loop with Algorithm 4), all thread blocks in lockstep.
//
// Per bundle t (positions [tP, min((t+1)P, npos)) of the partition's feature order):
//   A  column pass.  The bundle's work items (a column, or a chunk of at most kChunk nonzeros of a
//      long column) are split over the blocks in contiguous runs of balanced nonzero count (the
//      plan).  A block stages a batch of items: item records and w_j (one wave of loads), then the
//      batch's row indices and values and, for each, the row's coefficient pair (two waves, every
//      load of a wave in flight at once), all into shared memory.  One warp per item then reduces
//      g_j, h_j (Eq. 11 / generalised Hessian) from shared memory, computes d_j (Eq. 5) and
//      scatters d_j x_ij into delta (red.add.f64) from the staged copy, setting the row's touched
//      bit.  Chunks of one column combine through a per-column arrival counter: the last chunk in
//      computes d_j and publishes it; the other chunks scatter once it is published.
//   -- barrier 1
//   B  line search: every warp walks a fixed range of the touched-row bitmap, lists the touched
//      rows and sums the loss change of each for K step sizes beta^q (Eq. 10); every block also
//      sums Delta's parts (Eq. 7) and the L1 change of each step over a fixed slice of the
//      bundle.  Partial sums per block.
//   -- barrier 2 (the last block to arrive reduces the partials in block order and decides
//      accept / next K step sizes / cap; Eq. 6)
//   C  update: w_B += alpha d; each warp updates the maintained quantity and coefficients of
//      the rows it evaluated (Algorithm 4), clears delta and the bitmap.
//   -- barrier 3
// A bundle whose directions are all zero ends after barrier 1.
//
// Every wait between blocks is a bounded spin; at the bound the block records kErrTimeout
// and the launch ends (the host reports PCDN_ETIMEOUT).  With one block the barriers are
// __syncthreads() alone.

#include "pcdn_internal.cuh"

namespace pcdn {

template <int PREC>
struct StageA {
  Item items[kICap];
  int32_t ioff[kICap + 1];
  double wpos[kICap];
  int32_t row[kECap];
  float x[kECap];
  RecT<PREC> rec[kECap];
};

template <int PREC>
struct SharedWalk {
  int abort;
  int last;
  int nonzero;
  int scan_tot[kWalkWarps];
  Decision dec;
  double tot[kPartStride];
  double red[kWalkWarps][kPartStride];
  union {
    StageA<PREC> a;
    int32_t list[kWalkWarps][kListCap];
  } u;
};

// ---------------------------------------------------------------- barriers
__device__ __forceinline__ bool err_set(const WalkParams& p) { return ld_volatile_int(p.err) != 0; }

// Plain barrier over the grid.  Returns false when the launch must end.
template <class SH>
__device__ bool grid_barrier(const WalkParams& p, uint32_t& idx, SH& sh) {
  __syncthreads();
  if (gridDim.x > 1) {
    if (threadIdx.x == 0) {
      const uint32_t target = (idx + 1) * gridDim.x;
      red_release_add_u32(p.bar_count, 1u);
      uint32_t spins = 0;
      int abort = 0;
      while (ld_acquire_u32(p.bar_count) < target) {
        if (++spins > p.spin_limit) { atomicOr(p.err, kErrTimeout); abort = 1; break; }
        if ((spins & 1023u) == 0 && err_set(p)) { abort = 1; break; }
      }
      sh.abort = abort || err_set(p);
    }
  } else if (threadIdx.x == 0) {
    sh.abort = err_set(p);
  }
  ++idx;
  __syncthreads();
  return !sh.abort;
}

// Barrier whose last arriving block runs `fn` (the whole block) before releasing the others.
template <class SH, class Fn>
__device__ bool grid_barrier_reduce(const WalkParams& p, uint32_t& idx, SH& sh, Fn&& fn) {
  __syncthreads();
  if (gridDim.x > 1) {
    if (threadIdx.x == 0) {
      __threadfence();
      const uint32_t old = atom_acqrel_add_u32(p.bar_count, 1u);
      sh.last = (old == (idx + 1) * gridDim.x - 1);
    }
    __syncthreads();
    if (sh.last) {
      fn();
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release_u32(p.bar_gen, idx + 1);
        sh.abort = err_set(p);
      }
    } else if (threadIdx.x == 0) {
      uint32_t spins = 0;
      int abort = 0;
      while (ld_acquire_u32(p.bar_gen) < idx + 1) {
        if (++spins > p.spin_limit) { atomicOr(p.err, kErrTimeout); abort = 1; break; }
        if ((spins & 1023u) == 0 && err_set(p)) { abort = 1; break; }
      }
      sh.abort = abort || err_set(p);
    }
  } else {
    fn();
    __syncthreads();
    if (threadIdx.x == 0) sh.abort = err_set(p);
  }
  ++idx;
  __syncthreads();
  return !sh.abort;
}

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
  __device__ __forceinline__ double gsum() const { return warp_sum(g); }
  __device__ __forceinline__ double hsum() const { return warp_sum(h); }
};
template <> struct ColAcc<1> {
  float g = 0.0f, h = 0.0f;
  __device__ __forceinline__ void add(float x, const RecT<1>& r) {
    g = fmaf(x, r.cg, g);
    h = fmaf(x * x, r.ch, h);
  }
  __device__ __forceinline__ double gsum() const { return warp_sum((double)g); }
  __device__ __forceinline__ double hsum() const { return warp_sum((double)h); }
};

template <int PREC>
__device__ __forceinline__ double scatter_value(double d, float x) {
  if constexpr (PREC == 0) return d * (double)x;
  else return (double)((float)d * x);
}

__device__ __forceinline__ void scatter_one(const WalkParams& p, int32_t r, double v) {
  if (v != 0.0) {
    red_add_f64(p.delta + r, v);
    red_or_u32(p.touched + (r >> 5), 1u << (r & 31));
  }
}

// Scatter d x_ij of one work item (reloaded from global memory) into delta.
template <int PREC>
__device__ __forceinline__ void item_scatter_global(const WalkParams& p, const Item& it, double d) {
  const int lane = threadIdx.x & 31;
  const int64_t end = it.start + it.len;
  for (int64_t e = it.start + lane; e < end; e += kWarp) scatter_one(p, p.row_idx[e], scatter_value<PREC>(d, p.val[e]));
}

// g, h -> d for bundle position kl (lane 0 writes; returns d to all lanes).
__device__ __forceinline__ double finalize_column(const WalkParams& p, int32_t kl, double g, double h, double wj) {
  g *= p.c;
  h *= p.c;
  if (h <= 0.0) h = p.nu;
  const double d = newton_direction(g, h, wj);
  if ((threadIdx.x & 31) == 0) {
    p.gk[kl] = g;
    p.hk[kl] = h;
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

// Phase A for this block: items [i0, i1) of the bundle whose positions start at lo.
template <int LOSS, int PREC>
__device__ void column_pass(const WalkParams& p, SharedWalk<PREC>& sh, int64_t lo, int64_t i0, int64_t i1,
                            uint32_t stamp, uint32_t* anynz) {
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  StageA<PREC>& st = sh.u.a;
  const RecT<PREC>* rec = (const RecT<PREC>*)p.rec;
  for (int64_t i = i0; i < i1;) {
    const int nload = (int)min((int64_t)kICap, i1 - i);
    // wave 1: item records and w_j
    int len = 0;
    if (tid < nload) {
      const Item it = p.items[i + tid];
      st.items[tid] = it;
      st.wpos[tid] = p.w_pos[it.pos];
      len = it.len;
    }
    const int incl = block_scan_incl(sh, len);
    if (tid < nload) st.ioff[tid + 1] = incl;
    if (tid == 0) st.ioff[0] = 0;
    int nb = __syncthreads_count(tid < nload && incl <= kECap);  // the fitting items are a prefix
    if (nb == 0) nb = 1;  // an item never exceeds kECap (kChunk <= kECap)
    const int eb = st.ioff[nb];
    // waves 2 and 3: row indices and values, then the rows' coefficient pairs
    {
      int32_t rr[kECap / kWalkThreads];
      float xx[kECap / kWalkThreads];
#pragma unroll
      for (int u = 0; u < kECap / kWalkThreads; ++u) {
        const int v = tid + u * kWalkThreads;
        rr[u] = -1;
        xx[u] = 0.0f;
        if (v < eb) {
          int a = 0, b = nb - 1;  // largest j < nb with ioff[j] <= v
          while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (st.ioff[mid] <= v) a = mid;
            else b = mid - 1;
          }
          const int64_t e = st.items[a].start + (v - st.ioff[a]);
          rr[u] = ld_stream_i32(p.row_idx + e);
          xx[u] = ld_stream_f32(p.val + e);
        }
      }
#pragma unroll
      for (int u = 0; u < kECap / kWalkThreads; ++u) {
        const int v = tid + u * kWalkThreads;
        if (rr[u] >= 0) {
          st.rec[v] = rec[rr[u]];
          st.row[v] = rr[u];
          st.x[v] = xx[u];
        }
      }
    }
    __syncthreads();
    // one warp per item: reduce, direction, scatter
    for (int j = wib; j < nb; j += kWalkWarps) {
      const Item it = st.items[j];
      const int a = st.ioff[j], b = st.ioff[j + 1];
      ColAcc<PREC> acc;
      for (int v = a + lane; v < b; v += kWarp) acc.add(st.x[v], st.rec[v]);
      const double g = acc.gsum(), h = acc.hsum();
      const int32_t kl = (int32_t)(it.pos - lo);
      if (it.nch == 1) {
        const double d = finalize_column(p, kl, g, h, st.wpos[j]);
        if (d != 0.0) {
          if (lane == 0) red_or_u32(anynz, 1u);
          for (int v = a + lane; v < b; v += kWarp) scatter_one(p, st.row[v], scatter_value<PREC>(d, st.x[v]));
        }
      } else {
        const int64_t gi = i + j;  // global item index
        int last = 0;
        if (lane == 0) {
          p.part[2 * gi] = g;
          p.part[2 * gi + 1] = h;
          __threadfence();
          const uint32_t old = atomicAdd(p.col_cnt + kl, 1u);
          last = (old == (uint32_t)it.nch - 1u);
          if (last) __threadfence();
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        __syncwarp();
        if (last) {
          // fixed-order combine of the column's chunks: lane l sums chunks l, l+32, ..., then a tree
          const int64_t first = gi - it.chunk;
          double gs = 0.0, hs = 0.0;
          for (int cch = lane; cch < it.nch; cch += kWarp) {
            gs += p.part[2 * (first + cch)];
            hs += p.part[2 * (first + cch) + 1];
          }
          gs = warp_sum(gs);
          hs = warp_sum(hs);
          const double d = finalize_column(p, kl, gs, hs, st.wpos[j]);
          if (lane == 0) {
            if (d != 0.0) red_or_u32(anynz, 1u);
            p.col_cnt[kl] = 0u;
            __threadfence();
            st_release_u32(p.col_ready + kl, stamp);
          }
        }
      }
    }
    __syncthreads();  // the staging area is reused by the next batch
    i += nb;
  }
  // chunks of split columns scatter once their column's direction is published
  for (int64_t i = i0 + wib; i < i1; i += kWalkWarps) {
    const Item it = p.items[i];
    if (it.nch == 1) continue;
    const int32_t kl = (int32_t)(it.pos - lo);
    int ok = 1;
    double d = 0.0;
    if (lane == 0) {
      uint32_t spins = 0;
      while (ld_acquire_u32(p.col_ready + kl) != stamp) {
        if (++spins > p.spin_limit) { atomicOr(p.err, kErrTimeout); ok = 0; break; }
        if ((spins & 1023u) == 0 && err_set(p)) { ok = 0; break; }
      }
      if (ok) d = p.dk[kl];
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    d = __shfl_sync(0xffffffffu, d, 0);
    if (!ok) break;
    if (d != 0.0) item_scatter_global<PREC>(p, it, d);
  }
}

// ---------------------------------------------------------------- phase B: per-row line-search terms
template <int LOSS, int PREC>
struct LsAcc;

// FP64: direct loss change per row (Eq. 10 rewritten with log1p/expm1; Eq. 3 for the SVM).
template <int LOSS>
struct LsAcc<LOSS, 0> {
  double s[kMaxK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < kMaxK; ++q) s[q] = 0.0;
  }
  __device__ __forceinline__ void row(const WalkParams& p, int32_t r, const double* alpha, int K, bool halving) {
    const double dl = p.delta[r];
    const double mq = p.mq[r];
    const int y = p.y[r];
    if constexpr (LOSS == 0) {
      const double sinv = 1.0 / (1.0 + mq);
      if (halving) {
        // alpha_q = 2 alpha_{q+1}: expm1(-2u) = m (m + 2) with m = expm1(-u)
        double m = expm1(-alpha[K - 1] * dl);
#pragma unroll
        for (int q = kMaxK - 1; q >= 0; --q) {
          if (q < K) {
            const double u = alpha[q] * dl;
            s[q] += log1p(m * sinv) + (y < 0 ? u : 0.0);
            m = m * (m + 2.0);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          if (q < K) {
            const double u = alpha[q] * dl;
            s[q] += log1p(expm1(-u) * sinv) + (y < 0 ? u : 0.0);
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
  __device__ __forceinline__ double get(int q) const { return s[q]; }
};

// Mixed: FP32 remainder terms (non-negative), compensated FP32 sums per lane.
template <int LOSS>
struct LsAcc<LOSS, 1> {
  float s[kMaxK], cmp[kMaxK];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < kMaxK; ++q) { s[q] = 0.0f; cmp[q] = 0.0f; }
  }
  __device__ __forceinline__ void row(const WalkParams& p, int32_t r, const double* alpha, int K, bool) {
    const double dl = p.delta[r];
    const double mq = p.mq[r];
    const int y = p.y[r];
    if constexpr (LOSS == 0) {
      float e = (float)mq, pp, ss;
      if (e <= 1.0f) { ss = 1.0f / (1.0f + e); pp = e * ss; }
      else { const float rr = 1.0f / e; pp = 1.0f / (1.0f + rr); ss = rr * pp; }
      const bool use_p = pp <= ss;
      const float a = use_p ? pp : ss;
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) {
        if (q < K) {
          const float u = (float)(alpha[q] * dl);
          kahan_add(s[q], cmp[q], lr_remainder(a, use_p ? u : -u));
        }
      }
    } else {
      const double v = (double)y * dl;
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) {
        if (q < K) kahan_add(s[q], cmp[q], svm_remainder(mq, alpha[q] * v));
      }
    }
  }
  __device__ __forceinline__ double get(int q) const { return (double)s[q] - (double)cmp[q]; }
};

// Update of one touched row after acceptance with step alpha (Algorithm 4).
template <int LOSS, int PREC>
__device__ __forceinline__ void row_update(const WalkParams& p, int32_t r, double alpha) {
  const double dl = p.delta[r];
  double mq = p.mq[r];
  const int y = p.y[r];
  if constexpr (LOSS == 0) {
    if constexpr (PREC == 0) mq = mq * exp(alpha * dl);
    else mq = fma(mq, (double)expm1f((float)(alpha * dl)), mq);
  } else {
    mq = mq - alpha * (double)y * dl;
  }
  if (!mq_ok<LOSS>(mq)) atomicOr(p.err, kErrNumeric);
  p.mq[r] = mq;
  ((RecT<PREC>*)p.rec)[r] = RowCoef<LOSS, PREC>::make(mq, y);
}

// Walk this warp's bitmap range: list touched rows 32 words at a time, call fn(row) per row.
template <class Fn>
__device__ __forceinline__ void for_touched_rows(const WalkParams& p, int32_t* list, bool clear, Fn&& fn) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t W = (int64_t)gridDim.x * kWalkWarps;
  const int64_t gw = (int64_t)blockIdx.x * kWalkWarps + wib;
  const int64_t per = (p.nwords + W - 1) / W;
  const int64_t w0 = gw * per;
  const int64_t w1 = min(p.nwords, w0 + per);
  for (int64_t base = w0; base < w1; base += kWarp) {
    const int64_t wi = base + lane;
    const uint32_t word = (wi < w1) ? p.touched[wi] : 0u;
    if (__ballot_sync(0xffffffffu, word != 0u) == 0u) continue;
    const int cnt = __popc(word);
    int off = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, off, o);
      if (lane >= o) off += t;
    }
    const int total = __shfl_sync(0xffffffffu, off, 31);
    off -= cnt;
    uint32_t bits = word;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      list[off++] = (int32_t)(wi * 32 + b);
    }
    __syncwarp();
    for (int i = lane; i < total; i += kWarp) fn(list[i]);
    __syncwarp();
    if (clear && word != 0u) p.touched[wi] = 0u;
  }
}

// ---------------------------------------------------------------- the walker
template <int LOSS, int PREC>
__global__ void __launch_bounds__(kWalkThreads) walk_kernel(WalkParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SharedWalk<PREC>& sh = *reinterpret_cast<SharedWalk<PREC>*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int wib = tid >> 5;
  const int K = p.K;
  const int G = (int)gridDim.x;
  uint32_t bar = 0;
  if (tid == 0) sh.abort = 0;
  __syncthreads();

  for (int64_t t = p.t_begin; t < p.t_end; ++t) {
    const int64_t lo = t * (int64_t)p.P;
    const int64_t hi = min(p.npos, lo + (int64_t)p.P);
    const int32_t Pt = (int32_t)(hi - lo);
    const uint32_t stamp = p.stamp_base + (uint32_t)(t + 1);
    uint32_t* anynz = p.anynz + (t % 3);
    // The flag of bundle t+1 was last read (as bundle t-2's) before barrier 1 of bundle t-1, and
    // is next written after barrier 1 of bundle t: clear it in between.
    if (blockIdx.x == 0 && tid == 0) p.anynz[(t + 1) % 3] = 0u;

    // ---------------- A: column reductions, directions, scatter
    {
      const int64_t* pl = p.plan + t * (int64_t)(G + 1) + blockIdx.x;
      column_pass<LOSS, PREC>(p, sh, lo, pl[0], pl[1], stamp, anynz);
    }
    if (!grid_barrier(p, bar, sh)) return;

    if (tid == 0) sh.nonzero = (int)*(volatile uint32_t*)anynz;
    __syncthreads();
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

    // ---------------- B: line search passes
    int q0 = 0;
    Decision dec;
    const int64_t kpb = (Pt + G - 1) / G;  // bundle positions per block
    const int64_t k0 = min((int64_t)Pt, (int64_t)blockIdx.x * kpb), k1 = min((int64_t)Pt, k0 + kpb);
    int32_t* list = sh.u.list[wib];
    for (;;) {
      double alpha[kMaxK];
      {
        double a = 1.0;
        for (int q = 0; q < q0; ++q) a *= p.beta;
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          alpha[q] = a;
          a *= p.beta;
        }
      }
      const bool halving = (p.beta == 0.5);
      LsAcc<LOSS, PREC> acc;
      acc.zero();
      int nrows = 0;
      for_touched_rows(p, list, false, [&](int32_t r) {
        acc.row(p, r, alpha, K, halving);
        ++nrows;
      });
      // bundle-position terms of this block (Eq. 7 parts and the L1 change of each step)
      double pgd = 0.0, phd = 0.0, pl1 = 0.0, pq[kMaxK];
#pragma unroll
      for (int q = 0; q < kMaxK; ++q) pq[q] = 0.0;
      for (int64_t kl = k0 + tid; kl < k1; kl += kWalkThreads) {
        const double d = p.dk[kl];
        if (d == 0.0) continue;
        const double wj = p.w_pos[lo + kl];
        pgd += p.gk[kl] * d;
        phd += p.hk[kl] * d * d;
        pl1 += fabs(wj + d) - fabs(wj);
#pragma unroll
        for (int q = 0; q < kMaxK; ++q)
          if (q < K) pq[q] += fabs(wj + alpha[q] * d) - fabs(wj);
      }
      // block reduction in fixed order: lanes (tree), then warps
      {
        double v[kPartStride];
        v[0] = warp_sum(pgd);
        v[1] = warp_sum(phd);
        v[2] = warp_sum(pl1);
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) {
          v[3 + q] = (q < K) ? warp_sum(pq[q]) : 0.0;
          v[3 + kMaxK + q] = (q < K) ? warp_sum(acc.get(q)) : 0.0;
        }
        v[3 + 2 * kMaxK] = (double)warp_sum_int(nrows);
        if (lane == 0) {
#pragma unroll
          for (int f = 0; f < kPartStride; ++f) sh.red[wib][f] = v[f];
        }
        __syncthreads();
        if (tid < kPartStride) {
          double s = 0.0;
          for (int wv = 0; wv < kWalkWarps; ++wv) s += sh.red[wv][tid];
          p.cta_part[(int64_t)blockIdx.x * kPartStride + tid] = s;
        }
      }
      const int qbase = q0;
      const bool ok = grid_barrier_reduce(p, bar, sh, [&]() {
        // block-order reduction of all partials, then the Armijo decision (Eq. 6)
        double* tot = sh.tot;
        if (tid < kPartStride) {
          double s = 0.0;
          for (int b = 0; b < G; ++b) s += __ldcg(p.cta_part + (int64_t)b * kPartStride + tid);
          tot[tid] = s;
        }
        __syncthreads();
        if (tid == 0) {
          const double gd = tot[0], hdd = tot[1], l1 = tot[2];
          const double Delta = gd + p.gamma * hdd + l1;
          Decision dd;
          dd.state = kDecCap;
          dd.q = p.q_max;
          dd.alpha = 0.0;
          dd.Delta = Delta;
          dd.dF = 0.0;
          for (int q = 0; q < K && qbase + q < p.q_max; ++q) {
            const double a = alpha[q];
            double dF;
            if constexpr (PREC == 0) dF = p.c * tot[3 + kMaxK + q] + tot[3 + q];
            else dF = a * gd + p.c * tot[3 + kMaxK + q] + tot[3 + q];
            if (!(dF == dF)) atomicOr(p.err, kErrNumeric);
            if (dF <= p.sigma * a * Delta) {
              dd.state = kDecAccept;
              dd.q = qbase + q;
              dd.alpha = a;
              dd.dF = dF;
              break;
            }
          }
          if (dd.state != kDecAccept && qbase + K < p.q_max) {
            dd.state = kDecContinue;
            dd.q = qbase + K;
          }
          atomicAdd(p.counters + 2, 1ull);
          if (qbase == 0) atomicAdd(p.counters + 4, (unsigned long long)tot[3 + 2 * kMaxK]);
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
          *p.decision = dd;
        }
      });
      if (!ok) return;
      if (tid == 0) {
        const volatile Decision* vd = p.decision;
        sh.dec.state = vd->state;
        sh.dec.q = vd->q;
        sh.dec.alpha = vd->alpha;
        sh.dec.Delta = vd->Delta;
        sh.dec.dF = vd->dF;
      }
      __syncthreads();
      dec = sh.dec;
      if (dec.state != kDecContinue) break;
      q0 = dec.q;
    }

    // ---------------- C: update w_B, the touched rows, clear scratch
    const double a = dec.alpha;
    const bool accept = dec.state == kDecAccept;
    if (accept) {
      for (int64_t kl = k0 + tid; kl < k1; kl += kWalkThreads) {
        const double d = p.dk[kl];
        if (d != 0.0) p.w_pos[lo + kl] += a * d;
      }
    }
    for_touched_rows(p, list, true, [&](int32_t r) {
      if (accept) row_update<LOSS, PREC>(p, r, a);
      p.delta[r] = 0.0;
    });
    if (!grid_barrier(p, bar, sh)) return;
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

// Host launcher (cooperative launch: all blocks are co-resident, which the barriers need).
cudaError_t launch_walk(int loss, int prec, const WalkParams& p, int grid, cudaStream_t s) {
  void* args[] = {(void*)&p};
  const void* fn = walk_fn(loss, prec);
  const size_t smem = walk_smem(prec);
  if (grid > 1) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kWalkThreads), args, smem, s);
  return cudaLaunchKernel(fn, dim3(1), dim3(kWalkThreads), args, smem, s);
}

cudaError_t walk_max_blocks_per_sm(int loss, int prec, int* out) {
  cudaError_t e = walk_configure(loss, prec);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, walk_fn(loss, prec), kWalkThreads, walk_smem(prec));
}

}  // namespace pcdn
