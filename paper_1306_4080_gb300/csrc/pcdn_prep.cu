// Preparation, refresh and reduction kernels of the GB300 PCDN solver.
//
//   partition of an outer iteration (Eq. 8, Algorithm 3): per-feature splitmix64 keys
//     (Steele, Lea, Flood 2014) sorted by a stable LSD radix sort, ties by feature index;
//   column work items: a feature's nonzeros cut into chunks of at most kChunk for the walker;
//   row-major mirror of X: stable radix sort of the CSC entries by row (columns stay ascending
//     within each row), so z = Xw sums every row in column order;
//   refresh: z = Xw by rows, maintained quantity and per-sample coefficients from z;
//   KKT: fresh gradient of every feature and the l1 norm of the minimum-norm subgradient;
//   objective: Eq. 1 from z.
// Every reduction sums in a fixed order (lanes in a tree, warps and blocks in index order).

#include <type_traits>

#include "pcdn_prep.h"

namespace pcdn {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = kScanThreads * kScanItems;  // 4096

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int64_t kSortTile = kSortThreads * kSortRounds;  // 4096

constexpr int kRedThreads = 256;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline cudaError_t post(int64_t* launches) {
  if (launches) ++*launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ scan
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const int64_t* in, int64_t* out, int64_t n,
                                                                 int64_t* block_sums) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t e = base + i;
    const int64_t x = e < n ? in[e] : 0;
    v[i] = run;
    run += x;
  }
  // inclusive scan of thread totals in the warp
  int64_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (tid < 32) {
    int64_t wt = (tid < kScanThreads / 32) ? warp_tot[tid] : 0;
    int64_t wi = wt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (tid >= o) wi += t;
    }
    if (tid < kScanThreads / 32) warp_tot[tid] = wi - wt;  // exclusive warp offsets
    if (tid == kScanThreads / 32 - 1 && block_sums) block_sums[blockIdx.x] = wi;
  }
  __syncthreads();
  const int64_t off = warp_tot[wid] + incl - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t e = base + i;
    if (e < n) out[e] = v[i] + off;
  }
}

__global__ void scan_add_kernel(int64_t* out, int64_t n, const int64_t* block_off) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] += block_off[e / kScanTile];
}

// ------------------------------------------------------------------------------------ radix sort
template <typename K>
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const K* keys, int64_t n, int shift, int64_t nblocks,
                                                                 int64_t* hist) {
  __shared__ uint32_t cnt[256];
  const int tid = threadIdx.x;
  cnt[tid] = 0;
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t e = b0 + (int64_t)r * kSortThreads + tid;
    if (e < n) atomicAdd(&cnt[(uint32_t)(keys[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)tid * nblocks + blockIdx.x] = cnt[tid];
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const K* kin, const int32_t* vin, K* kout,
                                                                    int32_t* vout, int64_t n, int shift,
                                                                    int64_t nblocks, const int64_t* offs) {
  __shared__ int64_t base[256];
  __shared__ uint32_t running[256];
  __shared__ uint32_t wcnt[kSortWarps][256];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  base[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
  running[tid] = 0;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t b0 = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
    for (int i = 0; i < 8; ++i) wcnt[wid][lane * 8 + i] = 0;
    __syncthreads();
    const int64_t e = b0 + (int64_t)r * kSortThreads + tid;
    const bool valid = e < n;
    K key = 0;
    int32_t val = 0;
    uint32_t digit = 256u;
    if (valid) {
      key = kin[e];
      val = vin[e];
      digit = (uint32_t)(key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[wid][digit] = (uint32_t)__popc(peers);
    __syncthreads();
    {
      uint32_t acc = running[tid];
#pragma unroll
      for (int wv = 0; wv < kSortWarps; ++wv) {
        const uint32_t c = wcnt[wv][tid];
        wcnt[wv][tid] = acc;
        acc += c;
      }
      running[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = base[digit] + (int64_t)wcnt[wid][digit] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

template <typename K>
cudaError_t radix_sort_impl(K* k0, int32_t* v0, K* k1, int32_t* v1, int64_t n, int key_bits, int64_t* hist,
                            int64_t* ws, K** k_out, int32_t** v_out, cudaStream_t s, int64_t* launches) {
  K* ka = k0;
  K* kb = k1;
  int32_t* va = v0;
  int32_t* vb = v1;
  if (n > 1) {
    const int64_t nblocks = cdiv(n, kSortTile);
    for (int shift = 0; shift < key_bits; shift += 8) {
      sort_hist_kernel<K><<<(unsigned)nblocks, kSortThreads, 0, s>>>(ka, n, shift, nblocks, hist);
      cudaError_t e = post(launches);
      if (e != cudaSuccess) return e;
      e = scan_exclusive(hist, hist, 256 * nblocks, ws, s, launches);
      if (e != cudaSuccess) return e;
      sort_scatter_kernel<K><<<(unsigned)nblocks, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, nblocks, hist);
      e = post(launches);
      if (e != cudaSuccess) return e;
      K* tk = ka; ka = kb; kb = tk;
      int32_t* tv = va; va = vb; vb = tv;
    }
  }
  *k_out = ka;
  *v_out = va;
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------ partition
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// epoch_dev (may be NULL): the outer-iteration index is epoch + the value read from device memory,
// so that a captured graph of an outer iteration draws a new partition at every replay
__global__ void perm_keys_kernel(uint64_t seed, uint64_t epoch, const int64_t* epoch_dev, int64_t m, uint64_t* keys,
                                 int32_t* vals) {
  if (epoch_dev) epoch += (uint64_t)*epoch_dev;
  const uint64_t gamma = 0x9E3779B97F4A7C15ULL;
  // state of the epoch's stream: first output of the stream started at seed ^ epoch * C
  const uint64_t s_epoch = sm64_mix((seed ^ (epoch * 0xD1B54A32D192ED03ULL)) + gamma);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    keys[j] = sm64_mix(s_epoch + (uint64_t)(j + 1) * gamma);
    vals[j] = (int32_t)j;
  }
}

// ------------------------------------------------------------------------------------ work items
__global__ void item_count_kernel(const int32_t* perm, int64_t npos, const int64_t* col_ptr, int64_t* cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= npos; k += (int64_t)gridDim.x * blockDim.x) {
    if (k == npos) { cnt[k] = 0; continue; }
    const int32_t j = perm[k];
    const int64_t len = col_ptr[j + 1] - col_ptr[j];
    cnt[k] = len == 0 ? 1 : (len + kChunk - 1) / kChunk;
  }
}

__global__ void item_fill_kernel(const int32_t* perm, int64_t npos, const int64_t* col_ptr, const int64_t* item_ptr,
                                 const double* w, Item* items) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npos; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = perm[k];
    const int64_t a = col_ptr[j], len = col_ptr[j + 1] - a;
    const int64_t first = item_ptr[k];
    const int32_t nch = (int32_t)(item_ptr[k + 1] - first);
    for (int32_t c = 0; c < nch; ++c) {
      Item it;
      it.start = a + (int64_t)c * kChunk;
      const int64_t rem = len - (int64_t)c * kChunk;
      it.len = (int32_t)(rem < kChunk ? (rem > 0 ? rem : 0) : kChunk);
      it.pos = (int32_t)k;
      it.nch = nch;
      it.chunk = c;
      it.w = w ? w[j] : 0.0;
      items[first + c] = it;
    }
  }
}

// ------------------------------------------------------------------------------------ block plan
// lengths of items [0, cap]; entries past the walk's real item count (item_ptr[npos]) are 0
__global__ void item_len_kernel(const Item* items, int64_t cap, const int64_t* item_ptr, int64_t npos, int64_t* len) {
  const int64_t n_real = item_ptr[npos];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= cap; i += (int64_t)gridDim.x * blockDim.x)
    len[i] = i < n_real ? (int64_t)items[i].len : 0;
}

__global__ void plan_kernel(const int64_t* item_ptr, const int64_t* item_off, int64_t npos, int32_t P, int64_t nb, int G,
                            int64_t* plan) {
  const int64_t total = nb * (int64_t)(G + 1);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / (G + 1);
    const int c = (int)(idx - t * (G + 1));
    const int64_t lo = t * (int64_t)P;
    const int64_t hi = lo + P < npos ? lo + P : npos;
    const int64_t ib = item_ptr[lo], ie = item_ptr[hi];
    int64_t r;
    if (c == 0) {
      r = ib;
    } else if (c == G) {
      r = ie;
    } else {
      const int64_t z0 = item_off[ib], z = item_off[ie] - z0;
      const int64_t target = z0 + (int64_t)(((__int128)z * c) / G);
      int64_t a = ib, b = ie;  // first i in [ib, ie) with item_off[i] >= target (ie if none)
      while (a < b) {
        const int64_t mid = a + (b - a) / 2;
        if (item_off[mid] < target) a = mid + 1;
        else b = mid;
      }
      r = a;
    }
    plan[idx] = r;
  }
}

__global__ void gather_w_kernel(const double* w, const int32_t* perm, int64_t npos, double* w_pos) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npos; k += (int64_t)gridDim.x * blockDim.x)
    w_pos[k] = w[perm[k]];
}

__global__ void scatter_w_kernel(const double* w_pos, const int32_t* perm, int64_t npos, double* w) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npos; k += (int64_t)gridDim.x * blockDim.x)
    w[perm[k]] = w_pos[k];
}

// ------------------------------------------------------------------------------------ mirror
// Column of entry e: the last j with col_ptr[j] <= e (col_ptr ascending, col_ptr[m] = nnz > e).
__device__ __forceinline__ int64_t column_of(const int64_t* col_ptr, int64_t m, int64_t e) {
  int64_t lo = 0, hi = m;  // col_ptr[lo] <= e < col_ptr[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (col_ptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

constexpr int kSpan = 16;  // consecutive nonzeros per thread in the entry-parallel passes

// entry_col[e] = column of entry e; a thread takes kSpan consecutive entries (one search, then a
// walk), so a long column is spread over many threads.
__global__ void entry_col_kernel(const int64_t* col_ptr, int64_t m, int64_t nnz, int32_t* entry_col) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t * kSpan < nnz; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = t * kSpan, e1 = min(nnz, e0 + kSpan);
    int64_t j = column_of(col_ptr, m, e0);
    int64_t next = col_ptr[j + 1];
    for (int64_t e = e0; e < e1; ++e) {
      while (e >= next && j + 1 < m) next = col_ptr[++j + 1];  // j stays below m
      entry_col[e] = (int32_t)j;
    }
  }
}

__global__ void iota_kernel(int32_t* v, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    v[e] = (int32_t)e;
}

// ------------------------------------------------------------------------------------ validation
__global__ void validate_kernel(const int64_t* col_ptr, const int32_t* row_idx, const float* val, const int8_t* y,
                                int64_t n, int64_t m, int64_t nnz, int* flag) {
  const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid0 == 0 && (col_ptr[0] != 0 || col_ptr[m] != nnz)) atomicOr(flag, 1);
  for (int64_t j = tid0; j < m; j += stride) {
    const int64_t a = col_ptr[j], b = col_ptr[j + 1];
    if (b < a || a < 0 || b > nnz) { atomicOr(flag, 1); continue; }
  }
  for (int64_t e = tid0; e < nnz; e += stride) {
    const int32_t r = row_idx[e];
    if (r < 0 || r >= n || !isfinite(val[e])) atomicOr(flag, 2);
  }
  for (int64_t i = tid0; i < n; i += stride)
    if (y[i] != 1 && y[i] != -1) atomicOr(flag, 4);
}

// rows strictly ascending within every column (run after the column pointers passed): entry e
// (not the first of its column) must exceed entry e - 1; kSpan consecutive entries per thread
__global__ void validate_order_kernel(const int64_t* col_ptr, const int32_t* row_idx, int64_t m, int64_t nnz,
                                      int* flag) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t * kSpan < nnz; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = t * kSpan, e1 = min(nnz, e0 + kSpan);
    // every index stays in range even when col_ptr itself is malformed (this check runs in the same
    // launch sequence as the one that tests col_ptr): j in [0, m), e in [0, nnz)
    int64_t j = column_of(col_ptr, m, e0);
    int64_t start = col_ptr[j], next = col_ptr[j + 1];
    bool bad = false;
    for (int64_t e = e0; e < e1; ++e) {
      while (e >= next && j + 1 < m) {
        start = next;
        next = col_ptr[++j + 1];
      }
      if (e > start && row_idx[e] <= row_idx[e - 1]) bad = true;
    }
    if (bad) atomicOr(flag, 8);
  }
}

// ------------------------------------------------------------------------------------ refresh
__device__ __forceinline__ double row_loss(int loss, double z, int y) {
  const double yz = (double)y * z;
  if (loss == 0) return yz > 0 ? log1p(exp(-yz)) : (-yz + log1p(exp(yz)));
  const double b = 1.0 - yz;
  return b > 0 ? b * b : 0.0;
}

// One lane per row; each lane walks its row in column order with eight loads in flight, using a
// separate multiply and add per nonzero (the same rounding as a column-by-column accumulation).
template <int LOSS, int PREC>
__global__ void __launch_bounds__(kRedThreads) refresh_kernel(const int64_t* row_ptr, const int32_t* col_idx,
                                                              const float* rval, const int8_t* y, const double* w,
                                                              int64_t n, void* st, int write_state,
                                                              double* loss_part, int* err) {
  __shared__ double wsum[kRedThreads];
  double lsum = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    const int64_t a = row_ptr[i], b = row_ptr[i + 1];
    double z = 0.0;
    for (int64_t e0 = a; e0 < b; e0 += 8) {
      int32_t c[8];
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t e = e0 + u;
        c[u] = e < b ? col_idx[e] : -1;
        v[u] = e < b ? rval[e] : 0.0f;
      }
      double wv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) wv[u] = c[u] >= 0 ? w[c[u]] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (wv[u] != 0.0) z = __dadd_rn(z, __dmul_rn((double)v[u], wv[u]));
    }
    const int yi = y[i];
    if (loss_part) lsum += row_loss(LOSS, z, yi);
    if (write_state) {
      // FP64 keeps e^z (Algorithm 4), which holds |z| up to about 700; mixed keeps z itself
      if (PREC == 0 ? (LOSS == 0 && fabs(z) > 700.0) : !isfinite(z)) atomicOr(err, kErrRefresh);
      const double v = slot_from_z<LOSS, PREC>(z, yi);
      *st_mq(st, i) = v;
      *st_rec<PREC>(st, i) = slot_coef<LOSS, PREC>(v, yi);
    }
  }
  if (loss_part) {
    wsum[threadIdx.x] = lsum;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) wsum[threadIdx.x] += wsum[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = wsum[0];
  }
}

// Mixed precision: w as a pair of FP32 numbers hi + lo (w - hi rounded), about 48 significant bits.
__global__ void split_w_kernel(const double* w, int64_t m, float2* w2) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[j];
    const float hi = (float)v;
    w2[j] = make_float2(hi, (float)(v - (double)hi));
  }
}

// Mixed precision: z = Xw with T lanes per row in double-float arithmetic on the FP32 pipe (the
// FP64 pipe of this part runs at a small fraction of the FP32 rate).  Each product x_ij w_j is
// formed as x_ij hi_j exactly (error-free product by FMA) plus x_ij lo_j, summed as a double-float
// pair; the T partial sums combine in a fixed tree.  Relative error of z about 2^-44 of sum |x_ij w_j|.
// A warp sums 32 consecutive rows, 32/T at a time, keeps their sums in shared memory, then finishes
// them one lane per row (the FP64 part: e^z, the coefficients, the loss) with every lane busy.
// Every lane of a warp runs the same number of rounds, so the shuffles are full-warp.
template <int LOSS, int T>
__global__ void __launch_bounds__(kRedThreads) refresh_df_kernel(const int64_t* row_ptr, const int32_t* col_idx,
                                                                 const float* rval, const int8_t* y, const float2* w2,
                                                                 int64_t n, void* st, int write_state,
                                                                 double* loss_part, int* err) {
  __shared__ double wsum[kRedThreads];
  __shared__ float2 zs[kRedThreads / 32][32];
  constexpr int G = 32 / T;  // rows per round
  const int lane = threadIdx.x & 31;
  const int gl = lane & (T - 1);
  const int grp = lane / T;
  float2* zw = zs[threadIdx.x >> 5];
  const int64_t warp = ((int64_t)blockIdx.x * kRedThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kRedThreads) >> 5;
  double lsum = 0.0;
  for (int64_t r0 = warp * 32; r0 < n; r0 += nwarps * 32) {
#pragma unroll 1
    for (int sub = 0; sub < T; ++sub) {
      const int64_t i = r0 + sub * G + grp;
      const bool valid = i < n;
      const int64_t a = valid ? row_ptr[i] : 0, b = valid ? row_ptr[i + 1] : 0;
      dfloat acc = {0.0f, 0.0f};
      int64_t e = a + gl;
      for (; e + 3 * T < b; e += 4 * T) {
        int32_t c[4];
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = col_idx[e + u * T];
          v[u] = rval[e + u * T];
        }
        float2 wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) wv[u] = w2[c[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float ph = v[u] * wv[u].x;
          const float pl = fmaf(v[u], wv[u].y, fmaf(v[u], wv[u].x, -ph));
          acc = df_add(acc, dfloat{ph, pl});
        }
      }
      for (; e < b; e += T) {
        const float v = rval[e];
        const float2 wv = w2[col_idx[e]];
        const float ph = v * wv.x;
        const float pl = fmaf(v, wv.y, fmaf(v, wv.x, -ph));
        acc = df_add(acc, dfloat{ph, pl});
      }
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o));
      if (gl == 0) zw[sub * G + grp] = make_float2(acc.hi, acc.lo);
    }
    __syncwarp();
    const int64_t i = r0 + lane;
    if (i < n) {
      const float2 zz = zw[lane];
      const double z = (double)zz.x + (double)zz.y;
      const int yi = y[i];
      if (loss_part) lsum += row_loss(LOSS, z, yi);
      if (write_state) {
        // the pair of z itself (logistic) or of 1 - y z (L2-SVM), without a round trip through FP64
        if (!isfinite(z)) atomicOr(err, kErrRefresh);
        const dfloat zd = {zz.x, zz.y};
        const dfloat v = LOSS == 0 ? zd : df_add_f(yi > 0 ? df_neg(zd) : zd, 1.0f);
        *st_mq(st, i) = df_slot(v);
        *st_rec<1>(st, i) = RowCoef<LOSS, 1>::make(v, yi);
      }
    }
    __syncwarp();
  }
  if (loss_part) {
    wsum[threadIdx.x] = lsum;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) wsum[threadIdx.x] += wsum[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = wsum[0];
  }
}

template <int LOSS>
cudaError_t launch_refresh_df(int T, int grid, cudaStream_t s, const int64_t* row_ptr, const int32_t* col_idx,
                              const float* rval, const int8_t* y, const float2* w2, int64_t n, void* st,
                              int ws, double* loss_part, int* err) {
  if (T <= 8)
    refresh_df_kernel<LOSS, 8><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w2, n, st, ws, loss_part, err);
  else if (T <= 16)
    refresh_df_kernel<LOSS, 16><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w2, n, st, ws, loss_part, err);
  else
    refresh_df_kernel<LOSS, 32><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w2, n, st, ws, loss_part, err);
  return cudaGetLastError();
}

template <int LOSS, int PREC>
__global__ void rec_from_mq_kernel(const int8_t* y, int64_t n, void* st) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    *st_rec<PREC>(st, i) = slot_coef<LOSS, PREC>(*st_mq(st, i), y[i]);
}

// Mixed precision's stopping test (Section 5.1 reading): the gradient's per-sample coefficient cg in
// FP64 (as FP64 mode computes it from the maintained quantity), kept as a pair of FP32 numbers
// hi + lo in the record's last 8 bytes (mixed mode stores its FP32 coefficient pair in the 8 before),
// so that the KKT column sums run in double-float arithmetic on the FP32 pipe at FP64-grade accuracy.
template <int LOSS>
__global__ void kkt_coef_kernel(const int8_t* y, int64_t n, void* st) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double cg = coef64_of_mixed<LOSS>(*st_mq(st, i), y[i]).cg;
    const float hi = (float)cg;
    reinterpret_cast<float2*>(reinterpret_cast<SampleRec*>(st)[i].c)[1] = make_float2(hi, (float)(cg - (double)hi));
  }
}

// A state slot from one precision's form to the other's (FP64: e^z or b; mixed: the pair of z or
// b), then the coefficients.  A margin that FP64's e^z cannot hold (|z| above about 699) sets the
// range flag.
template <int LOSS, int TO>
__global__ void convert_state_kernel(const int8_t* y, int64_t n, void* st, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double s = *st_mq(st, i);
    double v;
    if constexpr (TO == 1) {
      v = df_slot(df_of(LOSS == 0 ? log(s) : s));
    } else {
      v = slot_value<LOSS, 1>(s);
      if (!mq_ok<LOSS>(v)) atomicOr(err, kErrRange);
    }
    *st_mq(st, i) = v;
    *st_rec<TO>(st, i) = slot_coef<LOSS, TO>(v, y[i]);
  }
}

// At w = 0: z = 0, so E = e^0 = 1 (logistic) and b = 1 - y 0 = 1 (L2-SVM), exactly what a refresh
// from z = Xw gives there.
template <int LOSS, int PREC>
__global__ void state_at_zero_kernel(const int8_t* y, int64_t n, void* st) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = slot_from_z<LOSS, PREC>(0.0, y[i]);
    *st_mq(st, i) = v;
    *st_rec<PREC>(st, i) = slot_coef<LOSS, PREC>(v, y[i]);
  }
}

// ------------------------------------------------------------------------------------ KKT
template <int PREC>
__global__ void __launch_bounds__(kRedThreads) kkt_item_kernel(const Item* items, int64_t n_items, const int32_t* row_idx,
                                                               const float* val, const void* st, double* gpart) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (kRedThreads / 32);
  const SampleRec* rec = reinterpret_cast<const SampleRec*>(st);
  constexpr int U = 4;  // entries per lane in flight: U index/value loads, then U gathers
  for (int64_t i = (int64_t)blockIdx.x * (kRedThreads / 32) + wid; i < n_items; i += warps) {
    const Item it = items[i];
    const int64_t end = it.start + it.len;
    // each lane sums its entries e = start + lane, + 32, ... in that order
    double acc = 0.0;  // FP64 mode
    dfloat dacc = {0.0f, 0.0f};  // mixed mode: x (hi + lo) as an error-free product plus x lo
    for (int64_t e0 = it.start + lane; e0 < end; e0 += 32 * U) {
      int32_t r[U];
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t e = e0 + 32 * u;
        r[u] = e < end ? row_idx[e] : -1;
        v[u] = e < end ? val[e] : 0.0f;
      }
      if constexpr (PREC == 0) {
        double cg[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cg[u] = r[u] >= 0 ? rec[r[u]].c[0] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (r[u] < 0) break;
          acc = fma((double)v[u], cg[u], acc);
        }
      } else {
        float2 cg[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          cg[u] = r[u] >= 0 ? reinterpret_cast<const float2*>(rec[r[u]].c)[1] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (r[u] < 0) break;
          const float ph = v[u] * cg[u].x;
          const float pl = fmaf(v[u], cg[u].y, fmaf(v[u], cg[u].x, -ph));
          dacc = df_add(dacc, dfloat{ph, pl});
        }
      }
    }
    if constexpr (PREC == 0) {
      const double g = warp_sum(acc);
      if (lane == 0) gpart[i] = g;
    } else {
      dacc = df_warp_sum(dacc);
      if (lane == 0) gpart[i] = df_value(dacc);
    }
  }
}

// Per feature: g_j from its items' partial sums, v_j the minimum-norm subgradient; block sums of
// |v_j|.  For shrinking, also g_j (g_out, by feature) and max_j |v_j| (vmax: the bits of a
// non-negative double, whose order as unsigned integers is the order of the values).
template <int PREC>
__global__ void __launch_bounds__(kRedThreads) kkt_col_kernel(const int64_t* item_ptr, const int32_t* perm, int64_t npos,
                                                              const double* gpart, const double* w, double c,
                                                              double l1, double l2, double* block_part,
                                                              double* g_out, unsigned long long* vmax) {
  __shared__ double red[kRedThreads];
  double acc = 0.0, vm = 0.0;
  const int lane = threadIdx.x & 31;
  auto part = [&](int64_t i) { return gpart[i]; };
  // a thread per feature; a feature of more than kLongItems items (a Zipf head column cut into
  // thousands of chunks) is summed by its whole warp, lane-strided and then a fixed butterfly
  constexpr int64_t kLongItems = 64;
  const int64_t stride = (int64_t)gridDim.x * kRedThreads;
  for (int64_t base = (int64_t)blockIdx.x * kRedThreads + (threadIdx.x & ~31); base < npos; base += stride) {
    const int64_t k = base + lane;
    const bool valid = k < npos;
    const int64_t i0 = valid ? item_ptr[k] : 0, i1 = valid ? item_ptr[k + 1] : 0;
    const bool long_col = i1 - i0 > kLongItems;
    double g = 0.0;
    if (!long_col)
      for (int64_t i = i0; i < i1; ++i) g += part(i);
    uint32_t lm = __ballot_sync(0xffffffffu, long_col);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int64_t a = __shfl_sync(0xffffffffu, i0, src), b = __shfl_sync(0xffffffffu, i1, src);
      double sl = 0.0;
      for (int64_t i = a + lane; i < b; i += 32) sl += part(i);
      sl = warp_sum(sl);
      if (lane == src) g = sl;
    }
    if (!valid) continue;
    g *= c;
    const int32_t j = perm[k];
    const double wj = w[j];
    if (l2 != 0.0) g += l2 * wj;  // the smooth part's gradient
    double v;
    if (wj > 0) v = g + l1;
    else if (wj < 0) v = g - l1;
    else v = fabs(g) > l1 ? (g > 0 ? g - l1 : g + l1) : 0.0;
    acc += fabs(v);
    vm = fmax(vm, fabs(v));
    if (g_out) g_out[j] = g;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_part[blockIdx.x] = red[0];
  if (vmax) {
    __syncthreads();
    red[threadIdx.x] = vm;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(vmax, (unsigned long long)__double_as_longlong(red[0]));
  }
}

// ------------------------------------------------------------------------------------ shrinking
// Feature j takes part in the next outer iteration unless w_j = 0 and |g_j| < l1 - M / s (g the
// smooth part's gradient, M the largest |v_j|, s the number of samples; l1 = 1 in the paper):
// outer-iteration shrinking with LIBLINEAR's margin, from the fresh gradient of the stopping test.
__device__ __forceinline__ bool feature_active(double g, double wj, double bound) {
  return wj != 0.0 || fabs(g) >= bound;
}
__device__ __forceinline__ double shrink_bound(const unsigned long long* vmax, int64_t n_samples, double l1) {
  return l1 - __longlong_as_double((long long)*vmax) / (double)n_samples;
}

// out[0] += active features, out[1] += their nonzeros.
__global__ void __launch_bounds__(kRedThreads) active_count_kernel(const double* g, const double* w, int64_t m,
                                                                   const int64_t* col_ptr,
                                                                   const unsigned long long* vmax, int64_t n_samples,
                                                                   double l1, unsigned long long* out) {
  __shared__ unsigned long long red[2][kRedThreads / 32];
  const double bound = shrink_bound(vmax, n_samples, l1);
  unsigned long long cnt = 0, nz = 0;
  for (int64_t j = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; j < m; j += (int64_t)gridDim.x * kRedThreads) {
    if (feature_active(g[j], w[j], bound)) {
      ++cnt;
      nz += (unsigned long long)(col_ptr[j + 1] - col_ptr[j]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = cnt;
    red[1][threadIdx.x >> 5] = nz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int i = 0; i < kRedThreads / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    if (a) atomicAdd(out, a);
    if (b) atomicAdd(out + 1, b);
  }
}

// flags[k] = 1 when feature perm[k] is active (k < m), flags[m] = 0.
__global__ void active_flags_kernel(const int32_t* perm, int64_t m, const double* g, const double* w,
                                    const unsigned long long* vmax, int64_t n_samples, double l1, int64_t* flags) {
  const double bound = shrink_bound(vmax, n_samples, l1);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= m; k += (int64_t)gridDim.x * blockDim.x) {
    if (k == m) { flags[k] = 0; continue; }
    const int32_t j = perm[k];
    flags[k] = feature_active(g[j], w[j], bound) ? 1 : 0;
  }
}

// The active features in partition order: out[pos[k]] = perm[k] for flagged k (a stable filter).
__global__ void compact_kernel(const int32_t* perm, int64_t m, const int64_t* flags, const int64_t* pos, int32_t* out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    if (flags[k]) out[pos[k]] = perm[k];
}

// Block sums of the penalty l1 |w_j| + (l2/2) w_j^2.
__global__ void abs_sum_kernel(const double* w, int64_t m, double l1, double l2, double* block_part) {
  __shared__ double red[kRedThreads];
  double acc = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; j < m; j += (int64_t)gridDim.x * kRedThreads) {
    const double wj = w[j];
    double r = l1 * fabs(wj);
    if (l2 != 0.0) r += 0.5 * l2 * wj * wj;
    acc += r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_part[blockIdx.x] = red[0];
}

// out = scale * sum(a[0..na)) + sum(b[0..nb)), each sum in index order by one thread of a tree
__global__ void finish_sum_kernel(const double* a, int na, double scale, const double* b, int nb, double* out) {
  __shared__ double red[kRedThreads];
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < na; i += kRedThreads) sa += a[i];
  for (int i = threadIdx.x; i < nb; i += kRedThreads) sb += b[i];
  red[threadIdx.x] = sa;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double ta = red[0];
  __syncthreads();
  red[threadIdx.x] = sb;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * ta + red[0];
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 4096) {
  int64_t g = cdiv(n > 0 ? n : 1, threads);
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

// ---------------------------------------------------------------------------------- host API
int64_t scan_workspace_elems(int64_t n) {
  int64_t tot = 0;
  while (n > kScanTile) {
    n = cdiv(n, kScanTile);
    tot += n + 8;
  }
  return tot + 8;
}

cudaError_t scan_exclusive(const int64_t* in, int64_t* out, int64_t n, int64_t* ws, cudaStream_t s, int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = cdiv(n, kScanTile);
  if (nb == 1) {
    scan_tile_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    return post(launches);
  }
  int64_t* sums = ws;
  scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  cudaError_t e = post(launches);
  if (e != cudaSuccess) return e;
  e = scan_exclusive(sums, sums, nb, ws + nb + 8, s, launches);
  if (e != cudaSuccess) return e;
  scan_add_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(out, n, sums);
  return post(launches);
}

int64_t radix_hist_elems(int64_t n) { return 256 * cdiv(n > 0 ? n : 1, kSortTile); }

cudaError_t radix_sort_u64(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int64_t n, int key_bits,
                           int64_t* hist, int64_t* ws, uint64_t** k_out, int32_t** v_out, cudaStream_t s,
                           int64_t* launches) {
  return radix_sort_impl<uint64_t>(k0, v0, k1, v1, n, key_bits, hist, ws, k_out, v_out, s, launches);
}
cudaError_t radix_sort_u32(uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int64_t n, int key_bits,
                           int64_t* hist, int64_t* ws, uint32_t** k_out, int32_t** v_out, cudaStream_t s,
                           int64_t* launches) {
  return radix_sort_impl<uint32_t>(k0, v0, k1, v1, n, key_bits, hist, ws, k_out, v_out, s, launches);
}

__global__ void advance_epoch_kernel(int64_t* epoch_dev) { *epoch_dev += 1; }

cudaError_t advance_epoch(int64_t* epoch_dev, cudaStream_t s, int64_t* launches) {
  advance_epoch_kernel<<<1, 1, 0, s>>>(epoch_dev);
  return post(launches);
}

cudaError_t perm_keys(uint64_t seed, int64_t epoch, const int64_t* epoch_dev, int64_t m, uint64_t* keys, int32_t* vals,
                      cudaStream_t s,
                      int64_t* launches) {
  perm_keys_kernel<<<grid_for(m, 256), 256, 0, s>>>(seed, (uint64_t)epoch, epoch_dev, m, keys, vals);
  return post(launches);
}

cudaError_t build_items(const int32_t* perm, int64_t npos, const int64_t* col_ptr, const double* w, int64_t* cnt_ws,
                        int64_t* item_ptr, Item* items, int64_t* scan_ws, cudaStream_t s, int64_t* launches) {
  item_count_kernel<<<grid_for(npos + 1, 256), 256, 0, s>>>(perm, npos, col_ptr, cnt_ws);
  cudaError_t e = post(launches);
  if (e != cudaSuccess) return e;
  e = scan_exclusive(cnt_ws, item_ptr, npos + 1, scan_ws, s, launches);
  if (e != cudaSuccess) return e;
  item_fill_kernel<<<grid_for(npos, 256), 256, 0, s>>>(perm, npos, col_ptr, item_ptr, w, items);
  return post(launches);
}

cudaError_t build_plan(const Item* items, int64_t n_items, const int64_t* item_ptr, int64_t npos, int32_t P, int64_t nb,
                       int G, int64_t* len_ws, int64_t* item_off, int64_t* plan, int64_t* scan_ws, cudaStream_t s,
                       int64_t* launches) {
  item_len_kernel<<<grid_for(n_items + 1, 256), 256, 0, s>>>(items, n_items, item_ptr, npos, len_ws);
  cudaError_t e = post(launches);
  if (e != cudaSuccess) return e;
  e = scan_exclusive(len_ws, item_off, n_items + 1, scan_ws, s, launches);
  if (e != cudaSuccess) return e;
  plan_kernel<<<grid_for(nb * (G + 1), 256), 256, 0, s>>>(item_ptr, item_off, npos, P, nb, G, plan);
  return post(launches);
}

cudaError_t gather_w(const double* w, const int32_t* perm, int64_t npos, double* w_pos, cudaStream_t s, int64_t* launches) {
  gather_w_kernel<<<grid_for(npos, 256), 256, 0, s>>>(w, perm, npos, w_pos);
  return post(launches);
}

cudaError_t scatter_w(const double* w_pos, const int32_t* perm, int64_t npos, double* w, cudaStream_t s, int64_t* launches) {
  scatter_w_kernel<<<grid_for(npos, 256), 256, 0, s>>>(w_pos, perm, npos, w);
  return post(launches);
}

cudaError_t entry_columns(const int64_t* col_ptr, int64_t m, int64_t nnz, int32_t* entry_col, cudaStream_t s,
                          int64_t* launches) {
  if (nnz <= 0) return cudaSuccess;
  entry_col_kernel<<<grid_for(cdiv(nnz, kSpan), 256), 256, 0, s>>>(col_ptr, m, nnz, entry_col);
  return post(launches);
}

cudaError_t iota_i32(int32_t* v, int64_t n, cudaStream_t s, int64_t* launches) {
  iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n);
  return post(launches);
}

cudaError_t validate_device(const int64_t* col_ptr, const int32_t* row_idx, const float* val, const int8_t* y, int64_t n,
                            int64_t m, int64_t nnz, int* flag, cudaStream_t s, int64_t* launches) {
  validate_kernel<<<grid_for(nnz > n ? nnz : n, 256), 256, 0, s>>>(col_ptr, row_idx, val, y, n, m, nnz, flag);
  cudaError_t e = post(launches);
  if (e != cudaSuccess) return e;
  if (nnz <= 0) return cudaSuccess;
  validate_order_kernel<<<grid_for(cdiv(nnz, kSpan), 256), 256, 0, s>>>(col_ptr, row_idx, m, nnz, flag);
  return post(launches);
}

cudaError_t refresh(int loss, int prec, const int64_t* row_ptr, const int32_t* col_idx, const float* rval,
                    const int8_t* y, const double* w, int64_t n, int64_t m, int64_t nnz, void* w2_scratch,
                    void* st, bool write_state, double* loss_part, int grid, int* err, cudaStream_t s,
                    int64_t* launches) {
  const int ws = write_state ? 1 : 0;
  // without per-block loss partials any block count works: twice the blocks for more loads in flight
  if (!loss_part) grid *= 2;
  if (prec == 1 && w2_scratch) {
    float2* w2 = static_cast<float2*>(w2_scratch);
    split_w_kernel<<<grid_for(m, 256), 256, 0, s>>>(w, m, w2);
    cudaError_t e = post(launches);
    if (e != cudaSuccess) return e;
    // lanes per row from the mean row length: about 4-8 nonzeros per lane
    const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
    const int T = mean < 64.0 ? 8 : (mean < 256.0 ? 16 : 32);
    if (loss == 0) e = launch_refresh_df<0>(T, grid, s, row_ptr, col_idx, rval, y, w2, n, st, ws, loss_part, err);
    else e = launch_refresh_df<1>(T, grid, s, row_ptr, col_idx, rval, y, w2, n, st, ws, loss_part, err);
    if (launches) ++*launches;
    return e;
  }
  if (loss == 0 && prec == 0)
    refresh_kernel<0, 0><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w, n, st, ws, loss_part, err);
  else if (loss == 0)
    refresh_kernel<0, 1><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w, n, st, ws, loss_part, err);
  else if (prec == 0)
    refresh_kernel<1, 0><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w, n, st, ws, loss_part, err);
  else
    refresh_kernel<1, 1><<<grid, kRedThreads, 0, s>>>(row_ptr, col_idx, rval, y, w, n, st, ws, loss_part, err);
  return post(launches);
}

cudaError_t rec_from_mq(int loss, int prec, const int8_t* y, int64_t n, void* st, cudaStream_t s, int64_t* launches) {
  const unsigned g = grid_for(n, 256);
  if (loss == 0 && prec == 0) rec_from_mq_kernel<0, 0><<<g, 256, 0, s>>>(y, n, st);
  else if (loss == 0) rec_from_mq_kernel<0, 1><<<g, 256, 0, s>>>(y, n, st);
  else if (prec == 0) rec_from_mq_kernel<1, 0><<<g, 256, 0, s>>>(y, n, st);
  else rec_from_mq_kernel<1, 1><<<g, 256, 0, s>>>(y, n, st);
  return post(launches);
}

cudaError_t convert_state(int loss, int to_prec, const int8_t* y, int64_t n, void* st, int* err, cudaStream_t s,
                          int64_t* launches) {
  const unsigned g = grid_for(n, 256);
  if (loss == 0 && to_prec == 0) convert_state_kernel<0, 0><<<g, 256, 0, s>>>(y, n, st, err);
  else if (loss == 0) convert_state_kernel<0, 1><<<g, 256, 0, s>>>(y, n, st, err);
  else if (to_prec == 0) convert_state_kernel<1, 0><<<g, 256, 0, s>>>(y, n, st, err);
  else convert_state_kernel<1, 1><<<g, 256, 0, s>>>(y, n, st, err);
  return post(launches);
}

cudaError_t state_at_zero(int loss, int prec, const int8_t* y, int64_t n, void* st, cudaStream_t s, int64_t* launches) {
  const unsigned g = grid_for(n, 256);
  if (loss == 0 && prec == 0) state_at_zero_kernel<0, 0><<<g, 256, 0, s>>>(y, n, st);
  else if (loss == 0) state_at_zero_kernel<0, 1><<<g, 256, 0, s>>>(y, n, st);
  else if (prec == 0) state_at_zero_kernel<1, 0><<<g, 256, 0, s>>>(y, n, st);
  else state_at_zero_kernel<1, 1><<<g, 256, 0, s>>>(y, n, st);
  return post(launches);
}

cudaError_t kkt_l1(int loss, int prec, const int8_t* y, int64_t n, const Item* items, int64_t n_items,
                   const int64_t* item_ptr, const int32_t* perm, int64_t npos, const int32_t* row_idx, const float* val,
                   void* st, const double* w, double c, double l1, double l2, double* gpart, double* block_part,
                   int grid, double* out, cudaStream_t s, int64_t* launches, double* g_out, unsigned long long* vmax) {
  cudaError_t e;
  if (prec == 1) {  // the FP64 coefficients the mixed-precision item pass reads
    if (loss == 0) kkt_coef_kernel<0><<<grid_for(n, 256), 256, 0, s>>>(y, n, st);
    else kkt_coef_kernel<1><<<grid_for(n, 256), 256, 0, s>>>(y, n, st);
    if ((e = post(launches)) != cudaSuccess) return e;
  }
  // the item pass writes one sum per item, no block partials: twice the blocks for more loads in flight
  if (prec == 0) kkt_item_kernel<0><<<2 * grid, kRedThreads, 0, s>>>(items, n_items, row_idx, val, st, gpart);
  else kkt_item_kernel<1><<<2 * grid, kRedThreads, 0, s>>>(items, n_items, row_idx, val, st, gpart);
  e = post(launches);
  if (e != cudaSuccess) return e;
  if (prec == 0)
    kkt_col_kernel<0><<<grid, kRedThreads, 0, s>>>(item_ptr, perm, npos, gpart, w, c, l1, l2, block_part, g_out, vmax);
  else
    kkt_col_kernel<1><<<grid, kRedThreads, 0, s>>>(item_ptr, perm, npos, gpart, w, c, l1, l2, block_part, g_out, vmax);
  e = post(launches);
  if (e != cudaSuccess) return e;
  finish_sum_kernel<<<1, kRedThreads, 0, s>>>(block_part, grid, 1.0, nullptr, 0, out);
  return post(launches);
}

cudaError_t active_count(const double* g, const double* w, int64_t m, const int64_t* col_ptr,
                         const unsigned long long* vmax, int64_t n_samples, double l1, unsigned long long* out,
                         cudaStream_t s, int64_t* launches) {
  active_count_kernel<<<grid_for(m, kRedThreads, 1024), kRedThreads, 0, s>>>(g, w, m, col_ptr, vmax, n_samples, l1,
                                                                              out);
  return post(launches);
}

cudaError_t compact_active(const int32_t* perm, int64_t m, const double* g, const double* w,
                           const unsigned long long* vmax, int64_t n_samples, double l1, int64_t* flags_ws,
                           int64_t* pos_ws, int64_t* scan_ws, int32_t* out, cudaStream_t s, int64_t* launches) {
  active_flags_kernel<<<grid_for(m + 1, 256), 256, 0, s>>>(perm, m, g, w, vmax, n_samples, l1, flags_ws);
  cudaError_t e = post(launches);
  if (e != cudaSuccess) return e;
  e = scan_exclusive(flags_ws, pos_ws, m + 1, scan_ws, s, launches);
  if (e != cudaSuccess) return e;
  compact_kernel<<<grid_for(m, 256), 256, 0, s>>>(perm, m, flags_ws, pos_ws, out);
  return post(launches);
}

cudaError_t objective_finish(const double* loss_part, int nb, const double* w, int64_t m, double c, double l1,
                             double l2, double* block_part, int grid, double* out, cudaStream_t s, int64_t* launches) {
  abs_sum_kernel<<<grid, kRedThreads, 0, s>>>(w, m, l1, l2, block_part);
  cudaError_t e = post(launches);
  if (e != cudaSuccess) return e;
  finish_sum_kernel<<<1, kRedThreads, 0, s>>>(loss_part, nb, c, block_part, grid, out);
  return post(launches);
}

}  // namespace pcdn
