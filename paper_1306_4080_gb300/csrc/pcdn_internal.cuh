// Internal device-side definitions of the GB300 PCDN solver.
//
// Layout in HBM (per problem):
//   X by columns: col_ptr int64[m+1], row_idx int32[nnz], val f32[nnz]   (read-only)
//   X by rows (mirror, for z = Xw): row_ptr int64[n+1], col_idx int32[nnz], rval f32[nnz]
//   y int8[n]; w f64[m]
//   mq f64[n]        maintained quantity: e^{w^T x_i} (logistic) or b_i = 1 - y_i w^T x_i (L2-SVM)
//   rec {cg, ch}[n]  per-sample coefficients of the column reductions, derived from mq:
//                    g_j = c sum_i x_ij cg_i, h_j = c sum_i x_ij^2 ch_i (f64 pairs, or f32 pairs
//                    in mixed precision).  One 8/16-byte gather per nonzero.
//   delta f64[n]     d^T x_i of the current bundle; zero outside the bundle step
//   touched u32[ceil(n/32)]  bit i set when row i received a d_j x_ij != 0 this bundle
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pcdn {

constexpr int kWarp = 32;
constexpr int kChunk = 512;        // max nonzeros of one column work item (512: best of 512, 1024, 2048 measured)
constexpr int kMaxK = 8;           // max step sizes per line-search pass
constexpr int kWalkThreads = 256;  // threads per walker block
constexpr int kWalkWarps = kWalkThreads / kWarp;
constexpr int kWarpRowCap = 256;   // touched rows whose values a warp stages at once
constexpr int kICap = 256;         // work items staged per batch of the column pass
constexpr int kECap = 2048;        // nonzeros staged per batch (= 8 per thread)
constexpr int kSplitCap = 64;      // chunks of split columns a block remembers for its deferred scatter
constexpr int kWarpChunks = 256;   // split columns of at most this many chunks are combined by one warp

constexpr int kErrTimeout = 1;
constexpr int kErrNumeric = 2;       // non-finite g, h or d
constexpr int kErrRange = 4;         // maintained quantity out of range (FP64's e^{w^T x} past about e^699)
constexpr int kErrRefresh = 8;       // z = Xw out of range on a recompute (FP64 |z| > 700, mixed not finite)

// One column work item: nonzeros [start, start+len) of the feature at permutation position pos,
// chunk `chunk` of `nch` chunks of that column.
// w is the feature's weight when the items are built: a bundle's own weights change only in its
// own step, so this is the value its column pass needs.
struct Item {
  int64_t start;
  int32_t len;
  int32_t pos;
  int32_t nch;
  int32_t chunk;
  double w;
};

// d^T x per row: FP64 in FP64 mode; FP32 in mixed mode, whose per-row arithmetic is FP32 anyway
// (FP64 instructions, conversions included, run at about 1/40 of the FP32 rate on this part).
template <int PREC> using DeltaT = typename std::conditional<PREC == 0, double, float>::type;

template <int PREC> struct RecT;
template <> struct __align__(16) RecT<0> { double cg, ch; };
template <> struct __align__(8) RecT<1> { float cg, ch; };

// Per-sample state: one 32-byte record per sample (one L2 sector), so that a pass over the touched
// samples reads and writes each one with a single access:
//   +0  mq   the maintained quantity (e^{w^T x_i}, or b_i = 1 - y_i w^T x_i)
//   +8  bak  mq before the bundle's speculative update (row-sorted walker)
//   +16 the column reductions' coefficient pair: RecT<0> (two doubles) or RecT<1> (two floats)
struct __align__(32) SampleRec {
  double mq;
  double bak;
  double c[2];
};
constexpr int kStateBytes = sizeof(SampleRec);
__host__ __device__ __forceinline__ double* st_mq(void* st, int64_t i) {
  return &reinterpret_cast<SampleRec*>(st)[i].mq;
}
__host__ __device__ __forceinline__ const double* st_mq(const void* st, int64_t i) {
  return &reinterpret_cast<const SampleRec*>(st)[i].mq;
}
template <int PREC>
__host__ __device__ __forceinline__ RecT<PREC>* st_rec(void* st, int64_t i) {
  return reinterpret_cast<RecT<PREC>*>(reinterpret_cast<SampleRec*>(st)[i].c);
}
template <int PREC>
__host__ __device__ __forceinline__ const RecT<PREC>* st_rec(const void* st, int64_t i) {
  return reinterpret_cast<const RecT<PREC>*>(reinterpret_cast<const SampleRec*>(st)[i].c);
}

// Decision of a line-search pass, written by the last block to arrive.
enum : int32_t { kDecAccept = 0, kDecContinue = 1, kDecCap = 2 };
struct Decision {
  int32_t state;
  int32_t q;      // accepted q (accept), next q0 (continue), q_max (cap)
  double alpha;
  double Delta;
  double dF;
  float alpha_f;  // alpha in FP32
};

// Per-pass sums: [0] sum g d, [1] sum h d^2, [2] sum |w+d|-|w|, [3, 3+K) sum |w + a_q d| - |w|,
// [3+K, 3+2K) line-search sums, [3+2K] a speculative state left the usable range, [3+2K+1] warps that
// could not write the full step's state in the line-search pass
constexpr int kPartStride = 3 + 2 * kMaxK + 2;
constexpr int kAccPad = 16;  // doubles per line-search accumulator (128 bytes)

struct WalkParams {
  // problem
  int64_t n, m, nnz;
  const int64_t* col_ptr;
  const int32_t* row_idx;
  const float* val;
  const int8_t* y;          // labels, padded to a multiple of 16 bytes (read as aligned words)
  double c;
  // state
  double* w_pos;            // w in position order (the partition's order) during the walk
  void* st;                 // [n] SampleRec
  void* delta;              // [n] d^T x of the bundle per row: DeltaT<PREC> (double or float)
  uint32_t* touched;
  int64_t nwords;
  // partition of this walk
  const int32_t* perm;      // position -> feature
  const Item* items;        // work items in position order
  const int64_t* item_ptr;  // [npos+1] first item of each position
  const int64_t* plan;      // [(t_end) * (gridDim.x + 1)] first item of each block in each bundle
  int64_t npos;             // number of positions (m for a solve, P for a single bundle)
  int32_t P;
  int64_t t_begin, t_end;   // bundles [t_begin, t_end) of this launch
  // bundle-local scratch, indexed by position within the bundle
  double* gk;
  double* hk;
  double* dk;
  double* part;             // [2 * items] partial (g, h) of chunks of split columns
  uint32_t* col_cnt;        // [2][P] chunks of a split column that published sums, by bundle parity
  uint32_t* anynz;          // unused
  // reductions and barriers
  double* lsacc;            // [3][kPartStride][kAccPad] sums over blocks of the line-search fields, by
                            // pass mod 3 (FP64 atomic adds; each field on its own 128-byte line)
  uint32_t* bar_count;
  uint32_t* bar_gen;
  uint32_t spin_limit;      // polls a wait may make before it gives up
  uint64_t wait_ns;         // global-timer nanoseconds a wait may last before it gives up
  // Armijo
  double sigma, beta, gamma, nu;
  float c_f, nu_f;          // c and nu in FP32 (mixed mode's column directions)
  // penalty l1 ||w||_1 + (l2/2) ||w||^2 (the paper's problem: l1 = 1, l2 = 0)
  double l1, l2;
  float l1_f, l2_f;
  int32_t q_max, K;         // K step sizes per line-search pass after the first
  int32_t K1;               // step sizes in the first pass
  // outputs
  int32_t* tr_q;            // [t_end] per-bundle records (indexed by bundle)
  double* tr_alpha;
  double* tr_Delta;
  double* tr_dF;
  unsigned long long* counters;  // [8]: ls_steps, cap_hits, passes, nnz, rows, bundles, coord_updates, nonzero-d bundles
  unsigned long long* bar1;      // barrier 1: arrivals
  uint32_t* nzc;                 // [2] blocks that found a nonzero direction, by barrier-1 parity
  int* err;
  // row-sorted layout (walk_rows_kernel): the entries of every bundle's columns grouped by row
  // (rows ascending, columns ascending within a row); entry s of bundle t lies in
  // [br_ptr[t], br_ptr[t+1]) and holds its row, its position k within the bundle and its value
  const int32_t* br_row;
  const int32_t* br_k;
  const float* br_val;
  const int64_t* br_ptr;    // [bundles + 1]
  const int64_t* br_plan;   // [bundles * (gridDim.x + 1)]: first entry of each block, at a row start
  double* lspart;           // [2][kPartStride][gridDim.x] per-block partial sums, by bundle parity
  float* dkf;               // [2 * P_cap] d in FP32 (mixed mode), by bundle parity
  int64_t P_cap;            // stride of the parity halves of gk, hk, dk, dkf
  int x_vec;                // row_idx and val are 16-byte aligned: 16-byte copies
  int br_vec;               // br_row, br_k, br_val are 16-byte aligned
};

// ---------------------------------------------------------------- memory-order helpers
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_acqrel_add_u32(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) { red_add_f64(p, v); }
__device__ __forceinline__ void red_add(float* p, float v) { red_add_f32(p, v); }
__device__ __forceinline__ void red_or_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------- bounded waits
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool err_set(const WalkParams& p) { return ld_volatile_int(p.err) != 0; }

// A wait between thread blocks gives up after p.spin_limit polls or p.wait_ns nanoseconds of the
// global timer, whichever comes first (the time bound keeps a legitimate wait on a GPU shared with
// many other kernels from giving up early; the poll bound lets a test make a wait run out).
// poll() returns 0 to keep waiting, 1 when the wait gave up (kErrTimeout recorded), 2 when another
// block recorded an error.
struct Waiter {
  uint32_t spins = 0;
  uint64_t t0 = 0;
  __device__ __forceinline__ int poll(const WalkParams& p) {
    ++spins;
    if (spins > p.spin_limit) {
      atomicOr(p.err, kErrTimeout);
      return 1;
    }
    if ((spins & 255u) == 0) {
      if (err_set(p)) return 2;
      const uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > p.wait_ns) {
        atomicOr(p.err, kErrTimeout);
        return 1;
      }
    }
    return 0;
  }
};

// ---------------------------------------------------------------- grid barriers
// The shared-memory struct SH of a walker holds: int abort, has_nz, nonzero; int scan_tot[].

// Plain barrier over the grid.  Returns false when the launch must end (a wait gave up, or a
// block recorded an error while this one waited).  With one block, a GPU-scope fence stands in for
// the release/acquire pair, so that the block's atomics (performed in L2) are seen by its later
// loads.
template <class SH>
__device__ bool grid_barrier(const WalkParams& p, uint32_t& idx, SH& sh) {
  __syncthreads();
  if (gridDim.x == 1 && threadIdx.x == 0) __threadfence();
  if (gridDim.x > 1) {
    if (threadIdx.x == 0) {
      const uint32_t target = (idx + 1) * gridDim.x;
      red_release_add_u32(p.bar_count, 1u);
      Waiter wt;
      int abort = 0;
      while (ld_acquire_u32(p.bar_count) < target) {
        if (wt.poll(p)) { abort = 1; break; }
      }
      sh.abort = abort;
    }
  }
  ++idx;
  __syncthreads();
  return !sh.abort;
}

// Split-phase form of grid_barrier: work between arrive and wait must neither write what other
// blocks read after the barrier nor read what they write before it.
__device__ __forceinline__ void grid_arrive(const WalkParams& p) {
  __syncthreads();
  if (gridDim.x > 1 && threadIdx.x == 0) red_release_add_u32(p.bar_count, 1u);
}
template <class SH>
__device__ bool grid_wait(const WalkParams& p, uint32_t& idx, SH& sh) {
  if (gridDim.x == 1 && threadIdx.x == 0) __threadfence();
  if (gridDim.x > 1 && threadIdx.x == 0) {
    const uint32_t target = (idx + 1) * gridDim.x;
    Waiter wt;
    int abort = 0;
    while (ld_acquire_u32(p.bar_count) < target) {
      if (wt.poll(p)) { abort = 1; break; }
    }
    sh.abort = abort;
  }
  ++idx;
  __syncthreads();
  return !sh.abort;
}

// Barrier 1: each block arrives on its own counter (bar1) and, when it found a nonzero direction,
// first adds 1 to the flag counter of the barrier's parity (nzc[n1 & 1]); the waiters learn whether
// any block did by comparing that counter with its value at the barrier of the same parity two
// barriers earlier (seen[0..1]).  A block that runs ahead can only reach the next barrier 1 of the
// same parity after every block has passed the one in between, so every block reads the same value.
template <class SH>
__device__ bool grid_barrier_flag(const WalkParams& p, uint32_t& n1, uint32_t& seen0, uint32_t& seen1, SH& sh) {
  __syncthreads();
  if (gridDim.x > 1) {
    const int par = (int)(n1 & 1);
    if (threadIdx.x == 0) {
      const uint64_t target = (uint64_t)(n1 + 1) * gridDim.x;
      if (sh.has_nz) atomicAdd(p.nzc + par, 1u);
      red_release_add_u64(p.bar1, 1ull);
      Waiter wt;
      int abort = 0;
      while (ld_acquire_u64(p.bar1) < target) {
        if (wt.poll(p)) { abort = 1; break; }
      }
      const uint32_t v = ld_acquire_u32(p.nzc + par);
      sh.nonzero = v != (par ? seen1 : seen0);
      sh.abort = abort;
      sh.scan_tot[0] = (int)v;
    }
    __syncthreads();
    if (par) seen1 = (uint32_t)sh.scan_tot[0];
    else seen0 = (uint32_t)sh.scan_tot[0];
  } else if (threadIdx.x == 0) {
    __threadfence();
    sh.nonzero = sh.has_nz;
  }
  ++n1;
  __syncthreads();
  return !sh.abort;
}

// Streaming loads of X (ld.global.cs: read about once per bundle step, so evicted first and the
// per-sample vectors keep their L2 lines).
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream_f32(const float* p) { return __ldcs(p); }

// ---------------------------------------------------------------- asynchronous copies to shared memory
// cp.async (global -> shared without registers); each thread waits for its own copies, a block
// barrier then makes all of them visible.  X goes through with an evict-first L2 policy.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async4_stream(void* dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------- warp reductions (fixed tree)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- direction (Eq. 4 / Eq. 5)
// argmin_d g d + h d^2/2 + l1 |w + d|; Eq. 5's branch conditions read with the +/-l1 terms (l1 = 1
// in the paper).
__device__ __forceinline__ double newton_direction(double g, double h, double w, double l1) {
  if (g + l1 <= h * w) return -(g + l1) / h;
  if (g - l1 >= h * w) return -(g - l1) / h;
  return -w;
}
// The same in FP32 (mixed mode), keeping d = -w exact.  A quotient past FP32's range (h near nu
// against a large g, as when every sample of the column has |w^T x_i| beyond about 90, where the
// logistic's FP32 curvature underflows) is formed in FP64 instead, so that d stays finite; its FP32
// copy is then infinite and the line search rejects each trial step.
__device__ __forceinline__ double newton_direction_f(float g, float h, float wf, double w, float l1) {
  float num;
  if (g + l1 <= h * wf) num = -(g + l1);
  else if (g - l1 >= h * wf) num = -(g - l1);
  else return -w;
  const float q = num / h;
  return isinf(q) ? (double)num / (double)h : (double)q;
}

// ---------------------------------------------------------------- double-float sums
// A sum carried as an unevaluated pair hi + lo of FP32 numbers (error-free TwoSum, Knuth), about
// 48 significant bits.  GB300 runs FP32 at many times its FP64 rate, so the mixed-precision path
// accumulates its FP64-grade sums in this form.
struct dfloat {
  float hi, lo;
};
__device__ __forceinline__ dfloat df_make(double v) {
  dfloat r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = err + a.lo + b.lo;
  dfloat r;
  r.hi = s + lo;
  r.lo = lo - (r.hi - s);
  return r;
}
__device__ __forceinline__ dfloat df_add_f(dfloat a, float b) {
  dfloat t;
  t.hi = b;
  t.lo = 0.0f;
  return df_add(a, t);
}
__device__ __forceinline__ double df_value(dfloat a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat{-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat df_abs(dfloat a) { return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? df_neg(a) : a; }
// scaling by a power of two is exact
__device__ __forceinline__ dfloat df_scale(dfloat a, float s) { return dfloat{a.hi * s, a.lo * s}; }
__device__ __forceinline__ dfloat df_shfl_xor(dfloat a, int o) {
  dfloat r;
  r.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
  r.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
  return r;
}
__device__ __forceinline__ dfloat df_warp_sum(dfloat a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return a;
}
// ---------------------------------------------------------------- per-sample coefficients
// Logistic (Eq. 11): with E = e^{z}, s = 1/(1+E), p = E/(1+E):
//   (tau(y z) - 1) y = -s (y = +1) or p (y = -1);  tau (1 - tau) = p s.
// L2-SVM (Appendix A, proof of Lemma 1(b)): b = 1 - y z; cg = -2 y max(b, 0), ch = 2 [b > 0].
template <int LOSS, int PREC> struct RowCoef;

template <> struct RowCoef<0, 0> {
  static __device__ __forceinline__ RecT<0> make(double E, int y) {
    double s = 1.0 / (1.0 + E);
    double p = E * s;
    RecT<0> r;
    r.cg = y > 0 ? -s : p;
    r.ch = p * s;
    return r;
  }
};
// Mixed precision keeps the maintained quantity as a double-float pair in the record's 8-byte slot:
// the margin z = w^T x_i for the logistic loss (the paper's maintained e^{w^T x_i} is e^z) and
// b = 1 - y w^T x_i for the L2-SVM.  An update adds the FP32 step alpha d^T x_i to the pair
// (error-free, on the FP32 pipe), so no per-sample work of this mode runs on the FP64 pipe, and the
// pair carries about 48 significant bits.
__device__ __forceinline__ dfloat slot_df(double s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(s);
  return dfloat{__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32))};
}
__device__ __forceinline__ double df_slot(dfloat v) {
  return __longlong_as_double((long long)((unsigned long long)__float_as_uint(v.hi) |
                                          ((unsigned long long)__float_as_uint(v.lo) << 32)));
}
// double-float of a double (the FP64 conversions of a once-per-outer-iteration pass)
__device__ __forceinline__ dfloat df_of(double v) {
  dfloat r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}
__device__ __forceinline__ double df_to_double(dfloat v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ bool df_pos(dfloat v) { return v.hi > 0.0f || (v.hi == 0.0f && v.lo > 0.0f); }

template <> struct RowCoef<0, 1> {
  // from the margin z: e^z in FP32 on whichever side keeps it at most 1
  static __device__ __forceinline__ RecT<1> make(dfloat z, int y) {
    const float zf = z.hi;
    float p, s;
    if (zf <= 0.0f) {  // 1 + e in [1, 2]: the fast reciprocal is accurate to 2 ulp
      const float e = expf(zf);
      s = __fdividef(1.0f, 1.0f + e);
      p = e * s;
    } else {
      const float r = expf(-zf);
      p = __fdividef(1.0f, 1.0f + r);
      s = r * p;
    }
    RecT<1> o;
    o.cg = y > 0 ? -s : p;
    o.ch = p * s;
    return o;
  }
};
template <> struct RowCoef<1, 0> {
  static __device__ __forceinline__ RecT<0> make(double b, int y) {
    RecT<0> r;
    r.cg = b > 0.0 ? -2.0 * (double)y * b : (y > 0 ? -0.0 : 0.0);
    r.ch = b > 0.0 ? 2.0 : 0.0;
    return r;
  }
};
template <> struct RowCoef<1, 1> {
  static __device__ __forceinline__ RecT<1> make(dfloat b, int y) {
    RecT<1> r;
    const bool pos = df_pos(b);
    r.cg = pos ? (y > 0 ? -2.0f * b.hi : 2.0f * b.hi) : (y > 0 ? -0.0f : 0.0f);
    r.ch = pos ? 2.0f : 0.0f;
    return r;
  }
};
// Every coefficient pair carries its sample's label in the sign bit of cg: set for y = +1 (cg is
// -s <= 0 for the logistic loss, -2 b for the L2-SVM, -0 when zero), clear for y = -1.
__device__ __forceinline__ int label_from_cg(double cg) { return __double_as_longlong(cg) < 0 ? 1 : -1; }
__device__ __forceinline__ int label_from_cg(float cg) { return __float_as_int(cg) < 0 ? 1 : -1; }

// Maintained quantity is usable: finite, and for the logistic loss E = e^{w^T x} in [2^-1009,
// 2^1010), i.e. |w^T x| below about 699.  Tested on the bits (sign and exponent), which keeps the
// test off the FP64 pipe.
template <int LOSS>
__device__ __forceinline__ bool mq_ok(double v) {
  const uint32_t se = (uint32_t)((unsigned long long)__double_as_longlong(v) >> 52);  // sign and exponent
  if (LOSS == 0) return se >= 14u && se <= 2032u;
  return (se & 0x7ffu) != 0x7ffu;
}
// Mixed precision's pair (the margin z itself for the logistic loss, b for the L2-SVM) is usable
// whenever it is finite: every coefficient it yields is formed with e^{-|z|}, which never overflows.
template <int LOSS>
__device__ __forceinline__ bool mq_ok(dfloat v) {
  return isfinite(v.hi) && isfinite(v.lo);
}

// The coefficient pair and usability of a record's state slot (a double in FP64 mode, a
// double-float pair in mixed mode).
template <int LOSS, int PREC>
__device__ __forceinline__ RecT<PREC> slot_coef(double slot, int y) {
  if constexpr (PREC == 0) return RowCoef<LOSS, 0>::make(slot, y);
  else return RowCoef<LOSS, 1>::make(slot_df(slot), y);
}
template <int LOSS, int PREC>
__device__ __forceinline__ bool slot_ok(double slot) {
  if constexpr (PREC == 0) return mq_ok<LOSS>(slot);
  else return mq_ok<LOSS>(slot_df(slot));
}
// FP64 coefficients of a mixed-precision slot.  Logistic: p = 1/(1+e^{-z}) and s = 1/(1+e^{z}) with
// the exponential taken on whichever side keeps it at most 1 (the same values as from E = e^z, for
// any finite z); L2-SVM: from b as in FP64 mode.
template <int LOSS>
__device__ __forceinline__ RecT<0> coef64_of_mixed(double slot, int y) {
  const double v = df_to_double(slot_df(slot));
  if constexpr (LOSS == 1) {
    return RowCoef<1, 0>::make(v, y);
  } else {
    double p, s;
    if (v <= 0.0) {
      const double e = exp(v);
      s = 1.0 / (1.0 + e);
      p = e * s;
    } else {
      const double r = exp(-v);
      p = 1.0 / (1.0 + r);
      s = r * p;
    }
    RecT<0> o;
    o.cg = y > 0 ? -s : p;
    o.ch = p * s;
    return o;
  }
}
// The state slot at a sample's z = w^T x_i (refresh): FP64 e^z or 1 - y z; mixed the pair of z or 1 - y z.
template <int LOSS, int PREC>
__device__ __forceinline__ double slot_from_z(double z, int y) {
  if constexpr (PREC == 0) return LOSS == 0 ? exp(z) : 1.0 - (double)y * z;
  else return df_slot(df_of(LOSS == 0 ? z : 1.0 - (double)y * z));
}
// The maintained quantity of the slot as a double: FP64 e^z or b; mixed e^z (from z) or b.
template <int LOSS, int PREC>
__device__ __forceinline__ double slot_value(double slot) {
  if constexpr (PREC == 0) return slot;
  else return LOSS == 0 ? exp(df_to_double(slot_df(slot))) : df_to_double(slot_df(slot));
}

// ---------------------------------------------------------------- line-search row terms
// Mixed precision, logistic: the loss change of a row at u = alpha d^T x_i is its first-order part
// cg u (cg the row's gradient coefficient) plus the remainder
//   R(v; a) = log(1 + a (e^v - 1)) - a v >= 0,  a = min(p, s) = 1/(1 + e^{|z|}) in [0, 1/2],
//   v = +/- alpha d^T x_i (z = w^T x_i),
// the cumulant generating function of a Bernoulli(a) variable minus its first cumulant.  For
// |v| <= 1/8 it is summed as the cumulant series up to order 7 (truncation below 1e-9 relative);
// beyond, evaluated directly (cancellation at most a factor 32).  For v > 20 it is taken from |z|:
// 1 + a (e^v - 1) = (e^{|z|} + e^v) / (1 + e^{|z|}), so with t = v - |z|
//   R = max(t, 0) + log1p(e^{-|t|}) - log1p(e^{-|z|}) - a v,
// which stays exact where a underflows FP32 (|z| beyond about 87: a confidently classified
// sample that a large trial step would flip, whose change is then about t, not 0).
__device__ __forceinline__ float lr_remainder(float a, float v, float az) {
  const float av = fabsf(v);
  if (!(av <= 3.0e38f)) return __int_as_float(0x7f800000);  // an infinite trial step: +inf, rejected
  if (av <= 0.125f) {
    float b = 1.0f - a, ab = a * b, t = b - a;
    float k2 = ab, k3 = ab * t, k4 = ab * (1.0f - 6.0f * ab), k5 = ab * t * (1.0f - 12.0f * ab);
    float k6 = ab * (1.0f - 30.0f * ab + 120.0f * ab * ab);
    float k7 = ab * t * (1.0f - 60.0f * ab + 360.0f * ab * ab);
    float s = k6 * (1.0f / 720.0f) + v * (k7 * (1.0f / 5040.0f));
    s = k5 * (1.0f / 120.0f) + v * s;
    s = k4 * (1.0f / 24.0f) + v * s;
    s = k3 * (1.0f / 6.0f) + v * s;
    s = k2 * 0.5f + v * s;
    return v * v * s;
  }
  float r;
  if (v > 20.0f) {
    const float t = v - az;
    r = fmaxf(t, 0.0f) + log1pf(expf(-fabsf(t))) - log1pf(expf(-az)) - a * v;
  } else {
    r = log1pf(a * expm1f(v)) - a * v;
  }
  return fmaxf(r, 0.0f);
}

// Mixed precision, L2-SVM: remainder of max(0, b - v)^2 - max(0, b)^2 after its first-order part
// -2 max(b, 0) v (= cg alpha d^T x_i), v = alpha y_i d^T x_i formed in FP32 (exact for
// beta = 1/2).  The sign of b - v is exact: the pair's high part decides unless it equals v,
// then its low part.
__device__ __forceinline__ float svm_remainder(dfloat b, float vf) {
  const float bf = b.hi;
  const bool b_pos = df_pos(b);
  const bool bn_pos = (bf != vf) ? (bf > vf) : (b.lo > 0.0f);
  if (b_pos) return bn_pos ? vf * vf : bf * (2.0f * vf - bf);
  if (bn_pos) {
    const float t = bf - vf;
    return t * t;
  }
  return 0.0f;
}

// ---------------------------------------------------------------- exact sums
// A sum carried exactly as an integer in units of 2^-88, in three signed limbs of 42 bits,
// v = l2 2^84 + l1 2^42 + l0 (l2 a signed 64-bit word, l0 and l1 in [0, 2^42) after fx_norm), plus
// flags for a term that is not finite or whose magnitude reaches 2^35 (1: positive, 2: negative,
// 4: NaN); a flagged sum reads as +-inf or NaN, which fails the line-search test.  Capped terms keep
// any sum of fewer than 2^24 of them inside l2's range (|v| < 2^59), so the limbs never wrap.  A
// line-search term that large is a trial step the test rejects anyway (an increase of the loss
// beyond what all samples' losses could give back).  Terms are truncated toward zero below 2^-88.  Integer additions are associative, so the sum does
// not depend on the order in which terms, lanes, warps or blocks are added: results repeat bit for
// bit whatever the order of atomic additions, on the integer pipes (this part's FP64 pipe runs at a
// small fraction of its FP32 and integer rates).
struct Fx {
  long long l0 = 0, l1 = 0, l2 = 0;
  unsigned fl = 0;
};
constexpr long long kFxMask = (1ll << 42) - 1;

__device__ __forceinline__ void fx_norm(Fx& a) {
  long long c = a.l0 >> 42;  // arithmetic shift: floor division
  a.l0 -= c << 42;
  a.l1 += c;
  c = a.l1 >> 42;
  a.l1 -= c << 42;
  a.l2 += c;
}
__device__ __forceinline__ void fx_add(Fx& a, const Fx& b) {
  a.l0 += b.l0;
  a.l1 += b.l1;
  a.l2 += b.l2;
  a.fl |= b.fl;
}
// adds (or subtracts) m 2^s (units of 2^-88; m < 2^53, s <= 122 and m 2^s < 2^147)
__device__ __forceinline__ void fx_add_bits(Fx& a, unsigned long long m, int s, bool neg) {
  if (s < 0) {
    if (s <= -53) return;
    m >>= -s;
    s = 0;
  }
  long long p0, p1, p2;
  if (s >= 84) {
    p0 = 0;
    p1 = 0;
    p2 = (long long)(m << (s - 84));
  } else {
    const int k = s >= 42 ? 1 : 0, r = s - 42 * k;
    const long long lo = (long long)((m << r) & (unsigned long long)kFxMask);
    const unsigned long long hi = r == 0 ? (m >> 42) : (m >> (42 - r));
    if (k == 0) {
      p0 = lo;
      p1 = (long long)(hi & (unsigned long long)kFxMask);
      p2 = (long long)(hi >> 42);
    } else {
      p0 = 0;
      p1 = lo;
      p2 = (long long)hi;
    }
  }
  if (neg) {
    a.l0 -= p0;
    a.l1 -= p1;
    a.l2 -= p2;
  } else {
    a.l0 += p0;
    a.l1 += p1;
    a.l2 += p2;
  }
}
__device__ __forceinline__ void fx_add_f(Fx& a, float x) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xffu);
  const bool neg = (u >> 31) != 0;
  if (e == 0xff) {
    a.fl |= (u & 0x7fffffu) ? 4u : (neg ? 2u : 1u);
    return;
  }
  if (e > 161) {  // |x| >= 2^35
    a.fl |= neg ? 2u : 1u;
    return;
  }
  if (e == 0) return;  // below 2^-126: far below the unit
  fx_add_bits(a, (unsigned long long)((u & 0x7fffffu) | 0x800000u), e - 62, neg);
}
__device__ __forceinline__ void fx_add_d(Fx& a, double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ffu);
  const bool neg = (u >> 63) != 0;
  if (e == 0x7ff) {
    a.fl |= (u & 0xfffffffffffffull) ? 4u : (neg ? 2u : 1u);
    return;
  }
  if (e > 1057) {  // |x| >= 2^35
    a.fl |= neg ? 2u : 1u;
    return;
  }
  if (e == 0) return;
  fx_add_bits(a, (u & 0xfffffffffffffull) | (1ull << 52), e - 987, neg);
}
__device__ __forceinline__ Fx fx_warp_sum(Fx a) {
  fx_norm(a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.l0 += __shfl_xor_sync(0xffffffffu, a.l0, o);
    a.l1 += __shfl_xor_sync(0xffffffffu, a.l1, o);
    a.l2 += __shfl_xor_sync(0xffffffffu, a.l2, o);
  }
  a.fl = __reduce_or_sync(0xffffffffu, a.fl);
  fx_norm(a);
  return a;
}
// the sum rounded to FP64 (the limbs normalised first; l0, l1 convert exactly)
__device__ __forceinline__ double fx_value(Fx a) {
  if (a.fl & 4u || (a.fl & 3u) == 3u) return __longlong_as_double(0x7ff8000000000000ll);
  if (a.fl & 1u) return __longlong_as_double(0x7ff0000000000000ll);
  if (a.fl & 2u) return __longlong_as_double((long long)0xfff0000000000000ull);
  fx_norm(a);
  return fma((double)a.l2, 0x1p-4, fma((double)a.l1, 0x1p-46, (double)a.l0 * 0x1p-88));
}
// global accumulator of 4 words: limbs, flags
__device__ __forceinline__ void fx_red_global(long long* g, const Fx& a) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(g), "l"(a.l0) : "memory");
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(g + 1), "l"(a.l1) : "memory");
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(g + 2), "l"(a.l2) : "memory");
  if (a.fl) asm volatile("red.global.or.b64 [%0], %1;" ::"l"(g + 3), "l"((long long)a.fl) : "memory");
}
__device__ __forceinline__ Fx fx_load_global(const long long* g) {
  Fx a;
  a.l0 = __ldcg(g);
  a.l1 = __ldcg(g + 1);
  a.l2 = __ldcg(g + 2);
  a.fl = (unsigned)__ldcg(g + 3);
  return a;
}

__device__ __forceinline__ void kahan_add(float& s, float& comp, float x) {
  float yv = x - comp;
  float t = s + yv;
  comp = (t - s) - yv;
  s = t;
}

}  // namespace pcdn
