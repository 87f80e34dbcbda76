// C ABI of the GB300 PCDN solver (declared in include/pcdn.h): problem set-up on the device,
// the outer-iteration loop of Algorithm 3 around the bundle walker, and the single-bundle
// entry used for parity checks.  All arithmetic of the method runs in the CUDA kernels of
// pcdn_walk.cu and pcdn_prep.cu; this file validates, allocates, launches and copies.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pcdn.h"
#include "pcdn_internal.cuh"
#include "pcdn_prep.h"
#include "pcdn_task.h"

namespace pcdn {
cudaError_t launch_walk(int loss, int prec, const WalkParams& p, int grid, cudaStream_t s, bool capturing);
cudaError_t walk_max_blocks_per_sm(int loss, int prec, int* out);
cudaError_t walk_configure(int loss, int prec);
cudaError_t launch_walk_rows(int loss, int prec, const WalkParams& p, int grid, cudaStream_t s, bool capturing);
cudaError_t walk_rows_max_blocks_per_sm(int loss, int prec, int* out);
int walk_rows_max_grid();
}  // namespace pcdn

using namespace pcdn;

namespace {

thread_local std::string g_err;

// An NVTX range for the lifetime of a scope (host-side phases in profiler timelines; free without a
// profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

namespace pcdn {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace pcdn

namespace {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (expr);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      if (e_ == cudaErrorMemoryAllocation) return fail(PCDN_ENOMEM, "%s: %s", #expr, cudaGetErrorString(e_)); \
      return fail(PCDN_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                             \
    }                                                                                               \
  } while (0)

// A device-side wait gives up after kDefaultWaitNs of the global timer (or after opts.spin_limit
// polls when the caller sets one).
constexpr uint64_t kDefaultWaitNs = uint64_t(10) * 1000000000ull;

// Device memory comes from one stream-ordered pool per device, owned by the library for the life of
// the process: allocations and frees are ordered on the problem's stream and never synchronise the
// device, so problems can be created and destroyed while other problems' solves run (the request
// server does exactly that).  Freed memory stays reserved for reuse up to kPoolKeep bytes or an
// eighth of the device, whichever is more.
constexpr uint64_t kPoolKeep = uint64_t(8) << 30;

cudaError_t library_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
    // freed memory kept reserved: 8 GiB, or an eighth of the device when that is more, so that a
    // large problem's creation (transient buffers of up to about 40 bytes per nonzero) followed by
    // its destruction and the next creation reuses mapped memory instead of mapping it again
    size_t mem_free = 0, mem_total = 0;
    if ((e = cudaMemGetInfo(&mem_free, &mem_total)) != cudaSuccess) return e;
    uint64_t keep = std::max<uint64_t>(kPoolKeep, (uint64_t)mem_total / 8);
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    // never make one problem's stream wait for another's to reuse memory freed there
    int no = 0;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no)) != cudaSuccess) return e;
    pools[dev] = pool;
  }
  *out = pools[dev];
  return cudaSuccess;
}

template <typename T>
cudaError_t dalloc(T** p, int64_t count, cudaStream_t s) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = library_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync((void**)p, sizeof(T) * (size_t)count, pool, s);
}

void dfree(void* q, cudaStream_t s) {
  if (q) cudaFreeAsync(q, s);
}

}  // namespace

struct pcdn_problem {
  int64_t n = 0, m = 0, nnz = 0;
  double c = 1.0;
  int loss = 0;
  bool owns_x = true;
  int device = 0;
  int sms = 0;
  // X by columns, labels
  int64_t* col_ptr = nullptr;
  int32_t* row_idx = nullptr;
  float* val = nullptr;
  int8_t* y = nullptr;
  int8_t* ylab = nullptr;  // own copy of y, padded to a multiple of 16 bytes (the walker reads aligned words)
  // X by rows
  int64_t* row_ptr = nullptr;
  int32_t* col_idx = nullptr;
  float* rval = nullptr;
  // state
  double* w = nullptr;
  double* w_pos = nullptr;  // w in the walk's position order
  SampleRec* st = nullptr;  // per-sample maintained quantity and coefficients (32-byte records)
  int rec_prec = 0;         // precision of the coefficient pairs in st
  double* delta = nullptr;
  uint32_t* touched = nullptr;
  int64_t nwords = 0;
  // identity-order work items (KKT)
  int32_t* id_perm = nullptr;
  int64_t* id_item_ptr = nullptr;
  Item* id_items = nullptr;
  int64_t n_id_items = 0;
  // per-epoch partition and items
  uint64_t* keys0 = nullptr;
  uint64_t* keys1 = nullptr;
  int32_t* vals0 = nullptr;
  int32_t* vals1 = nullptr;
  int64_t* cnt = nullptr;
  int64_t* item_ptr = nullptr;
  Item* items = nullptr;
  int64_t max_items = 0;
  int64_t* hist = nullptr;
  int64_t* scan_ws = nullptr;
  int64_t* item_len = nullptr;  // [max_items + 1]
  int64_t* item_off = nullptr;  // [max_items + 1]
  int64_t* plan = nullptr;
  int64_t plan_cap = 0;
  // bundle scratch (gk, hk, dk, dkf: two halves of P_cap, by bundle parity)
  int32_t P_cap = 0;
  double* gk = nullptr;
  double* hk = nullptr;
  double* dk = nullptr;
  float* dkf = nullptr;
  uint32_t* col_cnt = nullptr;
  double* part = nullptr;
  // row-sorted layout (allocated by the first walk that uses it)
  int32_t* entry_row = nullptr;  // row of every mirror entry
  int32_t* br_row = nullptr;
  int32_t* br_k = nullptr;
  float* br_val = nullptr;
  int64_t* br_ptr = nullptr;
  int64_t br_ptr_cap = 0;
  int64_t* br_plan = nullptr;
  int64_t br_plan_cap = 0;
  RowsWorkspace rws{};
  double* lspart = nullptr;
  // reductions, barriers, flags
  double* lsacc = nullptr;
  int max_grid = 1;
  uint32_t* sync = nullptr;  // [0] bar_count [1] bar_gen [2..3] barrier-1 flag counts [4..5] barrier-1 counter (64-bit)
  int* err = nullptr;
  unsigned long long* counters = nullptr;
  double* red_part = nullptr;  // block partials
  double* red_out = nullptr;   // [4]
  int red_grid = 0;
  // trace buffers (per epoch)
  int64_t tr_cap = 0;
  int32_t* tr_q = nullptr;
  double* tr_alpha = nullptr;
  double* tr_Delta = nullptr;
  double* tr_dF = nullptr;
  // outer-iteration index on the device (read by a captured outer iteration's partition)
  int64_t* epoch_dev = nullptr;
  // shrinking: g_j of every feature at the last stopping test, and [0] max |v_j| (bits of the
  // double), [1] active features, [2] their nonzeros (allocated by the first solve that shrinks)
  double* gfull = nullptr;
  unsigned long long* shr = nullptr;
  // penalty l1 ||w||_1 + (l2/2) ||w||^2 (Eq. 1: l1 = 1, l2 = 0; pcdn_set_penalty)
  double l1 = 1.0, l2 = 0.0;
  bool capturing = false;  // the stream is being captured into a graph
  // stream, events
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int64_t launches = 0;
  int64_t device_bytes = 0;
};

namespace {

template <typename T>
cudaError_t palloc(pcdn_problem* p, T** ptr, int64_t count) {
  cudaError_t e = dalloc(ptr, count, p->stream);
  if (e == cudaSuccess) p->device_bytes += (int64_t)sizeof(T) * (count > 0 ? count : 1);
  return e;
}

void free_all(pcdn_problem* p) {
  auto f = [p](void* q) { dfree(q, p->stream); };
  if (p->owns_x) {
    f(p->col_ptr); f(p->row_idx); f(p->val); f(p->y);
  }
  f(p->row_ptr); f(p->col_idx); f(p->rval); f(p->ylab);
  f(p->w); f(p->w_pos); f(p->st); f(p->delta); f(p->touched);
  f(p->item_len); f(p->item_off); f(p->plan);
  f(p->id_perm); f(p->id_item_ptr); f(p->id_items);
  f(p->keys0); f(p->keys1); f(p->vals0); f(p->vals1); f(p->cnt); f(p->item_ptr); f(p->items);
  f(p->hist); f(p->scan_ws);
  f(p->gk); f(p->hk); f(p->dk); f(p->dkf); f(p->col_cnt); f(p->part);
  f(p->entry_row); f(p->br_row); f(p->br_k); f(p->br_val); f(p->br_ptr); f(p->br_plan);
  f(p->rws.inv); f(p->rws.hist); f(p->rws.scan_ws); f(p->rws.k0); f(p->rws.k1); f(p->rws.v0); f(p->rws.v1);
  f(p->rws.rhist); f(p->lspart);
  f(p->lsacc); f(p->sync); f(p->err); f(p->counters); f(p->red_part); f(p->red_out);
  f(p->tr_q); f(p->tr_alpha); f(p->tr_Delta); f(p->tr_dF); f(p->epoch_dev);
  f(p->gfull); f(p->shr);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
}

// Columns [j0, j1) of a host CSC: rows in range and strictly ascending, values finite.  Returns the
// first failing column (or j1) and its message.
int64_t check_columns(const pcdn_csc* X, int64_t j0, int64_t j1, std::string* msg) {
  char buf[256];
  for (int64_t j = j0; j < j1; ++j) {
    const int64_t a = X->col_ptr[j], b = X->col_ptr[j + 1];
    if (b < a || a < 0 || b > X->nnz) {
      snprintf(buf, sizeof buf, "col_ptr decreases or leaves [0, nnz] at column %lld", (long long)j);
      *msg = buf;
      return j;
    }
    for (int64_t e = a; e < b; ++e) {
      const int32_t r = X->row_idx[e];
      if (r < 0 || r >= X->n_samples) {
        snprintf(buf, sizeof buf, "row index %d out of range in column %lld", r, (long long)j);
        *msg = buf;
        return j;
      }
      if (e > a && r <= X->row_idx[e - 1]) {
        snprintf(buf, sizeof buf, "rows not strictly ascending in column %lld", (long long)j);
        *msg = buf;
        return j;
      }
      if (!std::isfinite(X->val[e])) {
        snprintf(buf, sizeof buf, "non-finite value in column %lld", (long long)j);
        *msg = buf;
        return j;
      }
    }
  }
  return j1;
}

// Sizes and pointers of a host CSC (before any entry is read).
int check_host_shape(const pcdn_csc* X, const int8_t* y) {
  if (!X || !y) return fail(PCDN_EINVAL, "X and y must be given");
  if (X->n_samples <= 0 || X->n_features <= 0 || X->nnz < 0)
    return fail(PCDN_EINVAL, "n_samples and n_features must be positive, nnz >= 0");
  if (X->n_samples > INT32_MAX || X->n_features > INT32_MAX)
    return fail(PCDN_EINVAL, "n_samples and n_features must fit int32");
  if (X->nnz >= INT32_MAX) return fail(PCDN_EINVAL, "nnz must be below 2^31");
  if (!X->col_ptr || (X->nnz > 0 && (!X->row_idx || !X->val))) return fail(PCDN_EINVAL, "CSC arrays missing");
  if (X->col_ptr[0] != 0 || X->col_ptr[X->n_features] != X->nnz)
    return fail(PCDN_EINVAL, "col_ptr must start at 0 and end at nnz");
  return PCDN_OK;
}

// Every entry of a host CSC (shape checked) and every label.
int check_host_entries(const pcdn_csc* X, const int8_t* y) {
  // the columns in contiguous ranges of about equal nonzero count, one host thread each; the first
  // failing column over all ranges decides the message
  const int64_t m = X->n_features;
  int threads = (int)std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 16);
  if (X->nnz < (int64_t(1) << 20)) threads = 1;
  std::vector<int64_t> cut(threads + 1, m);
  cut[0] = 0;
  for (int t = 1; t < threads; ++t) {
    // first column whose start passes t/threads of the nonzeros (col_ptr may be malformed: clamp)
    const int64_t target = X->nnz / threads * t;
    int64_t lo = cut[t - 1], hi = m;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (X->col_ptr[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    cut[t] = std::max(lo, cut[t - 1]);
  }
  std::vector<int64_t> bad(threads, m);
  std::vector<std::string> msgs(threads);
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t)
    pool.emplace_back([&, t]() { bad[t] = check_columns(X, cut[t], cut[t + 1], &msgs[t]); if (bad[t] == cut[t + 1]) bad[t] = m; });
  bad[0] = check_columns(X, cut[0], cut[1], &msgs[0]);
  if (bad[0] == cut[1]) bad[0] = m;
  for (auto& th : pool) th.join();
  for (int t = 0; t < threads; ++t)
    if (bad[t] < m) return fail(PCDN_EINVAL, "%s", msgs[t].c_str());
  for (int64_t i = 0; i < X->n_samples; ++i)
    if (y[i] != 1 && y[i] != -1) return fail(PCDN_EINVAL, "label %d of sample %lld is not +1 or -1", (int)y[i], (long long)i);
  return PCDN_OK;
}

// Everything after X and y are on the device: mirror, state, workspaces.
int finish_create(pcdn_problem* p) {
  cudaStream_t s = p->stream;
  const int64_t n = p->n, m = p->m, nnz = p->nnz;
  CUDA_TRY(cudaGetDevice(&p->device));
  CUDA_TRY(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device));
  {
    const int64_t npad = (n + 15) / 16 * 16;
    CUDA_TRY(palloc(p, &p->ylab, npad));
    CUDA_TRY(cudaMemsetAsync(p->ylab, 0, npad, s));
    CUDA_TRY(cudaMemcpyAsync(p->ylab, p->y, n, cudaMemcpyDeviceToDevice, s));
  }

  // ---- row-major mirror: the CSC entries in row order, columns ascending within each row (the order
  // of the FP64 refresh's sums): row pointers from the row counts, entries by a stable counting sort
  // on the row index.  Every write stays inside the arrays whatever the entries hold, so this may
  // run while the host still checks them.
  CUDA_TRY(palloc(p, &p->row_ptr, n + 1));
  CUDA_TRY(palloc(p, &p->col_idx, nnz));
  CUDA_TRY(palloc(p, &p->rval, nnz));
  {
    const MirrorSizes z = mirror_sizes(n, nnz);
    MirrorWorkspace mw{};
    int64_t *counts = nullptr, *ws = nullptr;
    int32_t* ecol = nullptr;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
      dfree(counts, s); dfree(ws, s); dfree(ecol, s); dfree(mw.hist, s); dfree(mw.off, s); dfree(mw.scan_ws, s);
      dfree(mw.row0, s); dfree(mw.trow, s); dfree(mw.tcol, s); dfree(mw.tval, s);
    };
    if ((e = dalloc(&counts, n + 1, s)) || (e = dalloc(&ws, scan_workspace_elems(n + 1), s)) ||
        (e = dalloc(&ecol, std::max<int64_t>(nnz, 1), s)) || (e = dalloc(&mw.hist, z.hist, s)) ||
        (e = dalloc(&mw.off, z.hist, s)) || (e = dalloc(&mw.scan_ws, scan_workspace_elems(z.hist), s))) {
      cleanup();
      return fail(e == cudaErrorMemoryAllocation ? PCDN_ENOMEM : PCDN_ECUDA, "mirror workspace: %s", cudaGetErrorString(e));
    }
    if ((z.tmp_row && (e = dalloc(&mw.row0, nnz, s))) ||
        (z.tmp_triple && ((e = dalloc(&mw.trow, nnz, s)) || (e = dalloc(&mw.tcol, nnz, s)) ||
                          (e = dalloc(&mw.tval, nnz, s))))) {
      cleanup();
      return fail(e == cudaErrorMemoryAllocation ? PCDN_ENOMEM : PCDN_ECUDA, "mirror workspace: %s",
                  cudaGetErrorString(e));
    }
    if ((e = mirror_configure()) || (e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * (n + 1), s)) ||
        (e = mirror_row_counts(p->row_idx, nnz, n, counts, s, &p->launches)) ||
        (e = scan_exclusive(counts, p->row_ptr, n + 1, ws, s, &p->launches)) ||
        (nnz > 0 && (e = entry_columns(p->col_ptr, m, nnz, ecol, s, &p->launches))) ||
        (e = build_mirror(p->row_idx, ecol, p->val, nnz, n, mw, p->col_idx, p->rval, s, &p->launches))) {
      cleanup();
      return fail(PCDN_ECUDA, "mirror build: %s", cudaGetErrorString(e));
    }
    cleanup();
  }

  // ---- state
  p->nwords = (n + 31) / 32;
  CUDA_TRY(palloc(p, &p->w, m));
  CUDA_TRY(palloc(p, &p->w_pos, m));
  CUDA_TRY(palloc(p, &p->st, n));
  CUDA_TRY(palloc(p, &p->delta, n));
  CUDA_TRY(palloc(p, &p->touched, p->nwords));
  CUDA_TRY(cudaMemsetAsync(p->w, 0, sizeof(double) * m, s));
  CUDA_TRY(cudaMemsetAsync(p->delta, 0, sizeof(double) * n, s));
  CUDA_TRY(cudaMemsetAsync(p->touched, 0, sizeof(uint32_t) * p->nwords, s));

  // ---- workspaces
  p->max_items = m + nnz / kChunk + 2;
  const int64_t hm = radix_hist_elems(m);
  CUDA_TRY(palloc(p, &p->keys0, m));
  CUDA_TRY(palloc(p, &p->keys1, m));
  CUDA_TRY(palloc(p, &p->vals0, m));
  CUDA_TRY(palloc(p, &p->vals1, m));
  CUDA_TRY(palloc(p, &p->cnt, m + 1));
  CUDA_TRY(palloc(p, &p->item_ptr, m + 1));
  CUDA_TRY(palloc(p, &p->items, p->max_items));
  CUDA_TRY(palloc(p, &p->hist, hm));
  {
    int64_t scan_n = hm > m + 1 ? hm : m + 1;
    if (p->max_items + 1 > scan_n) scan_n = p->max_items + 1;
    CUDA_TRY(palloc(p, &p->scan_ws, scan_workspace_elems(scan_n)));
  }
  CUDA_TRY(palloc(p, &p->part, 2 * p->max_items));
  CUDA_TRY(palloc(p, &p->item_len, p->max_items + 1));
  CUDA_TRY(palloc(p, &p->item_off, p->max_items + 1));
  CUDA_TRY(palloc(p, &p->id_perm, m));
  CUDA_TRY(palloc(p, &p->id_item_ptr, m + 1));
  CUDA_TRY(palloc(p, &p->id_items, p->max_items));
  CUDA_TRY(cudaError_t(iota_i32(p->id_perm, m, s, &p->launches)));

  int bps = 2;
  for (int prec = 0; prec < 2; ++prec) {
    int b = 1;
    CUDA_TRY(walk_max_blocks_per_sm(p->loss, prec, &b));
    bps = std::min(bps, b);
    CUDA_TRY(walk_rows_max_blocks_per_sm(p->loss, prec, &b));
    bps = std::min(bps, b);
  }
  if (bps < 1) return fail(PCDN_ECUDA, "bundle walker cannot be resident on this device");
  p->max_grid = std::min(p->sms * bps, walk_rows_max_grid());
  CUDA_TRY(palloc(p, &p->lsacc, 3 * kPartStride * kAccPad));
  CUDA_TRY(palloc(p, &p->sync, 8));
  CUDA_TRY(palloc(p, &p->err, 4));
  CUDA_TRY(palloc(p, &p->counters, 8));
  CUDA_TRY(palloc(p, &p->epoch_dev, 1));
  // blocks of the refresh, KKT and objective reductions: 4 per SM, fewer for a small problem (about
  // 256 rows or work items per block), so that many small problems on one GPU do not flood it with
  // empty blocks
  {
    const int64_t work = std::max<int64_t>(n, m + nnz / kChunk);
    p->red_grid = (int)std::max<int64_t>(1, std::min<int64_t>(p->sms * 4, (work + 255) / 256));
  }
  CUDA_TRY(palloc(p, &p->red_part, 2 * (int64_t)p->red_grid));
  CUDA_TRY(palloc(p, &p->red_out, 4));
  CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int) * 4, s));
  CUDA_TRY(cudaEventCreate(&p->ev0));
  CUDA_TRY(cudaEventCreate(&p->ev1));
  CUDA_TRY(cudaStreamSynchronize(s));
  return PCDN_OK;
}

// The work items of the identity order (the KKT and objective passes over the columns), and the
// state at w = 0.  The items follow col_ptr: only for checked input.
int finish_create_checked(pcdn_problem* p) {
  cudaStream_t s = p->stream;
  CUDA_TRY(build_items(p->id_perm, p->m, p->col_ptr, nullptr, p->cnt, p->id_item_ptr, p->id_items, p->scan_ws, s,
                       &p->launches));
  CUDA_TRY(cudaMemcpyAsync(&p->n_id_items, p->id_item_ptr + p->m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  // w = 0: z = 0 for every sample, set directly (what a refresh from z = Xw gives there, bit for bit)
  CUDA_TRY(state_at_zero(p->loss, 0, p->y, p->n, p->st, s, &p->launches));
  p->rec_prec = 0;
  CUDA_TRY(cudaStreamSynchronize(s));
  return PCDN_OK;
}

int ensure_bundle_scratch(pcdn_problem* p, int32_t P) {
  if (P <= p->P_cap) return PCDN_OK;
  auto f = [p](void* q) { dfree(q, p->stream); };
  f(p->gk); f(p->hk); f(p->dk); f(p->dkf); f(p->col_cnt);
  p->gk = p->hk = p->dk = nullptr;
  p->dkf = nullptr;
  p->col_cnt = nullptr;
  p->P_cap = 0;
  CUDA_TRY(palloc(p, &p->gk, 2 * (int64_t)P));
  CUDA_TRY(palloc(p, &p->hk, 2 * (int64_t)P));
  CUDA_TRY(palloc(p, &p->dk, 2 * (int64_t)P));
  CUDA_TRY(palloc(p, &p->dkf, 2 * (int64_t)P));
  CUDA_TRY(palloc(p, &p->col_cnt, 2 * P));
  CUDA_TRY(cudaMemsetAsync(p->col_cnt, 0, sizeof(uint32_t) * 2 * P, p->stream));
  p->P_cap = P;
  return PCDN_OK;
}

int ensure_plan(pcdn_problem* p, int64_t entries) {
  if (entries <= p->plan_cap) return PCDN_OK;
  dfree(p->plan, p->stream);
  p->plan = nullptr;
  p->plan_cap = 0;
  CUDA_TRY(palloc(p, &p->plan, entries));
  p->plan_cap = entries;
  return PCDN_OK;
}

// The row-sorted walker's exact sums take fewer than 2^24 terms each (one per sample and per
// position at most): larger problems take the scatter layout.
constexpr int64_t kRowsMaxTerms = 1ll << 24;

// The row-sorted layout's arrays for a walk of nb bundles on G blocks (allocated once, the bundle
// pointers and block plan grown as needed; the radix-sort workspace only for more than kBins bundles).
int ensure_rows(pcdn_problem* p, int64_t nb, int G) {
  const int64_t nnz = p->nnz;
  if (p->n + p->m >= kRowsMaxTerms)
    return fail(PCDN_EINVAL, "the row-sorted layout needs n_samples + n_features below 2^24 (its exact sums take "
                             "fewer than 2^24 terms); use the scatter layout");
  if (!p->entry_row) {
    CUDA_TRY(rows_configure());
    CUDA_TRY(palloc(p, &p->entry_row, nnz));
    CUDA_TRY(palloc(p, &p->br_row, nnz));
    CUDA_TRY(palloc(p, &p->br_k, nnz));
    CUDA_TRY(palloc(p, &p->br_val, nnz));
    CUDA_TRY(palloc(p, &p->rws.inv, p->m));
    CUDA_TRY(palloc(p, &p->rws.hist, rows_hist_elems(nnz)));
    CUDA_TRY(palloc(p, &p->rws.scan_ws, scan_workspace_elems(std::max(rows_hist_elems(nnz), radix_hist_elems(nnz)))));
    CUDA_TRY(palloc(p, &p->lspart, 2 * (int64_t)kPartStride * p->max_grid));
    if (nnz > 0) CUDA_TRY(entry_rows(p->row_ptr, p->n, p->entry_row, p->stream, &p->launches));
  }
  if (nb > kBins && !p->rws.k0) {
    CUDA_TRY(palloc(p, &p->rws.k0, nnz));
    CUDA_TRY(palloc(p, &p->rws.k1, nnz));
    CUDA_TRY(palloc(p, &p->rws.v0, nnz));
    CUDA_TRY(palloc(p, &p->rws.v1, nnz));
    CUDA_TRY(palloc(p, &p->rws.rhist, radix_hist_elems(nnz)));
  }
  if (nb + 1 > p->br_ptr_cap) {
    dfree(p->br_ptr, p->stream);
    p->br_ptr = nullptr;
    p->br_ptr_cap = 0;
    CUDA_TRY(palloc(p, &p->br_ptr, nb + 1));
    p->br_ptr_cap = nb + 1;
  }
  const int64_t pe = nb * (int64_t)(G + 1);
  if (pe > p->br_plan_cap) {
    dfree(p->br_plan, p->stream);
    p->br_plan = nullptr;
    p->br_plan_cap = 0;
    CUDA_TRY(palloc(p, &p->br_plan, pe));
    p->br_plan_cap = pe;
  }
  return PCDN_OK;
}

// The walker layout of a walk on `grid` blocks (reading of PCDN_LAYOUT_AUTO): the row-sorted
// layout for FP64 solves on several blocks (repeatable bit for bit, and its solve measured within a
// few percent of the scatter layout's on the 2M x 3M workload), the scatter layout otherwise (mixed
// precision: the per-outer-iteration regrouping costs more than its walker saves).
int walk_layout(const pcdn_problem* p, const pcdn_opts* o, int grid) {
  if (o->layout == PCDN_LAYOUT_SCATTER || o->layout == PCDN_LAYOUT_ROWS) return o->layout;
  return (grid > 1 && o->prec == PCDN_PREC_FP64 && p->n + p->m < kRowsMaxTerms) ? PCDN_LAYOUT_ROWS
                                                                                : PCDN_LAYOUT_SCATTER;
}

int ensure_trace(pcdn_problem* p, int64_t nb) {
  if (nb <= p->tr_cap) return PCDN_OK;
  auto f = [p](void* q) { dfree(q, p->stream); };
  f(p->tr_q); f(p->tr_alpha); f(p->tr_Delta); f(p->tr_dF);
  p->tr_q = nullptr;
  p->tr_alpha = p->tr_Delta = p->tr_dF = nullptr;
  p->tr_cap = 0;
  CUDA_TRY(palloc(p, &p->tr_q, nb));
  CUDA_TRY(palloc(p, &p->tr_alpha, nb));
  CUDA_TRY(palloc(p, &p->tr_Delta, nb));
  CUDA_TRY(palloc(p, &p->tr_dF, nb));
  p->tr_cap = nb;
  return PCDN_OK;
}

int ensure_shrink(pcdn_problem* p) {
  if (p->gfull) return PCDN_OK;
  CUDA_TRY(palloc(p, &p->shr, 4));
  CUDA_TRY(palloc(p, &p->gfull, p->m));
  return PCDN_OK;
}

int status_from_flags(int h);

int device_status(pcdn_problem* p) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  return status_from_flags(h);
}

// The device error flags as a status code (and message).
int status_from_flags(int h) {
  if (h & kErrTimeout) return fail(PCDN_ETIMEOUT, "a device-side wait between thread blocks timed out");
  if (h & kErrNumeric) return fail(PCDN_ENUMERIC, "non-finite gradient, Hessian diagonal or direction");
  if (h & kErrRange)
    return fail(PCDN_ENUMERIC, "maintained quantity out of range (FP64 keeps e^{w^T x}, which holds |w^T x| up "
                               "to about 699; mixed precision keeps w^T x itself and has no such limit)");
  if (h & kErrRefresh)
    return fail(PCDN_ENUMERIC, "w^T x out of range when recomputing from z = Xw (FP64: |w^T x| > 700; "
                               "mixed: not finite)");
  return PCDN_OK;
}

// Per-bundle scratch back to its resting state (zero delta, empty bitmap, zero arrival counts):
// every entry point that starts stepping calls this, so a launch that ended early (a timeout)
// leaves nothing behind.
int reset_scratch(pcdn_problem* p) {
  CUDA_TRY(cudaMemsetAsync(p->delta, 0, sizeof(double) * p->n, p->stream));
  CUDA_TRY(cudaMemsetAsync(p->touched, 0, sizeof(uint32_t) * p->nwords, p->stream));
  if (p->P_cap > 0) CUDA_TRY(cudaMemsetAsync(p->col_cnt, 0, sizeof(uint32_t) * 2 * p->P_cap, p->stream));
  return PCDN_OK;
}

int do_refresh(pcdn_problem* p, int prec, bool write_state, bool with_loss) {
  // w_pos (position-order w, used only inside a walk) holds the mixed mode's split copy of w
  CUDA_TRY(refresh(p->loss, prec, p->row_ptr, p->col_idx, p->rval, p->y, p->w, p->n, p->m, p->nnz, p->w_pos, p->st,
                   write_state, with_loss ? p->red_part : nullptr, p->red_grid, p->err, p->stream, &p->launches));
  if (write_state) p->rec_prec = prec;
  return PCDN_OK;
}

// ||v||_1 into red_out[slot] (device); the caller copies.
// The maintained quantities at a solve's start point: a cold start (w = 0) has z = 0, so they are
// set directly (the values a refresh from z = Xw gives there, bit for bit) without the pass over X.
int start_state(pcdn_problem* p, int prec, bool cold) {
  if (!cold) return do_refresh(p, prec, true, false);
  CUDA_TRY(state_at_zero(p->loss, prec, p->y, p->n, p->st, p->stream, &p->launches));
  p->rec_prec = prec;
  return PCDN_OK;
}

// ||v||_1 into red_out[slot]; with shrink also g_j of every feature, max |v_j| and the count and
// nonzeros of the features active in the next outer iteration (p->shr).
int do_kkt(pcdn_problem* p, int slot, bool shrink = false) {
  if (shrink) CUDA_TRY(cudaMemsetAsync(p->shr, 0, sizeof(unsigned long long) * 3, p->stream));
  CUDA_TRY(kkt_l1(p->loss, p->rec_prec, p->y, p->n, p->id_items, p->n_id_items, p->id_item_ptr, p->id_perm, p->m,
                  p->row_idx, p->val, p->st,
                  p->w, p->c, p->l1, p->l2, p->part, p->red_part, p->red_grid, p->red_out + slot, p->stream,
                  &p->launches, shrink ? p->gfull : nullptr, shrink ? p->shr : nullptr));
  if (shrink)
    CUDA_TRY(active_count(p->gfull, p->w, p->m, p->col_ptr, p->shr, p->n, p->l1, p->shr + 1, p->stream,
                          &p->launches));
  return PCDN_OK;
}

// The partition perm of all features restricted to the active set of the last stopping test (in
// partition order), into the other radix-sort value buffer.
int shrink_partition(pcdn_problem* p, int32_t* perm, int32_t** out) {
  int32_t* dst = perm == p->vals0 ? p->vals1 : p->vals0;
  CUDA_TRY(compact_active(perm, p->m, p->gfull, p->w, p->shr, p->n, p->l1, p->cnt, p->item_off, p->scan_ws, dst,
                          p->stream, &p->launches));
  *out = dst;
  return PCDN_OK;
}

int do_objective(pcdn_problem* p, int slot) {
  int rc = do_refresh(p, p->rec_prec, false, true);
  if (rc) return rc;
  CUDA_TRY(objective_finish(p->red_part, p->red_grid, p->w, p->m, p->c, p->l1, p->l2, p->red_part + p->red_grid,
                            p->red_grid, p->red_out + slot, p->stream, &p->launches));
  return PCDN_OK;
}

int read_double(pcdn_problem* p, int slot, double* out) {
  CUDA_TRY(cudaMemcpyAsync(out, p->red_out + slot, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  return PCDN_OK;
}

int check_opts(const pcdn_opts* o) {
  if (!(o->sigma > 0 && o->sigma < 1)) return fail(PCDN_EINVAL, "sigma must be in (0, 1)");
  if (!(o->beta > 0 && o->beta < 1)) return fail(PCDN_EINVAL, "beta must be in (0, 1)");
  if (!(o->gamma >= 0 && o->gamma < 1)) return fail(PCDN_EINVAL, "gamma must be in [0, 1)");
  if (!(o->nu > 0)) return fail(PCDN_EINVAL, "nu must be positive");
  if (o->q_max < 1 || o->q_max > 1000) return fail(PCDN_EINVAL, "q_max must be in [1, 1000]");
  if (o->ls_batch < 0 || o->ls_batch > kMaxK) return fail(PCDN_EINVAL, "ls_batch must be in [0, %d]", kMaxK);
  if (o->max_epochs < 0) return fail(PCDN_EINVAL, "max_epochs must be >= 0");
  if (o->prec != PCDN_PREC_FP64 && o->prec != PCDN_PREC_MIXED) return fail(PCDN_EINVAL, "unknown precision");
  if (o->epoch0 < 0) return fail(PCDN_EINVAL, "epoch0 must be >= 0");
  if (!(o->kkt_ref >= 0) || !std::isfinite(o->kkt_ref)) return fail(PCDN_EINVAL, "kkt_ref must be >= 0 and finite");
  if (o->shrink != 0 && o->shrink != 1) return fail(PCDN_EINVAL, "shrink must be 0 or 1");
  if (o->layout < PCDN_LAYOUT_AUTO || o->layout > PCDN_LAYOUT_ROWS) return fail(PCDN_EINVAL, "unknown layout");
  return PCDN_OK;
}

int pick_grid(const pcdn_problem* p, const pcdn_opts* o, int32_t P) {
  int g;
  if (o->grid_ctas > 0) {
    g = o->grid_ctas < p->max_grid ? o->grid_ctas : p->max_grid;
  } else {
    // One block when a bundle's work fits one SM comfortably; the whole GPU otherwise.
    const double nnz_per_bundle = (double)p->nnz * (double)P / (double)p->m;
    g = (nnz_per_bundle < 8192.0 && p->n < (1 << 16)) ? 1 : p->max_grid;
  }
  // the block plan holds (bundles) x (blocks + 1) entries; keep it under 2^26
  const int64_t nb = (p->m + P - 1) / P;
  const int64_t cap = (int64_t(1) << 26) / (nb > 0 ? nb : 1) - 1;
  if (cap < g) g = cap < 1 ? 1 : (int)cap;
  return g;
}

// An event record on the problem's stream; inside a capture it becomes a record node of the graph.
cudaError_t record(cudaEvent_t ev, pcdn_problem* p) {
  return cudaEventRecordWithFlags(ev, p->stream, p->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Launch the walker over bundles [t0, t1) of the partition held in perm/items.
int run_walk(pcdn_problem* p, const pcdn_opts* o, const int32_t* perm, int64_t npos, int32_t P, int64_t t0, int64_t t1,
             int grid, float* ms) {
  WalkParams w{};
  w.n = p->n;
  w.m = p->m;
  w.nnz = p->nnz;
  w.col_ptr = p->col_ptr;
  w.row_idx = p->row_idx;
  w.val = p->val;
  w.y = p->ylab;
  w.c = p->c;
  w.w_pos = p->w_pos;
  w.st = p->st;
  w.delta = p->delta;
  w.touched = p->touched;
  w.nwords = p->nwords;
  w.perm = perm;
  w.items = p->items;
  w.item_ptr = p->item_ptr;
  w.plan = p->plan;
  w.npos = npos;
  w.P = P;
  w.t_begin = t0;
  w.t_end = t1;
  w.gk = p->gk;
  w.hk = p->hk;
  w.dk = p->dk;
  w.part = p->part;
  w.col_cnt = p->col_cnt;
  w.anynz = nullptr;
  w.bar1 = reinterpret_cast<unsigned long long*>(p->sync + 4);
  w.nzc = p->sync + 2;
  w.lsacc = p->lsacc;
  w.bar_count = p->sync;
  w.bar_gen = p->sync + 1;
  w.spin_limit = o->spin_limit ? o->spin_limit : 0xffffffffu;
  w.wait_ns = kDefaultWaitNs;
  w.sigma = o->sigma;
  w.beta = o->beta;
  w.gamma = o->gamma;
  w.nu = o->nu;
  w.c_f = (float)p->c;
  w.nu_f = (float)o->nu;
  w.l1 = p->l1;
  w.l2 = p->l2;
  w.l1_f = (float)p->l1;
  w.l2_f = (float)p->l2;
  w.q_max = o->q_max;
  // step sizes per pass: almost every bundle accepts q = 0, so the first pass tests that alone;
  // a further pass (one more barrier) tests four
  w.K1 = o->ls_batch > 0 ? o->ls_batch : 1;
  w.K = o->ls_batch > 0 ? o->ls_batch : 4;
  w.tr_q = p->tr_q;
  w.tr_alpha = p->tr_alpha;
  w.tr_Delta = p->tr_Delta;
  w.tr_dF = p->tr_dF;
  w.counters = p->counters;
  w.err = p->err;
  const int64_t nb = (npos + P - 1) / P;
  int rc = ensure_plan(p, nb * (grid + 1));
  if (rc) return rc;
  w.plan = p->plan;
  w.P_cap = p->P_cap;
  w.dkf = p->dkf;
  w.x_vec = ((uintptr_t)p->row_idx % 16 == 0 && (uintptr_t)p->val % 16 == 0) ? 1 : 0;
  const int layout = walk_layout(p, o, grid);
  CUDA_TRY(build_plan(p->items, p->max_items, p->item_ptr, npos, P, nb, grid, p->item_len, p->item_off, p->plan,
                      p->scan_ws, p->stream, &p->launches));
  if (layout == PCDN_LAYOUT_ROWS) {
    rc = ensure_rows(p, nb, grid);
    if (rc) return rc;
    CUDA_TRY(build_rows(perm, npos, p->m, P, nb, grid, p->col_idx, p->rval, p->entry_row, p->nnz, p->rws, p->br_row,
                        p->br_k, p->br_val, p->br_ptr, p->br_plan, p->stream, &p->launches));
    w.br_row = p->br_row;
    w.br_k = p->br_k;
    w.br_val = p->br_val;
    w.br_ptr = p->br_ptr;
    w.br_plan = p->br_plan;
    w.br_vec = 1;
    w.lspart = p->lspart;
  }
  CUDA_TRY(gather_w(p->w, perm, npos, p->w_pos, p->stream, &p->launches));
  CUDA_TRY(cudaMemsetAsync(p->sync, 0, sizeof(uint32_t) * 8, p->stream));
  CUDA_TRY(cudaMemsetAsync(p->lsacc, 0, sizeof(double) * 3 * kPartStride * kAccPad, p->stream));
  // split-column partial slots start all ones (unpublished) for the scatter walker's polled combine
  if (layout != PCDN_LAYOUT_ROWS) CUDA_TRY(cudaMemsetAsync(p->part, 0xFF, sizeof(double) * 2 * p->max_items, p->stream));
  CUDA_TRY(record(p->ev0, p));
  if (layout == PCDN_LAYOUT_ROWS) CUDA_TRY(launch_walk_rows(p->loss, (int)o->prec, w, grid, p->stream, p->capturing));
  else CUDA_TRY(launch_walk(p->loss, (int)o->prec, w, grid, p->stream, p->capturing));
  ++p->launches;
  CUDA_TRY(record(p->ev1, p));
  CUDA_TRY(scatter_w(p->w_pos, perm, npos, p->w, p->stream, &p->launches));
  if (ms) {
    CUDA_TRY(cudaEventSynchronize(p->ev1));
    CUDA_TRY(cudaEventElapsedTime(ms, p->ev0, p->ev1));
  }
  return PCDN_OK;
}

// The partition of outer iteration `epoch` into p->vals? -> returns the device pointer of perm.
int make_partition(pcdn_problem* p, uint64_t seed, int64_t epoch, int32_t** perm_out, const int64_t* epoch_dev = nullptr) {
  CUDA_TRY(perm_keys(seed, epoch, epoch_dev, p->m, p->keys0, p->vals0, p->stream, &p->launches));
  uint64_t* ko = nullptr;
  int32_t* vo = nullptr;
  CUDA_TRY(radix_sort_u64(p->keys0, p->vals0, p->keys1, p->vals1, p->m, 64, p->hist, p->scan_ws, &ko, &vo, p->stream,
                          &p->launches));
  *perm_out = vo;
  return PCDN_OK;
}

}  // namespace

// ---------------------------------------------------------------- non-blocking solve (pcdn_task.h)
namespace pcdn {

namespace {
// Scalars a stage leaves for the host (pinned, written by the stage's device-to-host copies).
struct Mail {
  double kkt;
  double F;
  int32_t err;
  int32_t pad;
  unsigned long long cnt[8];
  unsigned long long act[2];  // shrinking: features and nonzeros active in the next outer iteration
};
enum { kStageNone = 0, kStageStart = 1, kStageEpoch = 2, kStageFinal = 3, kStageEnded = 4 };
}  // namespace

struct SolveTask {
  Mail* mail = nullptr;
  cudaEvent_t ev = nullptr;
  pcdn_problem* p = nullptr;
  pcdn_opts o{};
  int32_t P = 0;
  double eps = 0.0;
  uint64_t seed = 0;
  int grid = 1;
  int64_t nb = 0;
  int stage = kStageNone;
  int rc = PCDN_OK;
  double kkt0 = 0.0, kref = 0.0, kkt_rel = 0.0, F = 0.0;
  int64_t epochs = 0;
  int converged = 0;
  double walk_ms = 0.0;
  int64_t launches0 = 0;
  // shrinking: features and nonzeros of the next outer iteration, nonzeros visited so far
  int64_t npos = 0, nnz_next = 0, nnz_visited = 0;
  bool shrunk = false;
  unsigned long long cnt[8] = {0};
  std::chrono::steady_clock::time_point t0;
  double wall_s = 0.0;
  // walker blocks: a shared budget for multi-block walkers, the blocks wanted, the blocks this
  // solve holds (taken at its start, returned at its end)
  BlockBudget* budget = nullptr;
  int want = 1;
  int held = 0;
  // an outer iteration captured as a CUDA graph at the solve's first outer iteration and replayed
  // for the others (one launch instead of ~45); the partition reads the iteration index from the
  // device, which the graph advances
  bool graphs = true;
  bool graph_tried = false;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  bool used_graph = false;
};

void task_set_blocks(SolveTask* t, BlockBudget* budget, int want) {
  if (!t) return;
  t->budget = budget;
  t->want = want < 1 ? 1 : want;
}

void task_set_graphs(SolveTask* t, bool on) {
  if (t) t->graphs = on;
}

bool task_used_graph(SolveTask* t) { return t && t->graph_kernels > 0 && t->graph_tried && t->used_graph; }

int walker_blocks_wanted(pcdn_problem* p, int32_t P) {
  if (!p || P < 1 || p->m < 1) return 1;
  const double nnz_b = (double)p->nnz * (double)P / (double)p->m;
  const double b = std::ceil(nnz_b / (double)kBlockNnz);
  return (int)std::max(1.0, std::min((double)std::min(kMaxBlocks, p->max_grid), b));
}

int device_walker_capacity(int* out) {
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int bps = 2;
  for (int loss = 0; loss < 2; ++loss)
    for (int prec = 0; prec < 2; ++prec) {
      int b = 1;
      CUDA_TRY(walk_max_blocks_per_sm(loss, prec, &b));
      bps = std::min(bps, b);
      CUDA_TRY(walk_rows_max_blocks_per_sm(loss, prec, &b));
      bps = std::min(bps, b);
    }
  if (bps < 1) return fail(PCDN_ECUDA, "bundle walker cannot be resident on this device");
  *out = std::min(sms * bps, walk_rows_max_grid());
  return PCDN_OK;
}

int task_create(SolveTask** out) {
  if (!out) return fail(PCDN_EINVAL, "out must be given");
  *out = nullptr;
  SolveTask* t = new (std::nothrow) SolveTask();
  if (!t) return fail(PCDN_ENOMEM, "host allocation");
  cudaError_t e = cudaHostAlloc((void**)&t->mail, sizeof(Mail), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    task_destroy(t);
    return fail(e == cudaErrorMemoryAllocation ? PCDN_ENOMEM : PCDN_ECUDA, "task set-up: %s", cudaGetErrorString(e));
  }
  std::memset(t->mail, 0, sizeof(Mail));
  *out = t;
  return PCDN_OK;
}

void task_destroy(SolveTask* t) {
  if (!t) return;
  if (t->ev) {
    cudaEventSynchronize(t->ev);
    cudaEventDestroy(t->ev);
  }
  if (t->mail) cudaFreeHost(t->mail);
  delete t;
}

namespace {

// The stage's scalars into the mailbox, then the stage's completion event.
int post(SolveTask* t, int kkt_slot, bool final_stage) {
  pcdn_problem* p = t->p;
  if (kkt_slot >= 0)
    CUDA_TRY(cudaMemcpyAsync(&t->mail->kkt, p->red_out + kkt_slot, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  if (kkt_slot == 1 && t->o.shrink)
    CUDA_TRY(cudaMemcpyAsync(t->mail->act, p->shr + 1, sizeof(t->mail->act), cudaMemcpyDeviceToHost, p->stream));
  if (final_stage) {
    CUDA_TRY(cudaMemcpyAsync(&t->mail->F, p->red_out, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaMemcpyAsync(t->mail->cnt, p->counters, sizeof(t->mail->cnt), cudaMemcpyDeviceToHost, p->stream));
  }
  CUDA_TRY(cudaMemcpyAsync(&t->mail->err, p->err, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(record(t->ev, p));
  return PCDN_OK;
}

void release_blocks(SolveTask* t) {
  if (t->held > 0 && t->budget) t->budget->free.fetch_add(t->held);
  t->held = 0;
}

// Walker blocks for the solve: up to t->want from the budget when at least two are free (a
// cooperative launch), else one (an ordinary launch).
void take_blocks(SolveTask* t) {
  int g = 1;
  if (t->budget && t->want > 1) {
    int f = t->budget->free.load();
    while (f >= 2) {
      const int take = std::min(f, t->want);
      if (t->budget->free.compare_exchange_weak(f, f - take)) {
        g = take;
        break;
      }
    }
  }
  t->held = g > 1 ? g : 0;
  pcdn_opts o = t->o;
  o.grid_ctas = g;
  t->grid = pick_grid(t->p, &o, t->P);
}

// One outer iteration: partition (Eq. 8) of iteration k (or of the index in epoch_dev, advanced at
// the end), work items, the bundle walk, refresh, KKT, the mailbox.
int epoch_body(SolveTask* t, int64_t k, int64_t* epoch_dev) {
  pcdn_problem* p = t->p;
  int32_t* perm = nullptr;
  int rc = make_partition(p, t->seed, k, &perm, epoch_dev);
  if (rc) return rc;
  if (t->shrunk && (rc = shrink_partition(p, perm, &perm))) return rc;
  const int64_t npos = t->shrunk ? t->npos : p->m;
  CUDA_TRY(build_items(perm, npos, p->col_ptr, p->w, p->cnt, p->item_ptr, p->items, p->scan_ws, p->stream,
                       &p->launches));
  rc = run_walk(p, &t->o, perm, npos, t->P, 0, (npos + t->P - 1) / t->P, t->grid, nullptr);
  if (rc) return rc;
  if (t->o.refresh) {
    rc = do_refresh(p, (int)t->o.prec, true, false);
    if (rc) return rc;
  }
  rc = do_kkt(p, 1, t->o.shrink != 0);
  if (rc) return rc;
  if (epoch_dev) CUDA_TRY(advance_epoch(epoch_dev, p->stream, &p->launches));
  return post(t, 1, false);
}

// Capture one outer iteration into t->exec; on any failure the task keeps issuing directly.
void capture_epoch(SolveTask* t) {
  pcdn_problem* p = t->p;
  t->graph_tried = true;
  if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  p->capturing = true;
  const int64_t l0 = p->launches;
  const int rc = epoch_body(t, t->o.epoch0, p->epoch_dev);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  p->capturing = false;
  const int64_t kernels = p->launches - l0;
  p->launches = l0;
  cudaGetLastError();
  if (rc != PCDN_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    g_err.clear();
    return;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  t->exec = ex;
  t->graph_kernels = kernels;
}

int issue_epoch(SolveTask* t, int64_t k) {
  NvtxRange range("issue outer iteration");
  pcdn_problem* p = t->p;
  // a shrinking solve's outer iterations differ in size: issued directly
  if (t->graphs && !t->graph_tried && !t->o.shrink) capture_epoch(t);
  t->stage = kStageEpoch;
  if (t->exec) {
    CUDA_TRY(cudaGraphLaunch(t->exec, p->stream));
    p->launches += t->graph_kernels;
    t->used_graph = true;
    return PCDN_OK;
  }
  return epoch_body(t, t->o.epoch0 + k, nullptr);
}

int issue_final(SolveTask* t) {
  int rc = do_objective(t->p, 0);
  if (rc) return rc;
  t->stage = kStageFinal;
  return post(t, -1, true);
}

int end_task(SolveTask* t, int rc) {
  release_blocks(t);
  if (t->exec) {
    cudaGraphExecDestroy(t->exec);  // freed once a launch still in flight completes
    t->exec = nullptr;
  }
  t->stage = kStageEnded;
  t->rc = rc;
  t->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t->t0).count();
  return rc;
}

}  // namespace

int task_start(SolveTask* t, pcdn_problem* p, int32_t P, double eps, uint64_t seed, const pcdn_opts* opts, int grid) {
  g_err.clear();
  if (!t || !p) return fail(PCDN_EINVAL, "task and problem must be given");
  if (t->stage != kStageNone && t->stage != kStageEnded) return fail(PCDN_EINVAL, "task has a solve in flight");
  if (P < 1 || P > p->m) return fail(PCDN_EINVAL, "P must be in [1, n_features]");
  if (!(eps > 0)) return fail(PCDN_EINVAL, "eps must be positive");
  pcdn_opts o;
  if (opts) o = *opts;
  else pcdn_default_opts(&o);
  int rc = check_opts(&o);
  if (rc) return rc;
  if (grid > 0) o.grid_ctas = grid;
  t->p = p;
  t->o = o;
  t->P = P;
  t->eps = eps;
  t->seed = seed;
  t->nb = (p->m + P - 1) / P;
  t->held = 0;
  t->graph_tried = false;
  t->exec = nullptr;
  t->used_graph = false;
  t->graph_kernels = 0;
  if (t->budget) take_blocks(t);
  else t->grid = pick_grid(p, &o, P);
  t->kkt0 = t->kkt_rel = t->F = t->walk_ms = 0.0;
  t->epochs = 0;
  t->npos = p->m;
  t->nnz_next = p->nnz;
  t->nnz_visited = 0;
  t->shrunk = false;
  t->converged = 0;
  t->rc = PCDN_OK;
  t->launches0 = p->launches;
  t->t0 = std::chrono::steady_clock::now();
  std::memset(t->cnt, 0, sizeof(t->cnt));
  if ((rc = ensure_bundle_scratch(p, P)) || (rc = ensure_trace(p, t->nb)) ||
      (rc = ensure_plan(p, t->nb * (t->grid + 1))) || (rc = reset_scratch(p)) || (o.shrink && (rc = ensure_shrink(p))) ||
      (walk_layout(p, &o, t->grid) == PCDN_LAYOUT_ROWS && (rc = ensure_rows(p, t->nb, t->grid))))
    return end_task(t, rc);
  // from here every failure ends the task (which returns its walker blocks)
  cudaError_t e = cudaSuccess;
  if ((!o.warm_start && (e = cudaMemsetAsync(p->w, 0, sizeof(double) * p->m, p->stream)) != cudaSuccess) ||
      (e = cudaMemsetAsync(p->err, 0, sizeof(int), p->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(p->counters, 0, sizeof(unsigned long long) * 8, p->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(p->epoch_dev, 0, sizeof(int64_t), p->stream)) != cudaSuccess)
    return end_task(t, fail(PCDN_ECUDA, "solve set-up: %s", cudaGetErrorString(e)));
  if ((rc = start_state(p, (int)o.prec, !o.warm_start)) || (rc = do_kkt(p, 2))) return end_task(t, rc);
  t->stage = kStageStart;
  rc = post(t, 2, false);
  if (rc) return end_task(t, rc);
  return PCDN_OK;
}

int task_poll(SolveTask* t, int* done) {
  *done = 0;
  if (!t || t->stage == kStageNone) return fail(PCDN_EINVAL, "no solve started");
  if (t->stage == kStageEnded) {
    *done = 1;
    return t->rc;
  }
  const cudaError_t q = cudaEventQuery(t->ev);
  if (q == cudaErrorNotReady) return PCDN_OK;
  int rc = PCDN_OK;
  if (q != cudaSuccess) {
    rc = fail(PCDN_ECUDA, "solve stage: %s", cudaGetErrorString(q));
  } else {
    rc = status_from_flags(t->mail->err);
  }
  if (rc) {
    *done = 1;
    return end_task(t, rc);
  }
  switch (t->stage) {
    case kStageStart:
      t->kkt0 = t->mail->kkt;
      t->kref = t->o.kkt_ref > 0 ? t->o.kkt_ref : t->kkt0;
      t->kkt_rel = t->kkt0 > 0 ? t->kkt0 / t->kref : 0.0;
      t->converged = t->kkt0 == 0.0 || (t->o.kkt_ref > 0 && t->kkt_rel <= t->eps);
      rc = (!t->converged && t->o.max_epochs > 0) ? issue_epoch(t, 0) : issue_final(t);
      break;
    case kStageEpoch: {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, t->p->ev0, t->p->ev1) == cudaSuccess) t->walk_ms += ms;
      cudaGetLastError();
      t->epochs += 1;
      t->nnz_visited += t->nnz_next;
      t->kkt_rel = t->kref > 0 ? t->mail->kkt / t->kref : 0.0;
      if (t->kkt_rel <= t->eps) t->converged = 1;
      // the next outer iteration's active set (all features when shrinking is off or the set is empty)
      t->shrunk = t->o.shrink && t->mail->act[0] > 0;
      t->npos = t->shrunk ? (int64_t)t->mail->act[0] : t->p->m;
      t->nnz_next = t->shrunk ? (int64_t)t->mail->act[1] : t->p->nnz;
      rc = (t->converged || t->epochs >= t->o.max_epochs) ? issue_final(t) : issue_epoch(t, t->epochs);
      break;
    }
    case kStageFinal:
      t->F = t->mail->F;
      std::memcpy(t->cnt, t->mail->cnt, sizeof(t->cnt));
      *done = 1;
      return end_task(t, t->converged ? PCDN_OK : PCDN_ENOTCONVERGED);
    default:
      break;
  }
  if (rc) {
    *done = 1;
    return end_task(t, rc);
  }
  return PCDN_OK;
}

int task_wait(SolveTask* t) {
  if (!t || t->stage == kStageNone || t->stage == kStageEnded) return PCDN_OK;
  CUDA_TRY(cudaEventSynchronize(t->ev));
  return PCDN_OK;
}

int task_result(SolveTask* t, double* w_out, pcdn_stats* stats) {
  if (!t || t->stage != kStageEnded) return fail(PCDN_EINVAL, "the solve has not ended");
  pcdn_problem* p = t->p;
  if (w_out) {
    CUDA_TRY(cudaMemcpyAsync(w_out, p->w, sizeof(double) * p->m, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->epochs = t->epochs;
    stats->bundles = (int64_t)t->cnt[5];
    stats->coord_updates = (int64_t)t->cnt[6];
    stats->ls_steps = (int64_t)t->cnt[0];
    stats->ls_cap_hits = (int64_t)t->cnt[1];
    stats->ls_passes = (int64_t)t->cnt[2];
    stats->nnz_visited = t->nnz_visited;
    stats->rows_touched = (int64_t)t->cnt[4];
    stats->kernel_launches = p->launches - t->launches0;
    stats->F_final = t->F;
    stats->kkt_rel = t->kkt_rel;
    stats->kkt0 = t->kkt0;
    stats->walk_s = t->walk_ms * 1e-3;
    stats->bytes_model = 16.0 * (double)stats->nnz_visited + 33.0 * (double)stats->rows_touched +
                         16.0 * (double)stats->coord_updates;
    stats->converged = t->converged;
    stats->walk_grid = t->grid;
    stats->wall_s = t->wall_s;
  }
  return t->rc;
}

int64_t problem_n_features(pcdn_problem* p) { return p ? p->m : 0; }
int64_t problem_nnz(pcdn_problem* p) { return p ? p->nnz : 0; }
bool problem_rows_layout_ok(pcdn_problem* p) { return p && p->n + p->m < kRowsMaxTerms; }

int64_t problem_bytes_estimate(int64_t n, int64_t m, int64_t nnz, int32_t P) {
  if (P < 1) P = 1;
  const int64_t max_items = m + nnz / kChunk + 2;
  const int64_t hm = radix_hist_elems(m);
  int64_t scan_n = std::max<int64_t>(std::max<int64_t>(hm, m + 1), max_items + 1);
  const int64_t nb = (m + P - 1) / P;
  int64_t b = 0;
  b += 8 * (m + 1) + 8 * nnz + n;                       // X by columns, labels
  b += (n + 15) / 16 * 16;                              // padded labels
  b += 8 * (n + 1) + 8 * nnz;                           // X by rows
  b += 16 * m + (int64_t)kStateBytes * n + 8 * n + 4 * ((n + 31) / 32);  // w, w_pos, sample records, delta, bitmap
  b += 16 * m + 8 * m + 16 * (m + 1) + (int64_t)sizeof(Item) * max_items;           // keys, values, cnt, item_ptr, items
  b += 8 * hm + 8 * scan_workspace_elems(scan_n) + 16 * max_items + 16 * (max_items + 1);
  b += 4 * m + 8 * (m + 1) + (int64_t)sizeof(Item) * max_items;                     // identity-order items
  b += 8 * 3 * kPartStride * kAccPad + 4096;                                         // accumulators, flags, partials
  b += 32 * (int64_t)P + 28 * nb + 16 * nb;                                          // bundle scratch, trace, plan (1 block)
  // the row mirror's build workspace, held while the problem is created: entry columns, the
  // counting sort's (row, col, val) arrays between passes, histograms and offsets, row counts
  const MirrorSizes z = mirror_sizes(n, nnz);
  const int64_t transient = 4 * nnz + 4 * nnz * z.tmp_row + 12 * nnz * z.tmp_triple + 16 * z.hist +
                            8 * scan_workspace_elems(z.hist) +
                            8 * (n + 1) + 8 * scan_workspace_elems(n + 1);
  return b + transient;
}

}  // namespace pcdn

extern "C" {

void pcdn_default_opts(pcdn_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->sigma = 0.01;
  o->beta = 0.5;
  o->gamma = 0.0;
  o->nu = 1e-12;
  o->q_max = 30;
  o->ls_batch = 0;
  o->max_epochs = 1000;
  o->prec = PCDN_PREC_FP64;
  o->warm_start = 0;
  o->grid_ctas = 0;
  o->refresh = 1;
  o->spin_limit = 0;
  o->layout = PCDN_LAYOUT_AUTO;
}

const char* pcdn_last_error(void) { return g_err.c_str(); }

int pcdn_create(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, pcdn_problem** out) {
  g_err.clear();
  NvtxRange range("pcdn_create");
  if (!out) return fail(PCDN_EINVAL, "out must be given");
  *out = nullptr;
  if (!(C > 0) || !std::isfinite(C)) return fail(PCDN_EINVAL, "C must be positive and finite");
  if (loss != PCDN_LOSS_LOGISTIC && loss != PCDN_LOSS_L2SVM) return fail(PCDN_EINVAL, "unknown loss");
  int rc = check_host_shape(X, y);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    rc = check_host_entries(X, y);  // bad input is PCDN_EINVAL with or without a device
    if (rc) return rc;
    return fail(PCDN_ECUDA, "no CUDA device");
  }
  pcdn_problem* p = new (std::nothrow) pcdn_problem();
  if (!p) return fail(PCDN_ENOMEM, "host allocation");
  p->n = X->n_samples;
  p->m = X->n_features;
  p->nnz = X->nnz;
  p->c = C;
  p->loss = (int)loss;
  p->owns_x = true;
  auto bail = [&](int code) { free_all(p); delete p; return code; };
  if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(PCDN_ECUDA, "stream creation failed"));
  p->own_stream = true;
  cudaError_t e;
  if ((e = palloc(p, &p->col_ptr, p->m + 1)) || (e = palloc(p, &p->row_idx, p->nnz)) || (e = palloc(p, &p->val, p->nnz)) ||
      (e = palloc(p, &p->y, p->n)))
    return bail(fail(e == cudaErrorMemoryAllocation ? PCDN_ENOMEM : PCDN_ECUDA, "input allocation: %s", cudaGetErrorString(e)));
  if ((e = cudaMemcpyAsync(p->col_ptr, X->col_ptr, sizeof(int64_t) * (p->m + 1), cudaMemcpyHostToDevice, p->stream)) ||
      (p->nnz > 0 && (e = cudaMemcpyAsync(p->row_idx, X->row_idx, sizeof(int32_t) * p->nnz, cudaMemcpyHostToDevice, p->stream))) ||
      (p->nnz > 0 && (e = cudaMemcpyAsync(p->val, X->val, sizeof(float) * p->nnz, cudaMemcpyHostToDevice, p->stream))) ||
      (e = cudaMemcpyAsync(p->y, y, p->n, cudaMemcpyHostToDevice, p->stream)))
    return bail(fail(PCDN_ECUDA, "input copy: %s", cudaGetErrorString(e)));
  // every entry is checked on the device right after the copies (the same tests as the host check),
  // while the row mirror and workspaces are built behind it (their writes stay inside their arrays
  // for any entries); what follows col_ptr (the work items) waits for the verdict.  A rejected
  // input is checked again on the host for a message that names the entry.
  int* flag = nullptr;
  if ((e = dalloc(&flag, 1, p->stream)) || (e = cudaMemsetAsync(flag, 0, sizeof(int), p->stream)) ||
      (e = validate_device(p->col_ptr, p->row_idx, p->val, p->y, p->n, p->m, p->nnz, flag, p->stream, &p->launches)))
    return bail(fail(PCDN_ECUDA, "validation launch: %s", cudaGetErrorString(e)));
  rc = finish_create(p);
  // the verdict, read once the stream is idle (a device-to-host copy into pageable memory in the
  // middle of the stream would hold the host until the copies ahead of it finished)
  cudaStreamSynchronize(p->stream);
  int hflag = 0;
  e = cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost);
  dfree(flag, p->stream);
  if (e != cudaSuccess) return bail(fail(PCDN_ECUDA, "validation: %s", cudaGetErrorString(e)));
  if (hflag) {
    const int rc_host = check_host_entries(X, y);
    const std::string msg = rc_host ? pcdn_last_error() : "";
    bail(PCDN_EINVAL);
    if (rc_host) {
      set_last_error(msg.c_str());
      return rc_host;
    }
    return fail(PCDN_EINVAL, "CSC/labels invalid (flags 0x%x)", hflag);
  }
  if (rc) return bail(rc);
  rc = finish_create_checked(p);
  if (rc) return bail(rc);
  *out = p;
  return PCDN_OK;
}

int pcdn_create_device(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, void* stream, pcdn_problem** out) {
  g_err.clear();
  NvtxRange range("pcdn_create_device");
  if (!out) return fail(PCDN_EINVAL, "out must be given");
  *out = nullptr;
  if (!X || !y) return fail(PCDN_EINVAL, "X and y must be given");
  if (!(C > 0) || !std::isfinite(C)) return fail(PCDN_EINVAL, "C must be positive and finite");
  if (loss != PCDN_LOSS_LOGISTIC && loss != PCDN_LOSS_L2SVM) return fail(PCDN_EINVAL, "unknown loss");
  if (X->n_samples <= 0 || X->n_features <= 0 || X->nnz < 0 || X->n_samples > INT32_MAX || X->n_features > INT32_MAX ||
      X->nnz >= INT32_MAX)
    return fail(PCDN_EINVAL, "bad sizes");
  if (!X->col_ptr || (X->nnz > 0 && (!X->row_idx || !X->val))) return fail(PCDN_EINVAL, "CSC arrays missing");
  pcdn_problem* p = new (std::nothrow) pcdn_problem();
  if (!p) return fail(PCDN_ENOMEM, "host allocation");
  p->n = X->n_samples;
  p->m = X->n_features;
  p->nnz = X->nnz;
  p->c = C;
  p->loss = (int)loss;
  p->owns_x = false;
  p->col_ptr = const_cast<int64_t*>(X->col_ptr);
  p->row_idx = const_cast<int32_t*>(X->row_idx);
  p->val = const_cast<float*>(X->val);
  p->y = const_cast<int8_t*>(y);
  auto bail = [&](int code) { free_all(p); delete p; return code; };
  if (stream) {
    p->stream = (cudaStream_t)stream;
    p->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(PCDN_ECUDA, "stream creation failed"));
    p->own_stream = true;
  }
  cudaError_t e;
  if ((e = palloc(p, &p->err, 4)) || (e = cudaMemsetAsync(p->err, 0, sizeof(int) * 4, p->stream)))
    return bail(fail(PCDN_ECUDA, "flag allocation: %s", cudaGetErrorString(e)));
  if ((e = validate_device(p->col_ptr, p->row_idx, p->val, p->y, p->n, p->m, p->nnz, p->err, p->stream, &p->launches)))
    return bail(fail(PCDN_ECUDA, "validation launch: %s", cudaGetErrorString(e)));
  int flag = 0;
  if ((e = cudaMemcpyAsync(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream)) ||
      (e = cudaStreamSynchronize(p->stream)))
    return bail(fail(PCDN_ECUDA, "validation: %s", cudaGetErrorString(e)));
  if (flag) return bail(fail(PCDN_EINVAL, "device CSC/labels invalid (flags 0x%x)", flag));
  dfree(p->err, p->stream);
  p->err = nullptr;
  int rc = finish_create(p);
  if (!rc) rc = finish_create_checked(p);
  if (rc) return bail(rc);
  *out = p;
  return PCDN_OK;
}

void pcdn_destroy(pcdn_problem* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  free_all(p);
  delete p;
}

int pcdn_set_w(pcdn_problem* p, const double* w) {
  g_err.clear();
  if (!p || !w) return fail(PCDN_EINVAL, "problem and w must be given");
  for (int64_t j = 0; j < p->m; ++j)
    if (!std::isfinite(w[j])) return fail(PCDN_EINVAL, "w[%lld] is not finite", (long long)j);
  CUDA_TRY(cudaMemcpyAsync(p->w, w, sizeof(double) * p->m, cudaMemcpyHostToDevice, p->stream));
  CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  int rc = reset_scratch(p);
  if (rc) return rc;
  rc = do_refresh(p, p->rec_prec, true, false);
  if (rc) return rc;
  return device_status(p);
}

int pcdn_set_C(pcdn_problem* p, double C) {
  g_err.clear();
  if (!p) return fail(PCDN_EINVAL, "problem must be given");
  if (!(C > 0) || !std::isfinite(C)) return fail(PCDN_EINVAL, "C must be positive and finite");
  // the maintained quantities and the per-sample coefficients do not involve c
  p->c = C;
  return PCDN_OK;
}

int pcdn_set_penalty(pcdn_problem* p, double l1, double l2) {
  g_err.clear();
  if (!p) return fail(PCDN_EINVAL, "problem must be given");
  if (!(l1 >= 0) || !(l2 >= 0) || !std::isfinite(l1) || !std::isfinite(l2))
    return fail(PCDN_EINVAL, "l1 and l2 must be finite and >= 0");
  if (l1 == 0.0 && l2 == 0.0) return fail(PCDN_EINVAL, "l1 and l2 must not both be 0");
  // like c, the penalty enters only the directions, Delta, the line search's penalty change and the
  // stopping test; w and the maintained quantities are kept
  p->l1 = l1;
  p->l2 = l2;
  return PCDN_OK;
}

int pcdn_get_w(pcdn_problem* p, double* w) {
  g_err.clear();
  if (!p || !w) return fail(PCDN_EINVAL, "problem and w must be given");
  CUDA_TRY(cudaMemcpyAsync(w, p->w, sizeof(double) * p->m, cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  return PCDN_OK;
}

int pcdn_objective(pcdn_problem* p, double* F) {
  g_err.clear();
  if (!p || !F) return fail(PCDN_EINVAL, "problem and F must be given");
  int rc = do_objective(p, 0);
  if (rc) return rc;
  return read_double(p, 0, F);
}

int pcdn_kkt(pcdn_problem* p, double* kkt) {
  g_err.clear();
  if (!p || !kkt) return fail(PCDN_EINVAL, "problem and kkt must be given");
  int rc = do_kkt(p, 1);
  if (rc) return rc;
  return read_double(p, 1, kkt);
}

int pcdn_permutation(pcdn_problem* p, uint64_t seed, int64_t epoch, int32_t* perm) {
  g_err.clear();
  if (!p || !perm || epoch < 0) return fail(PCDN_EINVAL, "problem, perm and epoch >= 0 must be given");
  int32_t* dperm = nullptr;
  int rc = make_partition(p, seed, epoch, &dperm);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(perm, dperm, sizeof(int32_t) * p->m, cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  return PCDN_OK;
}

int pcdn_memory(pcdn_problem* p, int64_t* bytes) {
  if (!p || !bytes) return fail(PCDN_EINVAL, "problem and bytes must be given");
  *bytes = p->device_bytes;
  return PCDN_OK;
}

int pcdn_bundle_step(pcdn_problem* p, const double* w_in, const int32_t* bundle, int32_t P, const pcdn_opts* opts,
                     double* g, double* h, double* d, double* Delta, int32_t* q, double* alpha, double* dF) {
  g_err.clear();
  NvtxRange range("pcdn_bundle_step");
  if (!p || !bundle) return fail(PCDN_EINVAL, "problem and bundle must be given");
  if (P < 1 || P > p->m) return fail(PCDN_EINVAL, "P must be in [1, n_features]");
  pcdn_opts o;
  if (opts) o = *opts;
  else pcdn_default_opts(&o);
  int rc = check_opts(&o);
  if (rc) return rc;
  {
    std::vector<uint8_t> seen((size_t)p->m, 0);
    for (int32_t k = 0; k < P; ++k) {
      const int32_t j = bundle[k];
      if (j < 0 || j >= p->m) return fail(PCDN_EINVAL, "bundle[%d] = %d out of range", k, j);
      if (seen[j]) return fail(PCDN_EINVAL, "feature %d repeated in the bundle", j);
      seen[j] = 1;
    }
  }
  const int prec = (int)o.prec;
  if (w_in) {
    for (int64_t j = 0; j < p->m; ++j)
      if (!std::isfinite(w_in[j])) return fail(PCDN_EINVAL, "w_in[%lld] is not finite", (long long)j);
    CUDA_TRY(cudaMemcpyAsync(p->w, w_in, sizeof(double) * p->m, cudaMemcpyHostToDevice, p->stream));
    rc = do_refresh(p, prec, true, false);
    if (rc) return rc;
  } else if (p->rec_prec != prec) {
    CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
    CUDA_TRY(convert_state(p->loss, prec, p->y, p->n, p->st, p->err, p->stream, &p->launches));
    p->rec_prec = prec;
    rc = device_status(p);
    if (rc) return rc;
  }
  rc = ensure_bundle_scratch(p, P);
  if (rc) return rc;
  rc = ensure_trace(p, 1);
  if (rc) return rc;
  rc = reset_scratch(p);
  if (rc) return rc;
  // the bundle is the feature order of a one-bundle walk
  CUDA_TRY(cudaMemcpyAsync(p->vals1, bundle, sizeof(int32_t) * P, cudaMemcpyHostToDevice, p->stream));
  CUDA_TRY(build_items(p->vals1, P, p->col_ptr, p->w, p->cnt, p->item_ptr, p->items, p->scan_ws, p->stream,
                       &p->launches));
  CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  CUDA_TRY(cudaMemsetAsync(p->counters, 0, sizeof(unsigned long long) * 8, p->stream));
  const int grid = pick_grid(p, &o, P);
  rc = run_walk(p, &o, p->vals1, P, P, 0, 1, grid, nullptr);
  if (rc) return rc;
  if (g) CUDA_TRY(cudaMemcpyAsync(g, p->gk, sizeof(double) * P, cudaMemcpyDeviceToHost, p->stream));
  if (h) CUDA_TRY(cudaMemcpyAsync(h, p->hk, sizeof(double) * P, cudaMemcpyDeviceToHost, p->stream));
  if (d) CUDA_TRY(cudaMemcpyAsync(d, p->dk, sizeof(double) * P, cudaMemcpyDeviceToHost, p->stream));
  int32_t hq = 0;
  double ha = 0, hD = 0, hF = 0;
  CUDA_TRY(cudaMemcpyAsync(&hq, p->tr_q, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaMemcpyAsync(&ha, p->tr_alpha, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaMemcpyAsync(&hD, p->tr_Delta, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaMemcpyAsync(&hF, p->tr_dF, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  rc = device_status(p);
  if (rc) return rc;
  if (q) *q = hq;
  if (alpha) *alpha = ha;
  if (Delta) *Delta = hD;
  if (dF) *dF = hF;
  return PCDN_OK;
}

int pcdn_solve(pcdn_problem* p, int32_t P, double eps, uint64_t seed, const pcdn_opts* opts, double* w_out,
               pcdn_stats* stats, pcdn_trace* trace) {
  g_err.clear();
  NvtxRange range("pcdn_solve");
  const auto t_start = std::chrono::steady_clock::now();
  if (!p) return fail(PCDN_EINVAL, "problem must be given");
  if (P < 1 || P > p->m) return fail(PCDN_EINVAL, "P must be in [1, n_features]");
  if (!(eps > 0)) return fail(PCDN_EINVAL, "eps must be positive");
  pcdn_opts o;
  if (opts) o = *opts;
  else pcdn_default_opts(&o);
  int rc = check_opts(&o);
  if (rc) return rc;
  const int prec = (int)o.prec;
  const int64_t nb = (p->m + P - 1) / P;
  const int64_t launches0 = p->launches;
  rc = ensure_bundle_scratch(p, P);
  if (rc) return rc;
  rc = ensure_trace(p, nb);
  if (rc) return rc;
  rc = reset_scratch(p);
  if (rc) return rc;
  if (o.shrink && (rc = ensure_shrink(p))) return rc;
  if (!o.warm_start) CUDA_TRY(cudaMemsetAsync(p->w, 0, sizeof(double) * p->m, p->stream));
  CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), p->stream));
  CUDA_TRY(cudaMemsetAsync(p->counters, 0, sizeof(unsigned long long) * 8, p->stream));
  rc = start_state(p, prec, !o.warm_start);
  if (rc) return rc;
  rc = do_kkt(p, 2);
  if (rc) return rc;
  double kkt0 = 0.0;
  rc = read_double(p, 2, &kkt0);
  if (rc) return rc;
  rc = device_status(p);
  if (rc) return rc;
  const int grid = pick_grid(p, &o, P);
  // the relative KKT's reference: the start point's, or the caller's (a resumed solve)
  const double kref = o.kkt_ref > 0 ? o.kkt_ref : kkt0;
  double kkt_rel = kkt0 > 0 ? kkt0 / kref : 0.0;
  int converged = kkt0 == 0.0 || (o.kkt_ref > 0 && kkt_rel <= eps);
  int64_t epochs = 0;
  double walk_ms = 0.0;
  // shrinking: features and nonzeros of the next outer iteration (all of them until a stopping test
  // has chosen an active set)
  int64_t npos = p->m, nnz_next = p->nnz, nnz_visited = 0, tr_off = 0;
  bool shrunk = false;
  for (int64_t k = 0; k < o.max_epochs && !converged; ++k) {
    NvtxRange iteration("outer iteration");
    int32_t* perm = nullptr;
    rc = make_partition(p, seed, o.epoch0 + k, &perm);
    if (rc) return rc;
    if (shrunk && (rc = shrink_partition(p, perm, &perm))) return rc;
    const int64_t nbk = (npos + P - 1) / P;
    CUDA_TRY(build_items(perm, npos, p->col_ptr, p->w, p->cnt, p->item_ptr, p->items, p->scan_ws, p->stream,
                         &p->launches));
    float ms = 0.0f;
    rc = run_walk(p, &o, perm, npos, P, 0, nbk, grid, &ms);
    if (rc) return rc;
    walk_ms += ms;
    nnz_visited += nnz_next;
    rc = device_status(p);
    if (rc) return rc;
    if (trace && (trace->q || trace->alpha || trace->Delta || trace->dF) && tr_off < trace->bundle_cap) {
      const int64_t cnt = std::min<int64_t>(nbk, trace->bundle_cap - tr_off);
      if (trace->q) CUDA_TRY(cudaMemcpyAsync(trace->q + tr_off, p->tr_q, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, p->stream));
      if (trace->alpha) CUDA_TRY(cudaMemcpyAsync(trace->alpha + tr_off, p->tr_alpha, sizeof(double) * cnt, cudaMemcpyDeviceToHost, p->stream));
      if (trace->Delta) CUDA_TRY(cudaMemcpyAsync(trace->Delta + tr_off, p->tr_Delta, sizeof(double) * cnt, cudaMemcpyDeviceToHost, p->stream));
      if (trace->dF) CUDA_TRY(cudaMemcpyAsync(trace->dF + tr_off, p->tr_dF, sizeof(double) * cnt, cudaMemcpyDeviceToHost, p->stream));
    }
    tr_off += nbk;
    if (trace && trace->epoch_features && k < trace->epoch_cap) trace->epoch_features[k] = npos;
    if (o.refresh) {
      rc = do_refresh(p, prec, true, false);
      if (rc) return rc;
    }
    rc = do_kkt(p, 1, o.shrink != 0);
    if (rc) return rc;
    unsigned long long act[2] = {0, 0};
    if (o.shrink) CUDA_TRY(cudaMemcpyAsync(act, p->shr + 1, sizeof(act), cudaMemcpyDeviceToHost, p->stream));
    double kk = 0.0;
    rc = read_double(p, 1, &kk);
    if (rc) return rc;
    rc = device_status(p);
    if (rc) return rc;
    epochs = k + 1;
    kkt_rel = kref > 0 ? kk / kref : 0.0;
    if (trace && trace->epoch_kkt && k < trace->epoch_cap) trace->epoch_kkt[k] = kkt_rel;
    if (kkt_rel <= eps) converged = 1;
    // an empty active set means v = 0 (every violating feature is active): the next outer
    // iteration, if any, visits every feature
    if (o.shrink && act[0] > 0) {
      shrunk = true;
      npos = (int64_t)act[0];
      nnz_next = (int64_t)act[1];
    } else {
      shrunk = false;
      npos = p->m;
      nnz_next = p->nnz;
    }
  }
  double F = 0.0;
  rc = do_objective(p, 0);
  if (rc) return rc;
  rc = read_double(p, 0, &F);
  if (rc) return rc;
  if (w_out) {
    CUDA_TRY(cudaMemcpyAsync(w_out, p->w, sizeof(double) * p->m, cudaMemcpyDeviceToHost, p->stream));
  }
  unsigned long long cnt[8] = {0};
  CUDA_TRY(cudaMemcpyAsync(cnt, p->counters, sizeof(cnt), cudaMemcpyDeviceToHost, p->stream));
  CUDA_TRY(cudaStreamSynchronize(p->stream));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->epochs = epochs;
    stats->bundles = (int64_t)cnt[5];
    stats->coord_updates = (int64_t)cnt[6];
    stats->ls_steps = (int64_t)cnt[0];
    stats->ls_cap_hits = (int64_t)cnt[1];
    stats->ls_passes = (int64_t)cnt[2];
    stats->nnz_visited = nnz_visited;
    stats->rows_touched = (int64_t)cnt[4];
    stats->kernel_launches = p->launches - launches0;
    stats->F_final = F;
    stats->kkt_rel = kkt_rel;
    stats->kkt0 = kkt0;
    stats->walk_s = walk_ms * 1e-3;
    stats->bytes_model = 16.0 * (double)stats->nnz_visited + 33.0 * (double)stats->rows_touched +
                         16.0 * (double)stats->coord_updates;
    stats->converged = converged;
    stats->walk_grid = grid;
    stats->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  return converged ? PCDN_OK : PCDN_ENOTCONVERGED;
}

}  // extern "C"
