// The row-major mirror of X: row_ptr, col_idx, rval with every row's entries in ascending column
// order (the order of the FP64 refresh's sums of z = Xw, Algorithm 4's recomputation).
//
// The CSC entries are in column order with rows ascending inside a column, so the mirror is the
// stable sort of the entries by row.  It is formed as a least-significant-digit counting sort on
// the row index, digits of at most 10 bits (up to 1024 bins, as few passes as the row count needs:
// one up to 1024 samples, two up to 2^20, three up to 2^30).  One pass:
//   count: per tile of 4096 entries a histogram of the digit, hist[digit * tiles + tile];
//   scan:  an exclusive scan of hist gives every (digit, tile) run its first output slot;
//   place: each warp ranks its entries among equal digits (ballots over the digit's bits), the
//          tile's entries are grouped by digit in shared memory, and each digit's run is written out
//          with consecutive stores (whole sectors instead of one scattered word per entry).
// Every pass is stable, so entries of one row keep their column order.  No atomics touch the
// output, and the result does not depend on scheduling.

#include <algorithm>

#include "pcdn_prep.h"

namespace pcdn {

namespace {

constexpr int kMTileWarps = 8;
constexpr int kMTileSteps = 16;
constexpr int kMTile = kMTileWarps * kMTileSteps * 32;  // 4096 entries
constexpr int kMBins = 1024;
constexpr int kMThreads = kMTileWarps * 32;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline cudaError_t post(int64_t* launches) {
  if (launches) ++*launches;
  return cudaGetLastError();
}

// Digit of a row index (bins a power of two; the mask keeps a malformed index inside the bins).
__device__ __forceinline__ int digit_of(int32_t r, int shift, int nbins) { return (int)(((uint32_t)r >> shift) & (uint32_t)(nbins - 1)); }

__global__ void __launch_bounds__(kMThreads) mirror_count_kernel(const int32_t* __restrict__ rows, int64_t nnz, int shift,
                                                                 int nbins, int64_t tiles, int64_t* __restrict__ hist) {
  __shared__ int cnt[kMBins];
  for (int b = threadIdx.x; b < nbins; b += kMThreads) cnt[b] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kMTile + threadIdx.x;
#pragma unroll 4
  for (int s = 0; s < kMTile / kMThreads; ++s) {
    const int64_t e = base + (int64_t)s * kMThreads;
    if (e < nnz) atomicAdd(&cnt[digit_of(__ldg(rows + e), shift, nbins)], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += kMThreads) hist[(int64_t)b * tiles + blockIdx.x] = cnt[b];
}

struct MirrorSmem {
  int cnt[kMTileWarps][kMBins];  // per-warp counts, then per-warp offsets within the digit's run
  int tloc[kMBins + 1];          // start of each digit's run in the tile
  int dst[kMBins];               // each digit's run: its first slot in the output
  int scan[kMTileWarps];
  int32_t row[kMTile];
  int32_t col[kMTile];
  float val[kMTile];
  int16_t dig[kMTile];
};

// One placement pass from (srow, scol, sval) to (drow, dcol, dval); LAST: the rows are not written
// (the output is col_idx and rval of the mirror).
template <bool LAST>
__global__ void __launch_bounds__(kMThreads) mirror_place_kernel(
    const int32_t* __restrict__ srow, const int32_t* __restrict__ scol, const float* __restrict__ sval, int64_t nnz,
    int shift, int nbins, int nbits, int64_t tiles, const int64_t* __restrict__ off, int32_t* __restrict__ drow,
    int32_t* __restrict__ dcol, float* __restrict__ dval) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MirrorSmem& sm = *reinterpret_cast<MirrorSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int b = lane; b < nbins; b += 32) sm.cnt[w][b] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * kMTile + (int64_t)w * (kMTileSteps * 32) + lane;
  int dg[kMTileSteps];
  int32_t rr[kMTileSteps];
#pragma unroll
  for (int s = 0; s < kMTileSteps; ++s) {
    const int64_t e = base + s * 32;
    rr[s] = e < nnz ? __ldg(srow + e) : 0;
    dg[s] = e < nnz ? digit_of(rr[s], shift, nbins) : -1;
  }
#pragma unroll
  for (int s = 0; s < kMTileSteps; ++s)
    if (dg[s] >= 0) atomicAdd(&sm.cnt[w][dg[s]], 1);
  __syncthreads();
  // per digit: the warps' offsets within its run and the run's length
  int tsum = 0;
  constexpr int kPerT = kMBins / kMThreads;
  int len[kPerT];
#pragma unroll
  for (int u = 0; u < kPerT; ++u) {
    const int b = tid * kPerT + u;
    if (b < nbins) sm.dst[b] = (int)off[(int64_t)b * tiles + blockIdx.x];
  }
#pragma unroll
  for (int u = 0; u < kPerT; ++u) {
    const int b = tid * kPerT + u;
    int run = 0;
    if (b < nbins) {
#pragma unroll
      for (int v = 0; v < kMTileWarps; ++v) {
        const int c = sm.cnt[v][b];
        sm.cnt[v][b] = run;
        run += c;
      }
    }
    len[u] = run;
    tsum += run;
  }
  int incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sm.scan[w] = incl;
  __syncthreads();
  int at = incl - tsum;
  for (int v = 0; v < w; ++v) at += sm.scan[v];
#pragma unroll
  for (int u = 0; u < kPerT; ++u) {
    const int b = tid * kPerT + u;
    if (b < nbins) sm.tloc[b] = at;
    at += len[u];
  }
  if (tid == kMThreads - 1) sm.tloc[nbins] = at;
  __syncthreads();
  // ranks (lanes with the same digit: one ballot per digit bit), then the entries into their runs
  // in shared memory
  const unsigned lt = (1u << lane) - 1u;
  int slot[kMTileSteps];
#pragma unroll
  for (int s = 0; s < kMTileSteps; ++s) {
    const int b = dg[s];
    unsigned peers = __ballot_sync(0xffffffffu, b >= 0);
    if (b < 0) peers = ~peers;
    for (int bit = 0; bit < nbits; ++bit) {
      const bool on = (b >> bit) & 1;
      const unsigned m = __ballot_sync(0xffffffffu, on);
      peers &= on ? m : ~m;
    }
    const int c0 = b >= 0 ? sm.cnt[w][b] : 0;
    __syncwarp();
    slot[s] = -1;
    if (b >= 0) {
      if ((peers & lt) == 0) sm.cnt[w][b] = c0 + __popc(peers);
      slot[s] = sm.tloc[b] + c0 + __popc(peers & lt);
    }
    __syncwarp();
  }
  constexpr int kGroup = 8;
#pragma unroll
  for (int g = 0; g < kMTileSteps; g += kGroup) {
    int32_t cc[kGroup];
    float vv[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t e = base + (g + u) * 32;
      cc[u] = slot[g + u] >= 0 ? __ldg(scol + e) : 0;
      vv[u] = slot[g + u] >= 0 ? __ldg(sval + e) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int d = slot[g + u];
      if (d >= 0) {
        sm.row[d] = rr[g + u];
        sm.col[d] = cc[u];
        sm.val[d] = vv[u];
        sm.dig[d] = (int16_t)dg[g + u];
      }
    }
  }
  __syncthreads();
  // the staged runs to the output: consecutive threads write consecutive slots of a run
  const int total = sm.tloc[nbins];
  for (int i = tid; i < total; i += kMThreads) {
    const int b = sm.dig[i];
    const int64_t d = (int64_t)sm.dst[b] + (i - sm.tloc[b]);
    if (!LAST) drow[d] = sm.row[i];
    dcol[d] = sm.col[i];
    dval[d] = sm.val[i];
  }
}

// Rows with an index outside [0, n) are not counted (input that the caller's check rejects).
__global__ void mirror_row_count_kernel(const int32_t* __restrict__ row_idx, int64_t nnz, int64_t n,
                                        unsigned long long* __restrict__ counts) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = __ldg(row_idx + e);
    if ((uint64_t)(uint32_t)r < (uint64_t)n) atomicAdd(counts + r, 1ull);
  }
}

void digits_of(int64_t n, int* passes, int* bits) {
  int key_bits = 1;
  while ((int64_t(1) << key_bits) < n) ++key_bits;
  *passes = (key_bits + 9) / 10;
  *bits = (key_bits + *passes - 1) / *passes;
}

}  // namespace

cudaError_t mirror_configure() {
  cudaError_t e = cudaFuncSetAttribute(mirror_place_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(MirrorSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(mirror_place_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(MirrorSmem));
}

MirrorSizes mirror_sizes(int64_t n, int64_t nnz) {
  MirrorSizes z;
  int passes, bits;
  digits_of(n, &passes, &bits);
  z.passes = passes;
  z.tiles = cdiv(nnz > 0 ? nnz : 1, kMTile);
  z.hist = (int64_t)(1 << bits) * z.tiles;
  z.tmp_row = passes >= 3 ? 1 : 0;
  z.tmp_triple = passes >= 2 ? 1 : 0;
  return z;
}

cudaError_t mirror_row_counts(const int32_t* row_idx, int64_t nnz, int64_t n, int64_t* counts, cudaStream_t s,
                              int64_t* launches) {
  if (nnz <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>(cdiv(nnz, 256), 16384);
  mirror_row_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(row_idx, nnz, n,
                                                           reinterpret_cast<unsigned long long*>(counts));
  return post(launches);
}

cudaError_t build_mirror(const int32_t* row_idx, const int32_t* entry_col, const float* val, int64_t nnz, int64_t n,
                         const MirrorWorkspace& ws, int32_t* col_idx, float* rval, cudaStream_t s, int64_t* launches) {
  if (nnz <= 0) return cudaSuccess;
  int passes, bits;
  digits_of(n, &passes, &bits);
  const int nbins = 1 << bits;
  const int64_t tiles = cdiv(nnz, kMTile);
  const int32_t* sr = row_idx;
  const int32_t* sc = entry_col;
  const float* sv = val;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * bits;
    const bool last = pass == passes - 1;
    mirror_count_kernel<<<(unsigned)tiles, kMThreads, 0, s>>>(sr, nnz, shift, nbins, tiles, ws.hist);
    cudaError_t e = post(launches);
    if (e != cudaSuccess) return e;
    e = scan_exclusive(ws.hist, ws.off, (int64_t)nbins * tiles, ws.scan_ws, s, launches);
    if (e != cudaSuccess) return e;
    if (last) {
      mirror_place_kernel<true><<<(unsigned)tiles, kMThreads, sizeof(MirrorSmem), s>>>(
          sr, sc, sv, nnz, shift, nbins, bits, tiles, ws.off, nullptr, col_idx, rval);
    } else {
      // the pass before the last one writes the workspace's triple; a first pass of three writes
      // its rows to the workspace and its columns and values to the output arrays (free until the
      // last pass, which reads the triple)
      const bool to_triple = pass == passes - 2;
      int32_t* dr = to_triple ? ws.trow : ws.row0;
      int32_t* dc = to_triple ? ws.tcol : col_idx;
      float* dv = to_triple ? ws.tval : rval;
      mirror_place_kernel<false><<<(unsigned)tiles, kMThreads, sizeof(MirrorSmem), s>>>(
          sr, sc, sv, nnz, shift, nbins, bits, tiles, ws.off, dr, dc, dv);
      sr = dr;
      sc = dc;
      sv = dv;
    }
    e = post(launches);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pcdn
