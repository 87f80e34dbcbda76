// The row-sorted bundle layout of one outer iteration (used by walk_rows_kernel).
//
// Algorithm 4 needs d^T x_i over the samples a bundle touches.  Instead of scattering d_j x_ij into
// a dense vector with atomics, the walker lets the owner of sample i sum its own terms: for every
// bundle t the entries of the bundle's columns are stored grouped by row (rows ascending, columns
// ascending within a row), each with its row, its position k within the bundle and its value.
// That layout is a stable partition of the row-major mirror of X by bundle index (the mirror is in
// row order with columns ascending, and bundle b holds the features at positions [bP, (b+1)P) of
// the partition, Eq. 8):
//   bundles <= kBins: one counting sort: per tile of 8192 entries a histogram of bundle indexes,
//     an exclusive scan over (bundle, tile), then every warp places its 1024 entries in order
//     (ranks among equal bundle indexes by warp match);
//   more bundles: a stable LSD radix sort of (bundle index, entry) pairs, then a gather.
// Entries of features outside the walk (shrinking) are left out.  br_plan cuts every bundle's
// entries into the walker's per-block ranges at row starts, balanced by entry count.

#include "pcdn_prep.h"

namespace pcdn {

namespace {

constexpr int kTileWarps = 8;
constexpr int kTileSteps = 16;                                    // 32 entries per step and warp
constexpr int kTile = kTileWarps * kTileSteps * 32;  // 4096 entries

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline cudaError_t post(int64_t* launches) {
  if (launches) ++*launches;
  return cudaGetLastError();
}

// Row of every mirror entry: a warp per row.
__global__ void entry_rows_kernel(const int64_t* row_ptr, int64_t n, int32_t* entry_row) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    const int64_t a = row_ptr[i], b = row_ptr[i + 1];
    for (int64_t e = a + lane; e < b; e += 32) entry_row[e] = (int32_t)i;
  }
}

// inv[perm[k]] = k for the walk's positions k < npos (inv preset to -1).
__global__ void positions_kernel(const int32_t* perm, int64_t npos, int32_t* inv) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npos; k += (int64_t)gridDim.x * blockDim.x)
    inv[perm[k]] = (int32_t)k;
}

// Position of mirror entry e's feature in the walk (-1: not in the walk).
__device__ __forceinline__ int32_t entry_pos(const int32_t* col_idx, const int32_t* inv, int64_t e, int64_t nnz) {
  return e < nnz ? __ldg(inv + __ldg(col_idx + e)) : -1;
}

// pos / P for a bundle index below kBins: an FP32 estimate, then one correction step (the estimate
// is within one of the quotient), instead of an integer division by a runtime divisor.
__device__ __forceinline__ int bundle_of(int32_t pos, int32_t P, float invP) {
  int b = (int)((float)pos * invP);
  const int r = pos - b * P;
  if (r < 0) --b;
  else if (r >= P) ++b;
  return b;
}

// Per tile: histogram of bundle indexes into hist[b * tiles + tile].
__global__ void __launch_bounds__(kTileWarps * 32) rows_count_kernel(const int32_t* col_idx, int64_t nnz,
                                                                      const int32_t* inv, int32_t P, float invP,
                                                                      int nb, int64_t tiles, int64_t* hist) {
  __shared__ int cnt[kBins];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)(threadIdx.x >> 5) * (kTileSteps * 32) + (threadIdx.x & 31);
  for (int s0 = 0; s0 < kTileSteps; s0 += 8) {
    int32_t pos[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) pos[u] = entry_pos(col_idx, inv, base + (s0 + u) * 32, nnz);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (pos[u] >= 0) atomicAdd(&cnt[bundle_of(pos[u], P, invP)], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[(int64_t)b * tiles + blockIdx.x] = cnt[b];
}

// Per tile: every entry to its place (off = exclusive scan of hist).  Warp w of the tile counts its
// entries per bundle; an entry's rank within its bundle in the tile is the entries of that bundle in
// earlier warps plus those earlier in this warp (warp match).  The tile's entries are first grouped
// by bundle in shared memory, then each bundle's run is written out with consecutive stores (the
// run's slots in the output are contiguous), so that the output is written in whole sectors rather
// than one scattered word per entry.
struct PlaceSmem {
  int cnt[kTileWarps][kBins];  // per-warp counts, then per-warp offsets within the bundle's run
  int tloc[kBins + 1];         // start of each bundle's run in the tile
  int dst[kBins];              // each bundle's run: its first slot in the output
  int scan[kTileWarps];
  int32_t row[kTile];
  int32_t k[kTile];
  float val[kTile];
  int16_t bun[kTile];  // each staged entry's bundle
};

__global__ void __launch_bounds__(kTileWarps * 32) rows_place_kernel(const int32_t* __restrict__ col_idx,
                                                                      const float* __restrict__ rval,
                                                                      const int32_t* __restrict__ entry_row,
                                                                      int64_t nnz, const int32_t* __restrict__ inv,
                                                                      int32_t P, float invP, int nb, int64_t tiles,
                                                                      const int64_t* __restrict__ off,
                                                                      int32_t* __restrict__ br_row,
                                                                      int32_t* __restrict__ br_k,
                                                                      float* __restrict__ br_val) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PlaceSmem& sm = *reinterpret_cast<PlaceSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int b = lane; b < nb; b += 32) sm.cnt[w][b] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)w * (kTileSteps * 32) + lane;
  int32_t pos[kTileSteps];
#pragma unroll
  for (int s = 0; s < kTileSteps; ++s) {
    pos[s] = entry_pos(col_idx, inv, base + s * 32, nnz);
    if (pos[s] >= 0) atomicAdd(&sm.cnt[w][bundle_of(pos[s], P, invP)], 1);
  }
  __syncthreads();
  // per bundle: the warps' offsets within its run, and the run's length (kBins / 256 bundles a thread)
  constexpr int kPerT = kBins / (kTileWarps * 32);
  int len[kPerT];
  int tsum = 0;
#pragma unroll
  for (int u = 0; u < kPerT; ++u) {
    const int b = tid * kPerT + u;
    if (b < nb) sm.dst[b] = (int)off[(int64_t)b * tiles + blockIdx.x];  // all loads of the tile in flight
  }
#pragma unroll
  for (int u = 0; u < kPerT; ++u) {
    const int b = tid * kPerT + u;
    int run = 0;
    if (b < nb) {
#pragma unroll
      for (int v = 0; v < kTileWarps; ++v) {
        const int c = sm.cnt[v][b];
        sm.cnt[v][b] = run;
        run += c;
      }
    }
    len[u] = run;
    tsum += run;
  }
  // runs start at an exclusive scan of the lengths over bundles
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
    if (b < nb) sm.tloc[b] = at;
    at += len[u];
  }
  if (tid == kTileWarps * 32 - 1) sm.tloc[nb] = at;
  __syncthreads();
  // ranks, then the entries into their runs in shared memory (eight steps' loads in flight)
  const unsigned lt = (1u << lane) - 1u;
  int nbits = 1;
  while ((1 << nbits) < nb) ++nbits;
  int slot[kTileSteps];
  int bun[kTileSteps];
#pragma unroll
  for (int s = 0; s < kTileSteps; ++s) {
    const int32_t ps = pos[s];
    const int b = ps >= 0 ? bundle_of(ps, P, invP) : -1;
    // lanes holding the same bundle index: one ballot per bit of the index (and one for validity)
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
    bun[s] = b;
    if (b >= 0) {
      if ((peers & lt) == 0) sm.cnt[w][b] = c0 + __popc(peers);
      slot[s] = sm.tloc[b] + c0 + __popc(peers & lt);
      pos[s] = ps - b * P;  // the position within the bundle
    }
    __syncwarp();
  }
  constexpr int kGroup = 8;
#pragma unroll
  for (int g = 0; g < kTileSteps; g += kGroup) {
    int32_t rr[kGroup];
    float vv[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t e = base + (g + u) * 32;
      rr[u] = slot[g + u] >= 0 ? entry_row[e] : 0;
      vv[u] = slot[g + u] >= 0 ? rval[e] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int d = slot[g + u];
      if (d >= 0) {
        sm.row[d] = rr[u];
        sm.k[d] = pos[g + u];
        sm.val[d] = vv[u];
        sm.bun[d] = (int16_t)bun[g + u];
      }
    }
  }
  __syncthreads();
  // the staged entries to the output in order: an entry's slot is its bundle's run start plus its
  // offset in the run (runs are contiguous in both, so consecutive threads write consecutive words
  // within a run)
  const int total = sm.tloc[nb];
  for (int i = tid; i < total; i += kTileWarps * 32) {
    const int b = sm.bun[i];
    const int64_t d = (int64_t)sm.dst[b] + (i - sm.tloc[b]);
    br_row[d] = sm.row[i];
    br_k[d] = sm.k[i];
    br_val[d] = sm.val[i];
  }
}

// General path: keys (bundle index, nb for entries outside the walk) and entry indexes.
__global__ void rows_keys_kernel(const int32_t* col_idx, int64_t nnz, const int32_t* inv, int32_t P, uint32_t nb,
                                 uint32_t* keys, int32_t* vals) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t pos = inv[col_idx[e]];
    keys[e] = pos >= 0 ? (uint32_t)(pos / P) : nb;
    vals[e] = (int32_t)e;
  }
}

__global__ void rows_gather_kernel(const uint32_t* keys, const int32_t* vals, int64_t nnz, uint32_t nb,
                                   const int32_t* col_idx, const float* rval, const int32_t* entry_row,
                                   const int32_t* inv, int32_t P, int32_t* br_row, int32_t* br_k, float* br_val) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = keys[s];
    if (b >= nb) continue;
    const int32_t e = vals[s];
    br_row[s] = entry_row[e];
    br_k[s] = inv[col_idx[e]] - (int32_t)b * P;
    br_val[s] = rval[e];
  }
}

// br_ptr[b] = first sorted entry with key >= b (b in [0, nb]).
__global__ void rows_ptr_kernel(const uint32_t* keys, int64_t nnz, uint32_t nb, int64_t* br_ptr) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= (int64_t)nb; b += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < (uint32_t)b) lo = mid + 1;
      else hi = mid;
    }
    br_ptr[b] = lo;
  }
}

// Counting-sort path: br_ptr[b] = off[b * tiles] (off has nb * tiles + 1 entries, the last the total).
__global__ void rows_ptr_from_off_kernel(const int64_t* off, int nb, int64_t tiles, int64_t* br_ptr) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x)
    br_ptr[b] = off[(int64_t)b * tiles];
}

// br_plan[t * (G+1) + c]: block c's first entry of bundle t, the first row start at or after an
// equal share of the bundle's entries; br_plan[t * (G+1) + G] = the bundle's end.
__global__ void rows_plan_kernel(const int64_t* br_ptr, const int32_t* br_row, int64_t nb, int G, int64_t* br_plan) {
  const int64_t total = nb * (int64_t)(G + 1);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / (G + 1);
    const int c = (int)(idx - t * (G + 1));
    const int64_t e0 = br_ptr[t], e1 = br_ptr[t + 1];
    int64_t s = e0 + ((e1 - e0) * c) / G;
    if (c == G) s = e1;
    while (s > e0 && s < e1 && br_row[s] == br_row[s - 1]) ++s;
    br_plan[idx] = s;
  }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 8192) {
  int64_t g = cdiv(n > 0 ? n : 1, threads);
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

// The placement kernel's shared memory exceeds the 48 KB default: set on the current device before
// the first build (not inside a stream capture).
cudaError_t rows_configure() {
  return cudaFuncSetAttribute(rows_place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PlaceSmem));
}

cudaError_t entry_rows(const int64_t* row_ptr, int64_t n, int32_t* entry_row, cudaStream_t s, int64_t* launches) {
  entry_rows_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(row_ptr, n, entry_row);
  return post(launches);
}

int64_t rows_tiles(int64_t nnz) { return cdiv(nnz > 0 ? nnz : 1, kTile); }
int64_t rows_hist_elems(int64_t nnz) { return (int64_t)kBins * rows_tiles(nnz) + 1; }

cudaError_t build_rows(const int32_t* perm, int64_t npos, int64_t m, int32_t P, int64_t nb, int G,
                       const int32_t* col_idx, const float* rval, const int32_t* entry_row, int64_t nnz,
                       const RowsWorkspace& ws, int32_t* br_row, int32_t* br_k, float* br_val, int64_t* br_ptr,
                       int64_t* br_plan, cudaStream_t s, int64_t* launches) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.inv, 0xff, sizeof(int32_t) * m, s)) != cudaSuccess) return e;
  positions_kernel<<<grid_for(npos, 256), 256, 0, s>>>(perm, npos, ws.inv);
  if ((e = post(launches)) != cudaSuccess) return e;
  if (nb <= kBins) {
    const int64_t tiles = rows_tiles(nnz);
    const int64_t hn = nb * tiles + 1;
    if ((e = cudaMemsetAsync(ws.hist + hn - 1, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
    if (nnz > 0) {
      rows_count_kernel<<<(unsigned)tiles, kTileWarps * 32, 0, s>>>(col_idx, nnz, ws.inv, P, 1.0f / (float)P, (int)nb,
                                                                     tiles, ws.hist);
      if ((e = post(launches)) != cudaSuccess) return e;
    } else if ((e = cudaMemsetAsync(ws.hist, 0, sizeof(int64_t) * hn, s)) != cudaSuccess) {
      return e;
    }
    if ((e = scan_exclusive(ws.hist, ws.hist, hn, ws.scan_ws, s, launches)) != cudaSuccess) return e;
    if (nnz > 0) {
      rows_place_kernel<<<(unsigned)tiles, kTileWarps * 32, sizeof(PlaceSmem), s>>>(col_idx, rval, entry_row, nnz, ws.inv, P,
                                                                     1.0f / (float)P, (int)nb, tiles, ws.hist, br_row,
                                                                     br_k, br_val);
      if ((e = post(launches)) != cudaSuccess) return e;
    }
    rows_ptr_from_off_kernel<<<grid_for(nb + 1, 256), 256, 0, s>>>(ws.hist, (int)nb, tiles, br_ptr);
    if ((e = post(launches)) != cudaSuccess) return e;
  } else {
    int bits = 1;
    while ((int64_t(1) << bits) <= nb) ++bits;
    uint32_t* ko = ws.k0;
    int32_t* vo = ws.v0;
    if (nnz > 0) {
      rows_keys_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(col_idx, nnz, ws.inv, P, (uint32_t)nb, ws.k0, ws.v0);
      if ((e = post(launches)) != cudaSuccess) return e;
      if ((e = radix_sort_u32(ws.k0, ws.v0, ws.k1, ws.v1, nnz, bits, ws.rhist, ws.scan_ws, &ko, &vo, s, launches)) !=
          cudaSuccess)
        return e;
      rows_gather_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(ko, vo, nnz, (uint32_t)nb, col_idx, rval, entry_row, ws.inv,
                                                            P, br_row, br_k, br_val);
      if ((e = post(launches)) != cudaSuccess) return e;
    }
    rows_ptr_kernel<<<grid_for(nb + 1, 256), 256, 0, s>>>(ko, nnz, (uint32_t)nb, br_ptr);
    if ((e = post(launches)) != cudaSuccess) return e;
  }
  rows_plan_kernel<<<grid_for(nb * (G + 1), 256), 256, 0, s>>>(br_ptr, br_row, nb, G, br_plan);
  return post(launches);
}

}  // namespace pcdn
