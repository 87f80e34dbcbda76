// Host-side launchers of the preparation, refresh and reduction kernels (pcdn_prep.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pcdn_internal.cuh"

namespace pcdn {

// ---- scan --------------------------------------------------------------------------------
// Exclusive prefix sum of n int64 values (in-place allowed).  Workspace from scan_workspace().
int64_t scan_workspace_elems(int64_t n);
cudaError_t scan_exclusive(const int64_t* in, int64_t* out, int64_t n, int64_t* ws, cudaStream_t s, int64_t* launches);

// ---- stable LSD radix sort of (key, value) pairs, 8-bit digits ------------------------------
// Sorts the low `key_bits` bits; result in (*k_out, *v_out), which point at either the input or
// the alternate buffers.  hist must hold radix_hist_elems(n) int64; ws scan_workspace_elems(that).
int64_t radix_hist_elems(int64_t n);
cudaError_t radix_sort_u64(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int64_t n, int key_bits,
                           int64_t* hist, int64_t* ws, uint64_t** k_out, int32_t** v_out, cudaStream_t s,
                           int64_t* launches);
cudaError_t radix_sort_u32(uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int64_t n, int key_bits,
                           int64_t* hist, int64_t* ws, uint32_t** k_out, int32_t** v_out, cudaStream_t s,
                           int64_t* launches);

// ---- partition of one outer iteration (Eq. 8) ------------------------------------------------
// perm_keys: key_j = splitmix64 output j+1 of the stream of (seed, epoch); values j.  With
// epoch_dev (device, may be NULL) the epoch is epoch + the value read there when the kernel runs.
cudaError_t perm_keys(uint64_t seed, int64_t epoch, const int64_t* epoch_dev, int64_t m, uint64_t* keys, int32_t* vals,
                      cudaStream_t s, int64_t* launches);
// *epoch_dev += 1 (one thread)
cudaError_t advance_epoch(int64_t* epoch_dev, cudaStream_t s, int64_t* launches);

// ---- column work items ------------------------------------------------------------------------
// For positions [0, npos) of `perm`: item_ptr[npos+1] and items[] (chunks of <= kChunk nonzeros),
// each carrying its feature's current weight (w may be NULL: 0).
cudaError_t build_items(const int32_t* perm, int64_t npos, const int64_t* col_ptr, const double* w, int64_t* cnt_ws,
                        int64_t* item_ptr, Item* items, int64_t* scan_ws, cudaStream_t s, int64_t* launches);

// Block plan of a walk: item_off = exclusive prefix of item lengths over [0, n_items] (n_items
// may exceed the walk's real count item_ptr[npos]; the excess counts as empty); for bundle t and
// block c in [0, G], plan[t*(G+1)+c] = first item of block c (nonzeros balanced over blocks;
// an item never splits between blocks).
cudaError_t build_plan(const Item* items, int64_t n_items, const int64_t* item_ptr, int64_t npos, int32_t P, int64_t nb,
                       int G, int64_t* len_ws, int64_t* item_off, int64_t* plan, int64_t* scan_ws, cudaStream_t s,
                       int64_t* launches);
// w in position order for a walk, and back.
cudaError_t gather_w(const double* w, const int32_t* perm, int64_t npos, double* w_pos, cudaStream_t s, int64_t* launches);
cudaError_t scatter_w(const double* w_pos, const int32_t* perm, int64_t npos, double* w, cudaStream_t s, int64_t* launches);

// ---- row-major mirror (pcdn_mirror.cu) ---------------------------------------------------------
// Column of every CSC entry (bounded by m for any col_ptr).
cudaError_t entry_columns(const int64_t* col_ptr, int64_t m, int64_t nnz, int32_t* entry_col, cudaStream_t s,
                          int64_t* launches);
cudaError_t iota_i32(int32_t* v, int64_t n, cudaStream_t s, int64_t* launches);
// Entries per row into counts[0..n) (zeroed by the caller); indexes outside [0, n) are skipped.
cudaError_t mirror_row_counts(const int32_t* row_idx, int64_t nnz, int64_t n, int64_t* counts, cudaStream_t s,
                              int64_t* launches);
struct MirrorSizes {
  int passes;      // counting-sort passes (digits of at most 10 bits)
  int64_t tiles;   // tiles of 4096 entries
  int64_t hist;    // histogram elements per pass
  int tmp_row;     // 1: a row array of nnz entries (three passes)
  int tmp_triple;  // 1: a (row, col, val) triple of nnz entries (two or three passes)
};
MirrorSizes mirror_sizes(int64_t n, int64_t nnz);
struct MirrorWorkspace {
  int64_t* hist;     // [hist]
  int64_t* off;      // [hist]
  int64_t* scan_ws;  // [scan_workspace_elems(hist)]
  int32_t* row0;     // [nnz] if tmp_row
  int32_t* trow;     // [nnz] each if tmp_triple
  int32_t* tcol;
  float* tval;
};
cudaError_t mirror_configure();
// col_idx/rval[nnz]: the entries (row_idx, entry_col, val) stably sorted by row.  Writes stay inside
// the arrays for any row index (malformed input gives a wrong order, never a stray write).
cudaError_t build_mirror(const int32_t* row_idx, const int32_t* entry_col, const float* val, int64_t nnz, int64_t n,
                         const MirrorWorkspace& ws, int32_t* col_idx, float* rval, cudaStream_t s, int64_t* launches);

// ---- row-sorted bundle layout (pcdn_rows.cu) ---------------------------------------------------
// Row of every entry of the row-major mirror.
cudaError_t entry_rows(const int64_t* row_ptr, int64_t n, int32_t* entry_row, cudaStream_t s, int64_t* launches);
// Bundle counts up to kBins use one counting sort; more use a radix sort.
constexpr int kBins = 1024;
struct RowsWorkspace {
  int32_t* inv;       // [m] position of each feature in the walk, -1 outside it
  int64_t* hist;      // [rows_hist_elems(nnz)] (counting sort)
  int64_t* scan_ws;   // scan workspace for max(rows_hist_elems, radix_hist_elems) elements
  uint32_t* k0;       // radix sort keys and values [nnz] each (only for more than kBins bundles)
  uint32_t* k1;
  int32_t* v0;
  int32_t* v1;
  int64_t* rhist;     // [radix_hist_elems(nnz)]
};
cudaError_t rows_configure();
int64_t rows_tiles(int64_t nnz);
int64_t rows_hist_elems(int64_t nnz);
// The walk's entries by bundle, grouped by row (see pcdn_rows.cu): br_row/br_k/br_val[nnz],
// br_ptr[nb + 1], br_plan[nb * (G + 1)].
cudaError_t build_rows(const int32_t* perm, int64_t npos, int64_t m, int32_t P, int64_t nb, int G,
                       const int32_t* col_idx, const float* rval, const int32_t* entry_row, int64_t nnz,
                       const RowsWorkspace& ws, int32_t* br_row, int32_t* br_k, float* br_val, int64_t* br_ptr,
                       int64_t* br_plan, cudaStream_t s, int64_t* launches);

// ---- validation (device-resident input) -------------------------------------------------------
cudaError_t validate_device(const int64_t* col_ptr, const int32_t* row_idx, const float* val, const int8_t* y,
                            int64_t n, int64_t m, int64_t nnz, int* flag, cudaStream_t s, int64_t* launches);

// ---- maintained quantities --------------------------------------------------------------------
// z = Xw by rows; each sample's maintained quantity and coefficients (SampleRec) from z (write_state),
// optional per-block loss partial sums.
// FP64 (prec 0, or no scratch): one lane per row, separate multiply and add in column order.
// Mixed (prec 1 with w2_scratch, 8 bytes per feature): double-float sums on the FP32 pipe.
cudaError_t refresh(int loss, int prec, const int64_t* row_ptr, const int32_t* col_idx, const float* rval,
                    const int8_t* y, const double* w, int64_t n, int64_t m, int64_t nnz, void* w2_scratch,
                    void* st, bool write_state, double* loss_part, int grid, int* err, cudaStream_t s,
                    int64_t* launches);
// The maintained quantities and coefficients at w = 0 (mq = 1 for both losses), without reading X.
cudaError_t state_at_zero(int loss, int prec, const int8_t* y, int64_t n, void* st, cudaStream_t s, int64_t* launches);
// The coefficients from the current state slot (of precision prec).
cudaError_t rec_from_mq(int loss, int prec, const int8_t* y, int64_t n, void* st, cudaStream_t s, int64_t* launches);
// The state slots converted to precision to_prec's form (FP64: e^z or b; mixed: a double-float pair
// of z or b) and their coefficients (a precision switch without recomputing z = Xw); a margin too
// large for FP64's e^z sets kErrRange in *err.
cudaError_t convert_state(int loss, int to_prec, const int8_t* y, int64_t n, void* st, int* err, cudaStream_t s,
                          int64_t* launches);

// ---- reductions -------------------------------------------------------------------------------
// Minimum-norm subgradient l1 norm from the samples' coefficients, over work items of all columns:
// FP64 mode from the FP64 coefficient pair; mixed mode from the FP64 coefficient recomputed from mq
// and summed in double-float arithmetic (kkt_coef_kernel).
// When g_out / vmax are given (shrinking): g_j of every feature into g_out[j], and the largest
// |v_j| into *vmax (as the bits of the double; *vmax zeroed by the caller).
// l1, l2: the penalty l1 ||w||_1 + (l2/2) ||w||^2 (g is the smooth part's gradient).
cudaError_t kkt_l1(int loss, int prec, const int8_t* y, int64_t n, const Item* items, int64_t n_items,
                   const int64_t* item_ptr, const int32_t* perm, int64_t npos, const int32_t* row_idx, const float* val,
                   void* st, const double* w, double c, double l1, double l2, double* gpart, double* block_part,
                   int grid, double* out, cudaStream_t s, int64_t* launches, double* g_out = nullptr,
                   unsigned long long* vmax = nullptr);

// ---- shrinking (between outer iterations) ------------------------------------------------------
// A feature is active unless w_j = 0 and |g_j| < l1 - M / n_samples, M = *vmax (the largest |v_j|).
// out[0] += active features, out[1] += their nonzeros (out zeroed by the caller).
cudaError_t active_count(const double* g, const double* w, int64_t m, const int64_t* col_ptr,
                         const unsigned long long* vmax, int64_t n_samples, double l1, unsigned long long* out,
                         cudaStream_t s, int64_t* launches);
// The active features of partition perm[0..m), in partition order, into out[0..count) (a stable
// filter; flags_ws and pos_ws hold m + 1 entries each).
cudaError_t compact_active(const int32_t* perm, int64_t m, const double* g, const double* w,
                           const unsigned long long* vmax, int64_t n_samples, double l1, int64_t* flags_ws,
                           int64_t* pos_ws, int64_t* scan_ws, int32_t* out, cudaStream_t s, int64_t* launches);
// out = c * sum(loss_part[0..nb)) + sum_j (l1 |w_j| + (l2/2) w_j^2)
cudaError_t objective_finish(const double* loss_part, int nb, const double* w, int64_t m, double c, double l1,
                             double l2, double* block_part, int grid, double* out, cudaStream_t s,
                             int64_t* launches);

}  // namespace pcdn
