// Objective F(w) for callers that cannot allocate device memory.
//
// Some hosts of this library own every byte of device memory themselves: an application that
// hands all GPU memory to its own pool or budget and forbids libraries from calling cudaMalloc
// behind its back, or a latency-bound serving loop that allows no allocator calls (which may
// synchronise the device) on its request path.  pcdn_objective_noalloc serves them: it takes
// the caller's device buffers for X, y, w and the result, and keeps its own scratch -- z = Xw
// and two arrays of per-block partial sums -- in one file-scope __device__ array of fixed size,
// which every GPU that loads this library holds until the process exits.
//
// The first call on a device looks up that array's device address with cudaGetSymbolAddress
// (the name is only a host-side stand-in; passing it to a kernel would be wrong) and remembers
// it for later calls on that device.  With CUDA's lazy module loading (the default), that first
// call is also when the library's module is loaded on the device and the array is placed there:
// the one allocation this entry point ever causes happens then, so a caller that may not allocate
// on its request path makes one call at set-up (outside any stream capture).  A cudaDeviceReset
// discards the array and the remembered address; after a reset, call pcdn_objective_noalloc only
// after reloading the library.  Every call shares the one array: z is cleared at the start of each
// call, and calls that overlap on the GPU (on different streams, or from several host threads
// without ordering) race on it.
//
// The paper has no counterpart to this entry point.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "pcdn.h"

namespace pcdn {
void set_last_error(const char* msg);  // pcdn_api.cu: the message pcdn_last_error() returns
}  // namespace pcdn

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocBlocks = 512;

// [0, PCDN_NOALLOC_MAX_SAMPLES): z;  then kNoallocBlocks loss partials, kNoallocBlocks |w| partials,
// and one flag word (a row index outside [0, n_samples) was met).
constexpr int64_t kScratchDoubles = PCDN_NOALLOC_MAX_SAMPLES + 2 * kNoallocBlocks + 1;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

int noalloc_fail(int code, const char* msg) {
  pcdn::set_last_error(msg);
  return code;
}

__global__ void noalloc_zero(double* z, int64_t n, double* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0.0;
}

// z = X w over the columns with w_j != 0 (one warp per column).  Every column's range is clamped to
// [0, nnz): a column pointer outside it, or one that decreases, sets the flag instead of being read
// past the arrays.
__global__ void noalloc_xw(const int64_t* col_ptr, const int32_t* row_idx, const float* val, const double* w, int64_t n,
                           int64_t m, int64_t nnz, double* z, double* flag) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; j < m; j += warps) {
    const double wj = w[j];
    if (wj == 0.0) continue;
    int64_t a = col_ptr[j], b = col_ptr[j + 1];
    if (a < 0 || b > nnz || b < a) {
      if (lane == 0) *flag = 1.0;
      a = a < 0 ? 0 : (a > nnz ? nnz : a);
      b = b < a ? a : (b > nnz ? nnz : b);
    }
    for (int64_t e = a + lane; e < b; e += 32) {
      const int32_t r = row_idx[e];
      if (r < 0 || r >= n) {
        *flag = 1.0;
        continue;
      }
      atomicAdd(z + r, (double)val[e] * wj);
    }
  }
}

// per-block sums of the losses phi(z_i) (Eq. 2 or Eq. 3) and of |w_j|, each in a fixed order; a
// label other than +1 or -1 sets the flag
__global__ void noalloc_partials(const double* z, const int8_t* y, int64_t n, int loss, const double* w, int64_t m,
                                 double* part_loss, double* part_w, double* flag) {
  __shared__ double red[kNoallocThreads];
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kNoallocThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kNoallocThreads) {
    if (y[i] != 1 && y[i] != -1) *flag = 1.0;
    const double yz = (double)y[i] * z[i];
    if (loss == PCDN_LOSS_LOGISTIC) a += yz > 0 ? log1p(exp(-yz)) : (-yz + log1p(exp(yz)));
    else a += (1.0 - yz) > 0 ? (1.0 - yz) * (1.0 - yz) : 0.0;
  }
  for (int64_t j = (int64_t)blockIdx.x * kNoallocThreads + threadIdx.x; j < m; j += (int64_t)gridDim.x * kNoallocThreads)
    b += fabs(w[j]);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part_loss[blockIdx.x] = red[0];
  __syncthreads();
  red[threadIdx.x] = b;
  __syncthreads();
  for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part_w[blockIdx.x] = red[0];
}

// F = C * sum(part_loss) + sum(part_w); NaN when the flag is set
__global__ void noalloc_finish(const double* part_loss, const double* part_w, int nb, double C, const double* flag,
                               double* F) {
  __shared__ double red[kNoallocThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += kNoallocThreads) {
    a += part_loss[i];
    b += part_w[i];
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double ta = red[0];
  __syncthreads();
  red[threadIdx.x] = b;
  __syncthreads();
  for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *F = (*flag != 0.0) ? nan("") : C * ta + red[0];
}

// Device address of the scratch array on the current device (looked up once per device).
int scratch_on_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(PCDN_ECUDA, "no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(PCDN_ECUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(PCDN_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PCDN_OK;
}

}  // namespace

extern "C" int pcdn_objective_noalloc(const pcdn_csc* X, const int8_t* y, double C, pcdn_loss loss, const double* w,
                                      double* F, void* stream) {
  pcdn::set_last_error("");
  if (!X || !y || !w || !F || !X->col_ptr || (X->nnz > 0 && (!X->row_idx || !X->val)))
    return noalloc_fail(PCDN_EINVAL, "X (with its arrays), y, w and F must be given");
  if (X->n_samples <= 0 || X->n_features <= 0 || X->nnz < 0)
    return noalloc_fail(PCDN_EINVAL, "n_samples and n_features must be positive, nnz >= 0");
  if (X->n_samples > PCDN_NOALLOC_MAX_SAMPLES)
    return noalloc_fail(PCDN_EINVAL, "n_samples exceeds PCDN_NOALLOC_MAX_SAMPLES (262144), the size of the "
                                     "fixed scratch array of pcdn_objective_noalloc");
  if (!(C > 0) || !std::isfinite(C)) return noalloc_fail(PCDN_EINVAL, "C must be positive and finite");
  if (loss != PCDN_LOSS_LOGISTIC && loss != PCDN_LOSS_L2SVM) return noalloc_fail(PCDN_EINVAL, "unknown loss");
  double* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  double* z = scratch;
  double* part_loss = scratch + PCDN_NOALLOC_MAX_SAMPLES;
  double* part_w = part_loss + kNoallocBlocks;
  double* flag = part_w + kNoallocBlocks;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = X->n_samples, m = X->n_features;
  int gz = (int)((n + kNoallocThreads - 1) / kNoallocThreads);
  if (gz > kNoallocBlocks) gz = kNoallocBlocks;
  noalloc_zero<<<gz, kNoallocThreads, 0, s>>>(z, n, flag);
  int gx = (int)((m * 32 + kNoallocThreads - 1) / kNoallocThreads);
  if (gx > 4096) gx = 4096;
  noalloc_xw<<<gx, kNoallocThreads, 0, s>>>(X->col_ptr, X->row_idx, X->val, w, n, m, X->nnz, z, flag);
  noalloc_partials<<<kNoallocBlocks, kNoallocThreads, 0, s>>>(z, y, n, (int)loss, w, m, part_loss, part_w, flag);
  noalloc_finish<<<1, kNoallocThreads, 0, s>>>(part_loss, part_w, kNoallocBlocks, C, flag, F);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(PCDN_ECUDA, cudaGetErrorString(e));
  return PCDN_OK;
}
