// lbm_field_sum_noalloc: FP64 sum and non-finite count of a caller-provided FP32
// device array, with no memory allocation of any kind.
//
// For callers that cannot allocate device memory when they need the sum -- for
// example code that runs under a fixed, pre-planned memory budget, or inside a
// framework that forbids cudaMalloc/cudaFree (and allocating library calls) on its
// hot path.  The two-pass reduction is the same as the one behind lbm_reduce, but
// its per-block partial sums live in a file-scope __device__ array instead of memory
// the context allocated.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kThreads = 256;
// Fixed number of partial blocks: the reduction grid-strides over the input, so the
// scratch size does not depend on n.
constexpr int kParts = 1024;
constexpr int kMaxDevices = 64;

// Scratch: kParts (sum, non-finite count) pairs.  16 KiB per device, held by every GPU
// that loads the library until the process exits.  Shared by all calls on a device.
static __device__ __align__(256) double g_sum_scratch[2 * kParts];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_sum_scratch on the current device, looked up once per device.
// In host code the symbol is only a stand-in, so it is never passed to a kernel.
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sum_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Pass 1: block b accumulates elements b*256 + t, striding by the grid, in FP64, then
// folds its threads in a fixed order into scratch[2b] (sum) and scratch[2b + 1]
// (non-finite count).  Every pair a call reads is written earlier in the same call.
// The index is 64-bit: for n up to 2^31 - 1 the last stride (up to kParts * kThreads =
// 2^18) would pass INT_MAX, so i stays below n + 2^18 < 2^32 without overflow.
__global__ void __launch_bounds__(kThreads) k_sum_partial(const float* __restrict__ x, long long n,
                                                          double* __restrict__ scratch) {
  double sum = 0.0, bad = 0.0;
  const long long stride = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = static_cast<long long>(blockIdx.x) * kThreads + threadIdx.x; i < n; i += stride) {
    const float v = x[i];
    sum += v;
    if (!isfinite(v)) bad += 1.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_down_sync(0xffffffffu, sum, o);
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  __shared__ double sh[2][kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = sum;
    sh[1][threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += sh[threadIdx.x][w];
    scratch[2 * blockIdx.x + threadIdx.x] = v;
  }
}

// Pass 2: one block folds `parts` pairs in a fixed order into out[0], out[1].
__global__ void __launch_bounds__(kThreads) k_sum_final(const double* __restrict__ scratch,
                                                        int parts, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  for (int k = 0; k < 2; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < parts; b += kThreads) v += scratch[2 * b + k];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

}  // namespace

extern "C" lbm_status lbm_field_sum_noalloc(const float* field, long long n, double* out,
                                            void* cuda_stream) {
  if (!out) {
    lbm::set_global_error("lbm_field_sum_noalloc: out must not be NULL");
    return LBM_EINVAL;
  }
  if (n < 0 || n > INT_MAX) {
    lbm::set_global_error("lbm_field_sum_noalloc: n = " + std::to_string(n) +
                          " is outside [0, 2^31 - 1]");
    return LBM_EINVAL;
  }
  if (n > 0 && !field) {
    lbm::set_global_error("lbm_field_sum_noalloc: field must not be NULL");
    return LBM_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) {
    lbm::set_global_error(std::string("lbm_field_sum_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = static_cast<int>((n + kThreads - 1) / kThreads);
  const int parts = blocks < 1 ? 1 : (blocks < kParts ? blocks : kParts);
  k_sum_partial<<<parts, kThreads, 0, st>>>(field, n, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_sum_final<<<1, kThreads, 0, st>>>(scratch, parts, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    lbm::set_global_error(std::string("lbm_field_sum_noalloc: launch: ") + cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}
