// stdg_slab_norm_noalloc: the 2-norm of a device vector without any device
// allocation, for callers that must not allocate (see include/stdg.h).
//
// The same norm as stdg_slab_norm up to FP64 rounding: FP64 squares, per-block
// partial sums and one fixed-order final reduction, but with blocks of 16384
// values and a device square root (stdg_slab_norm blocks differently and takes
// the root on the host).  The per-block partial sums live in a file-scope
// static __device__ array instead of memory owned by a context.
#include <mutex>

#include "stdg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 64;                              // values per thread
constexpr size_t kChunk = (size_t)kThreads * kPerThread;    // values per block (16384)
constexpr int kMaxBlocks = 4096;                            // partial sums in the static array
static_assert((size_t)kMaxBlocks * kChunk == STDG_NORM_NOALLOC_MAX_LEN, "limit in stdg.h");
constexpr int kMaxDevices = 64;

// One partial sum per block; shared by every call on a device (32 KB).
static __device__ __align__(256) double g_norm_partials[kMaxBlocks];

std::mutex g_setup_mu;
double* g_partials_ptr[kMaxDevices] = {};

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
  return t;
}

// Block b writes sum_{i in chunk b} x_i^2 to partials[b]; every slot in [0, nb)
// is overwritten, so nothing has to start at zero.
__global__ void __launch_bounds__(kThreads) partial_kernel(const double* __restrict__ x, size_t len,
                                                           double* __restrict__ partials) {
  const size_t base = (size_t)blockIdx.x * kChunk;
  double acc = 0.0;
#pragma unroll 8
  for (int q = 0; q < kPerThread; ++q) {
    const size_t i = base + (size_t)q * kThreads + threadIdx.x;
    if (i < len) acc = fma(x[i], x[i], acc);
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// out[0] = sqrt(sum_{b < nb} partials[b]) in a fixed order.
__global__ void __launch_bounds__(kThreads) final_kernel(const double* __restrict__ partials, int nb,
                                                         double* __restrict__ out) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) acc += partials[b];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) out[0] = sqrt(t);
}

// Device address of the static partials for the current device, looked up once per device
// and kept: valid in the device's primary context until the device is reset (documented in
// stdg.h; a reset or a caller-made driver context would need a fresh lookup).
stdg_status partials_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return STDG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_norm_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return STDG_ERR_CUDA;
    }
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return STDG_OK;
}

}  // namespace

extern "C" stdg_status stdg_slab_norm_noalloc(const double* x, size_t len, double* out, void* cuda_stream) {
  if (!out || (len > 0 && !x)) return STDG_ERR_INVALID_ARG;
  if (len > STDG_NORM_NOALLOC_MAX_LEN) return STDG_ERR_INVALID_ARG;
  // an error pending from earlier work on this thread belongs to its owner: leave it
  // unconsumed and launch nothing, so that the check after the launches sees only ours
  if (cudaPeekAtLastError() != cudaSuccess) return STDG_ERR_CUDA;
  double* partials = nullptr;
  stdg_status st = partials_for_current_device(&partials);
  if (st != STDG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (int)((len + kChunk - 1) / kChunk);
  if (nb > 0) partial_kernel<<<nb, kThreads, 0, s>>>(x, len, partials);
  final_kernel<<<1, kThreads, 0, s>>>(partials, nb, out);
  if (cudaGetLastError() != cudaSuccess) return STDG_ERR_CUDA;
  return STDG_OK;
}
