// Vector kernels of the Newton-GMRES slab solver (see blas.cuh).
#include "blas.cuh"
#include "warp_scatter.cuh"

#include <stdint.h>

#include <type_traits>

namespace stdg {

namespace {

// Block-reduce K accumulators (FP64 adds: about K per lane for the warp step) and store
// them at out[0..K).
template <int K>
__device__ __forceinline__ void block_store(const double (&acc)[K], double* out) {
  static_assert(K >= 1 && K <= 32, "at most 32 rows");
  constexpr int KP = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  __shared__ double red[kRedThreads / 32][K];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double a[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) a[i] = i < K ? acc[i] : 0.0;
  int row = 0;
  WarpScatter<KP, 16>::run(a, lane, row);
  if ((lane & (32 / KP - 1)) == 0 && row < K) red[wid][row] = a[0];
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[q][threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// Per-thread arithmetic precision: FP32 data is combined in FP32 (an FP64
// operation per element would make the FP32 passes FP64-pipe bound); FP64
// data in FP64.  Cross-thread sums are always FP64.
template <class TV> struct Compute { using type = double; };
template <> struct Compute<float> { using type = float; };

template <class TV, class TW, int K>
__global__ void __launch_bounds__(kRedThreads) multidot_kernel(const TV* __restrict__ V, size_t ld,
                                                               const TW* __restrict__ w, size_t L,
                                                               double* __restrict__ partials) {
  using CT = typename Compute<TV>::type;
  CT acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = CT(0);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t start = 0;
  if constexpr (std::is_same<TV, float>::value && std::is_same<TW, float>::value) {
    // FP32 rows: 16-byte loads (four values per load) when every row is 16-byte aligned
    if (ld % 4 == 0 && ((uintptr_t)V & 15) == 0 && ((uintptr_t)w & 15) == 0) {
      const size_t L4 = L / 4;
      const float4* w4 = reinterpret_cast<const float4*>(w);
      for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < L4; q += stride) {
        const float4 wv = w4[q];
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const float4 x = reinterpret_cast<const float4*>(V + (size_t)i * ld)[q];
          acc[i] = fmaf(x.w, wv.w, fmaf(x.z, wv.z, fmaf(x.y, wv.y, fmaf(x.x, wv.x, acc[i]))));
        }
      }
      start = L4 * 4;
    }
  }
  for (size_t idx = start + (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < L; idx += stride) {
    const CT wv = (CT)w[idx];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = fma((CT)V[(size_t)i * ld + idx], wv, acc[i]);
  }
  double accd[K];
#pragma unroll
  for (int i = 0; i < K; ++i) accd[i] = (double)acc[i];
  block_store<K>(accd, partials + (size_t)blockIdx.x * kPartialStride);
}

// w -= sum_i c_i V_i; the sum is formed in the basis precision and added to w
// in w's precision (FP32 basis into an FP64 w: one FP64 add per element).
template <class TV, class TW>
__global__ void __launch_bounds__(kRedThreads) update_kernel(TW* __restrict__ w, const TV* __restrict__ V, size_t ld,
                                                             int k, const __grid_constant__ Coefs c, size_t L) {
  using CT = typename Compute<TV>::type;
  using WT = typename Compute<TW>::type;
  __shared__ CT cn[kMaxDots];  // -c in the compute precision, converted once per block
  if (threadIdx.x < kMaxDots) cn[threadIdx.x] = threadIdx.x < k ? (CT)(-c.c[threadIdx.x]) : CT(0);
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t start = 0;
  if constexpr (std::is_same<TV, float>::value && std::is_same<TW, float>::value) {
    // FP32 rows: 16-byte loads and stores when every row is 16-byte aligned
    if (ld % 4 == 0 && ((uintptr_t)V & 15) == 0 && ((uintptr_t)w & 15) == 0) {
      const size_t L4 = L / 4;
      float4* w4 = reinterpret_cast<float4*>(w);
      for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < L4; q += stride) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        int i = 0;
        for (; i + 2 <= k; i += 2) {
          const float4 x = reinterpret_cast<const float4*>(V + (size_t)i * ld)[q];
          const float4 y = reinterpret_cast<const float4*>(V + (size_t)(i + 1) * ld)[q];
          a.x = fmaf(cn[i], x.x, a.x); a.y = fmaf(cn[i], x.y, a.y);
          a.z = fmaf(cn[i], x.z, a.z); a.w = fmaf(cn[i], x.w, a.w);
          b.x = fmaf(cn[i + 1], y.x, b.x); b.y = fmaf(cn[i + 1], y.y, b.y);
          b.z = fmaf(cn[i + 1], y.z, b.z); b.w = fmaf(cn[i + 1], y.w, b.w);
        }
        if (i < k) {
          const float4 x = reinterpret_cast<const float4*>(V + (size_t)i * ld)[q];
          a.x = fmaf(cn[i], x.x, a.x); a.y = fmaf(cn[i], x.y, a.y);
          a.z = fmaf(cn[i], x.z, a.z); a.w = fmaf(cn[i], x.w, a.w);
        }
        float4 o = w4[q];
        o.x += a.x + b.x; o.y += a.y + b.y; o.z += a.z + b.z; o.w += a.w + b.w;
        w4[q] = o;
      }
      start = L4 * 4;
    }
  }
  if constexpr (std::is_same<CT, double>::value && std::is_same<WT, double>::value) {
    // FP64 basis and w: one FMA chain from w (k FMAs per element, no extra adds on the
    // FP64 pipe); four loads issued ahead of their FMAs
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < L; idx += stride) {
      double acc = (double)w[idx];
      int i = 0;
      for (; i + 4 <= k; i += 4) {
        const double v0 = (double)V[(size_t)i * ld + idx], v1 = (double)V[(size_t)(i + 1) * ld + idx];
        const double v2 = (double)V[(size_t)(i + 2) * ld + idx], v3 = (double)V[(size_t)(i + 3) * ld + idx];
        acc = fma(cn[i], v0, acc);
        acc = fma(cn[i + 1], v1, acc);
        acc = fma(cn[i + 2], v2, acc);
        acc = fma(cn[i + 3], v3, acc);
      }
      for (; i < k; ++i) acc = fma(cn[i], (double)V[(size_t)i * ld + idx], acc);
      w[idx] = (TW)acc;
    }
    return;
  }
  for (size_t idx = start + (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < L; idx += stride) {
    CT x0 = CT(0), x1 = CT(0), x2 = CT(0), x3 = CT(0);
    int i = 0;
    for (; i + 4 <= k; i += 4) {
      x0 = fma(cn[i], (CT)V[(size_t)i * ld + idx], x0);
      x1 = fma(cn[i + 1], (CT)V[(size_t)(i + 1) * ld + idx], x1);
      x2 = fma(cn[i + 2], (CT)V[(size_t)(i + 2) * ld + idx], x2);
      x3 = fma(cn[i + 3], (CT)V[(size_t)(i + 3) * ld + idx], x3);
    }
    for (; i < k; ++i) x0 = fma(cn[i], (CT)V[(size_t)i * ld + idx], x0);
    w[idx] = (TW)((WT)w[idx] + (WT)((x0 + x1) + (x2 + x3)));
  }
}

__global__ void reduce_kernel(const double* __restrict__ partials, int nblk, double* __restrict__ out) {
  // one block per output index; fixed-order tree
  __shared__ double sh[kRedThreads];
  const int i = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partials[(size_t)b * kPartialStride + i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = sh[0];
}

template <class TX, class TY>
__global__ void scale_add_kernel(TY* y, const TX* x, double a, const TX* z, double b, size_t L) {
  // y may alias x or z (in-place scaling and updates): no __restrict__ here
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < L; idx += stride) {
    double v = a * (double)x[idx];
    if (z) v = fma(b, (double)z[idx], v);
    y[idx] = (TY)v;
  }
}

template <class T>
__global__ void tnode_scale_add_kernel(T* y, const T* x, double a, const TimeWeights w, const T* z, double b,
                                       long long nelem, int s, int blk) {
  // y may alias x or z: no __restrict__ here
  const size_t total = (size_t)nelem * s * blk;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const int m = (int)((idx / blk) % s);
    double v = a * w.w[m] * (double)x[idx];
    if (z) v = fma(b, (double)z[idx], v);
    y[idx] = (T)v;
  }
}

__global__ void lodg_combine_kernel(double* __restrict__ R, const double* __restrict__ U,
                                    const double* __restrict__ F, const double* __restrict__ u_prev,
                                    const StageMatrix A, double dt, int form, long long nelem, int s, int blk) {
  const size_t total = (size_t)nelem * blk;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double idt = 1.0 / dt;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const size_t e = idx / blk, q = idx % blk;
    const size_t base = e * s * blk + q;
    const double un = u_prev[idx];
    for (int m = 0; m < s; ++m) {
      double acc = 0.0;
      if (form == 0) {
        for (int j = 0; j < s; ++j) acc = fma(A.a[m][j], F[base + (size_t)j * blk], acc);
        R[base + (size_t)m * blk] = (U[base + (size_t)m * blk] - un) - dt * acc;
      } else {
        for (int j = 0; j < s; ++j) acc = fma(A.a[m][j], U[base + (size_t)j * blk] - un, acc);
        R[base + (size_t)m * blk] = acc * idt - F[base + (size_t)m * blk];
      }
    }
  }
}

template <class T>
__global__ void broadcast_kernel(T* __restrict__ U, const T* __restrict__ u, long long nelem, int s, int blk) {
  const size_t total = (size_t)nelem * s * blk;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    size_t e = idx / ((size_t)s * blk);
    size_t q = idx % blk;
    U[idx] = u[e * blk + q];
  }
}

// one thread per (element, value of a temporal node): s reads, s writes, coalesced in the value
__global__ void temporal_mix_kernel(double* __restrict__ Y, const double* __restrict__ X, const StageMatrix E,
                                    long long nelem, int s, int blk) {
  const size_t total = (size_t)nelem * blk;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const size_t e = idx / blk, q = idx % blk;
    const double* x = X + e * s * blk + q;
    double xv[8];
    for (int j = 0; j < s; ++j) xv[j] = x[(size_t)j * blk];
    double* y = Y + e * s * blk + q;
    for (int m = 0; m < s; ++m) {
      double a = 0.0;
      for (int j = 0; j < s; ++j) a = fma(E.a[m][j], xv[j], a);
      y[(size_t)m * blk] = a;
    }
  }
}

template <class T>
__global__ void extract_kernel(T* __restrict__ u, const T* __restrict__ U, long long nelem, int s, int blk) {
  const size_t total = (size_t)nelem * blk;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    size_t e = idx / blk, q = idx % blk;
    u[idx] = U[(e * s + (s - 1)) * blk + q];
  }
}

unsigned grid_for(size_t L) {
  size_t b = (L + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Blocks of the dot pass: one wave (the resident blocks of this row count on every SM), at
// most the partials buffer's nblk rows; cached per instantiation.
template <class TV, class TW, int K>
int multidot_grid(int nblk) {
  static int per_sm = 0;
  static int sms = 0;
  if (per_sm == 0) {
    int dev = 0, occ = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, multidot_kernel<TV, TW, K>, kRedThreads, 0) !=
            cudaSuccess ||
        occ < 1)
      occ = 1;
    sms = n > 0 ? n : 1;
    per_sm = occ;
  }
  const int g = per_sm * sms;
  return g < nblk ? g : nblk;
}

template <class TV, class TW, int K>
cudaError_t multidot_k(const TV* V, size_t ld, const TW* w, size_t L, double* partials, int nblk, cudaStream_t st,
                       int* used) {
  const int g = multidot_grid<TV, TW, K>(nblk);
  multidot_kernel<TV, TW, K><<<g, kRedThreads, 0, st>>>(V, ld, w, L, partials);
  if (used) *used = g;
  return cudaGetLastError();
}

}  // namespace

template <class TV, class TW>
cudaError_t multidot(const TV* V, size_t ld, int k, const TW* w, size_t L, double* partials, int nblk,
                     cudaStream_t st, int* used) {
#define STDG_DOT_CASE(K) \
  case K: return multidot_k<TV, TW, K>(V, ld, w, L, partials, nblk, st, used);
  switch (k) {
    STDG_DOT_CASE(1) STDG_DOT_CASE(2) STDG_DOT_CASE(3) STDG_DOT_CASE(4) STDG_DOT_CASE(5) STDG_DOT_CASE(6)
    STDG_DOT_CASE(7) STDG_DOT_CASE(8) STDG_DOT_CASE(9) STDG_DOT_CASE(10) STDG_DOT_CASE(11) STDG_DOT_CASE(12)
    STDG_DOT_CASE(13) STDG_DOT_CASE(14) STDG_DOT_CASE(15) STDG_DOT_CASE(16) STDG_DOT_CASE(17) STDG_DOT_CASE(18)
    STDG_DOT_CASE(19) STDG_DOT_CASE(20) STDG_DOT_CASE(21) STDG_DOT_CASE(22) STDG_DOT_CASE(23) STDG_DOT_CASE(24)
    STDG_DOT_CASE(25) STDG_DOT_CASE(26) STDG_DOT_CASE(27) STDG_DOT_CASE(28) STDG_DOT_CASE(29) STDG_DOT_CASE(30)
    STDG_DOT_CASE(31) STDG_DOT_CASE(32)
    default: return cudaErrorInvalidValue;
  }
#undef STDG_DOT_CASE
}

template <class TV, class TW>
cudaError_t update(TW* w, const TV* V, size_t ld, int k, const Coefs& c, size_t L, cudaStream_t st) {
  if (k < 1 || k > kMaxDots) return cudaErrorInvalidValue;
  update_kernel<TV, TW><<<grid_for(L), kRedThreads, 0, st>>>(w, V, ld, k, c, L);
  return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partials, int nblk, int count, double* out, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  reduce_kernel<<<count, kRedThreads, 0, st>>>(partials, nblk, out);
  return cudaGetLastError();
}

template <class TX, class TY>
cudaError_t scale_add(TY* y, const TX* x, double a, const TX* z, double b, size_t L, cudaStream_t st) {
  scale_add_kernel<TX, TY><<<grid_for(L), 256, 0, st>>>(y, x, a, z, b, L);
  return cudaGetLastError();
}

template <class T>
cudaError_t tnode_scale_add(T* y, const T* x, double a, const TimeWeights& w, const T* z, double b,
                            long long nelem, int s, int blk, cudaStream_t st) {
  tnode_scale_add_kernel<T><<<grid_for((size_t)nelem * s * blk), 256, 0, st>>>(y, x, a, w, z, b, nelem, s, blk);
  return cudaGetLastError();
}

cudaError_t lodg_combine(double* R, const double* U, const double* F, const double* u_prev, const StageMatrix& A,
                         double dt, int form, long long nelem, int s, int blk, cudaStream_t st) {
  lodg_combine_kernel<<<grid_for((size_t)nelem * blk), 256, 0, st>>>(R, U, F, u_prev, A, dt, form, nelem, s, blk);
  return cudaGetLastError();
}

template <class T>
cudaError_t broadcast_slab(T* U, const T* u, long long nelem, int s, int blk, cudaStream_t st) {
  broadcast_kernel<T><<<grid_for((size_t)nelem * s * blk), 256, 0, st>>>(U, u, nelem, s, blk);
  return cudaGetLastError();
}

cudaError_t temporal_mix(double* Y, const double* X, const StageMatrix& E, long long nelem, int s, int blk,
                         cudaStream_t st) {
  if (s < 1 || s > 8) return cudaErrorInvalidValue;
  temporal_mix_kernel<<<grid_for((size_t)nelem * blk), 256, 0, st>>>(Y, X, E, nelem, s, blk);
  return cudaGetLastError();
}

template <class T>
cudaError_t extract_last(T* u, const T* U, long long nelem, int s, int blk, cudaStream_t st) {
  extract_kernel<T><<<grid_for((size_t)nelem * blk), 256, 0, st>>>(u, U, nelem, s, blk);
  return cudaGetLastError();
}

template cudaError_t multidot<double, double>(const double*, size_t, int, const double*, size_t, double*, int, cudaStream_t,
                                              int*);
template cudaError_t multidot<float, float>(const float*, size_t, int, const float*, size_t, double*, int, cudaStream_t,
                                            int*);
template cudaError_t update<double, double>(double*, const double*, size_t, int, const Coefs&, size_t, cudaStream_t);
template cudaError_t update<float, float>(float*, const float*, size_t, int, const Coefs&, size_t, cudaStream_t);
template cudaError_t update<float, double>(double*, const float*, size_t, int, const Coefs&, size_t, cudaStream_t);
template cudaError_t scale_add<double, double>(double*, const double*, double, const double*, double, size_t, cudaStream_t);
template cudaError_t scale_add<double, float>(float*, const double*, double, const double*, double, size_t, cudaStream_t);
template cudaError_t scale_add<float, float>(float*, const float*, double, const float*, double, size_t, cudaStream_t);
template cudaError_t scale_add<float, double>(double*, const float*, double, const float*, double, size_t, cudaStream_t);
template cudaError_t tnode_scale_add<double>(double*, const double*, double, const TimeWeights&, const double*, double,
                                             long long, int, int, cudaStream_t);
template cudaError_t tnode_scale_add<float>(float*, const float*, double, const TimeWeights&, const float*, double,
                                            long long, int, int, cudaStream_t);
template cudaError_t broadcast_slab<double>(double*, const double*, long long, int, int, cudaStream_t);
template cudaError_t extract_last<double>(double*, const double*, long long, int, int, cudaStream_t);

}  // namespace stdg
