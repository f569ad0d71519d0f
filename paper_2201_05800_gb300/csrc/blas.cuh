// Vector kernels of the Newton-GMRES slab solver: batched dot products for
// Gram-Schmidt (V^T w), the fused update w -= V c (with the dots of the
// updated w against V and its squared norm, so that the classical
// Gram-Schmidt re-orthogonalisation pass costs no extra read), linear
// combinations x += V y, and slab utilities.
//
// Reductions are deterministic: a fixed grid (independent of the vector
// length) writes per-block partial sums in a fixed order, and a second kernel
// sums the partials in a fixed tree.  FP64 accumulation throughout.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace stdg {

constexpr int kRedThreads = 256;
constexpr int kMaxDots = 32;   // dot products per pass held in registers
constexpr int kPartialStride = 72;  // doubles per block in the partials buffer (>= kMaxDots+1, x8 aligned)

// partials[b*kPartialStride + i] = sum over block b of scale(V_i) . w (i < k <= kMaxDots)
template <class TV, class TW>
cudaError_t multidot(const TV* V, size_t ld, int k, const TW* w, size_t L, double* partials, int nblk,
                     cudaStream_t st);

// w -= sum_i coef[i] V_i (i < k); if dots: partials also receive V_i . w_new (i < k) and
// |w_new|^2 at index k; else only |w_new|^2 at index 0 when norm is set.
template <class TV, class TW>
cudaError_t update(TW* w, const TV* V, size_t ld, int k, const double* coef, double coef_sign, size_t L,
                   double* partials, int nblk, bool dots, bool norm, cudaStream_t st);

// out[i] = sum_b partials[b*kPartialStride + i] for i < count (one block per output).
cudaError_t reduce_partials(const double* partials, int nblk, int count, double* out, cudaStream_t st);

// y = a * x (+ b * z if z)
template <class TX, class TY>
cudaError_t scale_add(TY* y, const TX* x, double a, const TX* z, double b, size_t L, cudaStream_t st);

// U[e][m][:] = u[e][:] for all m (initial guess 1 (x) u^n)
template <class T>
cudaError_t broadcast_slab(T* U, const T* u, long long nelem, int s, int per_node_block, cudaStream_t st);
// u[e][:] = U[e][s-1][:]
template <class T>
cudaError_t extract_last(T* u, const T* U, long long nelem, int s, int per_node_block, cudaStream_t st);

}  // namespace stdg
