// Vector kernels of the Newton-GMRES slab solver: batched dot products for
// Gram-Schmidt (V^T w, with |w|^2 when w is the last row), the update
// w -= sum_i c_i V_i with the coefficients passed by value, and slab
// utilities.
//
// Reductions are deterministic: a fixed grid (independent of the vector
// length) writes per-block partial sums in a fixed order, and a second kernel
// sums the partials in a fixed tree.  FP64 accumulation throughout.  The dot
// kernel is instantiated for every row count 1..kMaxDots so that no FP64
// instruction is issued for an absent row (predicated-off FP64 instructions
// still occupy the FP64 pipe).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace stdg {

constexpr int kRedThreads = 256;
constexpr int kMaxDots = 32;        // rows per dot pass (Krylov basis + the new vector)
constexpr int kPartialStride = 40;  // doubles per block in the partials buffer (>= kMaxDots)

// Coefficients of an update, passed by value in the kernel parameters.
struct Coefs {
  double c[kMaxDots];
};

// partials[b*kPartialStride + i] = sum over block b of V_i . w   (i < k <= kMaxDots), for the
// blocks b < *used (at most nblk: one wave of the resident blocks of this row count).
template <class TV, class TW>
cudaError_t multidot(const TV* V, size_t ld, int k, const TW* w, size_t L, double* partials, int nblk,
                     cudaStream_t st, int* used);

// w -= sum_{i<k} c.c[i] V_i   (k <= kMaxDots)
template <class TV, class TW>
cudaError_t update(TW* w, const TV* V, size_t ld, int k, const Coefs& c, size_t L, cudaStream_t st);

// out[i] = sum_b partials[b*kPartialStride + i] for i < count (one block per output).
cudaError_t reduce_partials(const double* partials, int nblk, int count, double* out, cudaStream_t st);

// y = a * x (+ b * z if z); y may alias x or z
template <class TX, class TY>
cudaError_t scale_add(TY* y, const TX* x, double a, const TX* z, double b, size_t L, cudaStream_t st);

// Per temporal node weights of a slab, passed by value.
struct TimeWeights {
  double w[8];
};
// y[e][m][q] = a * w[m] * x[e][m][q] (+ b * z[e][m][q] if z); y may alias x or z
template <class T>
cudaError_t tnode_scale_add(T* y, const T* x, double a, const TimeWeights& w, const T* z, double b,
                            long long nelem, int s, int per_node_block, cudaStream_t st);

// Method-of-lines (Lobatto IIIC) stage residual from F(U), per value q of a node block:
//   form 0:  R_m = U_m - u^n - dt sum_j A[m][j] F_j            (Eq. DG_vs_RK:RK)
//   form 1:  R_m = sum_j Ainv[m][j] (U_j - u^n) / dt - F_m     (the A^-1 form, Eq. Jacobian_Ainv)
struct StageMatrix {
  double a[8][8];
};
cudaError_t lodg_combine(double* R, const double* U, const double* F, const double* u_prev, const StageMatrix& A,
                         double dt, int form, long long nelem, int s, int per_node_block, cudaStream_t st);

// Y[e][m][:] = sum_j E[m][j] X[e][j][:]: a temporal-node mix (E s x s) applied to every
// element and spatial node; Y and X must not overlap
cudaError_t temporal_mix(double* Y, const double* X, const StageMatrix& E, long long nelem, int s, int per_node_block,
                         cudaStream_t st);

// U[e][m][:] = u[e][:] for all m (initial guess 1 (x) u^n)
template <class T>
cudaError_t broadcast_slab(T* U, const T* u, long long nelem, int s, int per_node_block, cudaStream_t st);
// u[e][:] = U[e][s-1][:]
template <class T>
cudaError_t extract_last(T* u, const T* U, long long nelem, int s, int per_node_block, cudaStream_t st);

}  // namespace stdg
