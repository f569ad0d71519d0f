// Dispatch of the fused space-time operator kernel over (dimension, equation,
// mode, precision, n, s).  Hot (n, s) combinations have fully specialised
// instantiations; every other combination runs the runtime-sized kernel
// (n <= 8, s <= 5).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace stdg {

template <class T> cudaError_t launch_advection(int dim, int mode, const OpArgs<T>& k, cudaStream_t st);
template <class T> cudaError_t launch_burgers(int dim, int mode, const OpArgs<T>& k, cudaStream_t st);
template <class T> cudaError_t launch_euler1(int mode, const OpArgs<T>& k, cudaStream_t st);
template <class T> cudaError_t launch_euler2(int mode, const OpArgs<T>& k, cudaStream_t st);
template <class T> cudaError_t launch_euler3(int mode, const OpArgs<T>& k, cudaStream_t st);
// Tangent-only FP32 exact J v for the specialised Euler shapes (jv_tangent.cu); *handled = false
// when the shape or the alignment is not covered (nothing launched).
cudaError_t launch_jv_tangent(int dim, int eq, const OpArgs<float>& k, cudaStream_t st, bool* handled,
                              bool tensor_cores = false);

// Shared memory of one CTA (must match op_smem_bytes in operator.cuh).
inline size_t operator_smem_bytes(int dim, int r, size_t tsize, int mode, int n, int s, int epb) {
  int nd = 1;
  for (int a = 0; a < dim; ++a) nd *= n;
  size_t ndp = (size_t)(nd | 1);
  (void)s;
  size_t vbytes = mode == kModeJvExact ? 2 * tsize : tsize;
  size_t b = (size_t)epb * r * ndp * tsize;
  if (mode == kModeJvExact) b += (size_t)epb * r * ndp * tsize;
  b += (size_t)epb * dim * r * ndp * vbytes;
  b += (size_t)epb * r * ndp * vbytes;
  b += (size_t)epb * dim * ndp * vbytes;
  b += (size_t)(3 * kMaxN * kMaxN + kMaxS * kMaxS) * tsize;
  if (r == 1) {  // viscous term of the scalar equations: gradients and face jumps
    b += (size_t)epb * dim * ndp * vbytes;
    b += (size_t)epb * dim * 2 * (nd / n) * vbytes;
  }
  b += (size_t)epb * dim * 2 * sizeof(int);  // neighbour elements of the tile
  return b;
}

template <class T>
inline cudaError_t launch_operator(int dim, int eq, int mode, const OpArgs<T>& k, cudaStream_t st) {
  switch (eq) {
    case STDG_ADVECTION: return launch_advection<T>(dim, mode, k, st);
    case STDG_BURGERS: return launch_burgers<T>(dim, mode, k, st);
    case STDG_EULER:
      if (dim == 1) return launch_euler1<T>(mode, k, st);
      if (dim == 2) return launch_euler2<T>(mode, k, st);
      if (dim == 3) return launch_euler3<T>(mode, k, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stdg
