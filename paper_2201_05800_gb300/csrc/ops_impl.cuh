// Launch helpers shared by the per-equation instantiation units.
#pragma once

#include "operator.cuh"
#include "ops.h"

namespace stdg {

template <int DIM, int EQ, class T, int MODE, int NPX, int NTX, bool FIXED>
cudaError_t launch_inst(const OpArgs<T>& k, cudaStream_t st) {
  auto kern = st_operator_kernel<DIM, EQ, T, MODE, NPX, NTX, FIXED>;
  constexpr int R = Phys<EQ, DIM>::R;
  const size_t smem = op_smem_bytes<DIM, R, T, MODE>(k.n, k.s, k.epb);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int threads = k.epb * k.nd;
  if (threads > 256) threads = 256;
  threads = (threads + 31) / 32 * 32;
  const long long blocks = (k.nelem + k.epb - 1) / k.epb * (k.msplit > 1 ? k.msplit : 1);
  kern<<<(unsigned)blocks, threads, smem, st>>>(k);
  return cudaGetLastError();
}

template <int DIM, int EQ, class T, int NPX, int NTX, bool FIXED>
cudaError_t launch_modes(int mode, const OpArgs<T>& k, cudaStream_t st) {
  switch (mode) {
    case kModeResidual: return launch_inst<DIM, EQ, T, kModeResidual, NPX, NTX, FIXED>(k, st);
    case kModeJvFD: return launch_inst<DIM, EQ, T, kModeJvFD, NPX, NTX, FIXED>(k, st);
    case kModeJvExact: return launch_inst<DIM, EQ, T, kModeJvExact, NPX, NTX, FIXED>(k, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int DIM, int EQ, class T>
cudaError_t launch_generic(int mode, const OpArgs<T>& k, cudaStream_t st) {
  if (k.n > kMaxN || k.s > kMaxS || k.n < 2 || k.s < 2) return cudaErrorInvalidValue;
  return launch_modes<DIM, EQ, T, kMaxN, kMaxS, false>(mode, k, st);
}

}  // namespace stdg
