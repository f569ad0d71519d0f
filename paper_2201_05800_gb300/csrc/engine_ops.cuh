// Physics-dependent kernels of the batched engine (engine.cuh): point-block
// build and the two space-time operator passes (FP64 residual, FP32 exact
// Jacobian-vector product), each walking the engine's work-item lists.
#pragma once

#include <type_traits>

#include "engine.cuh"
#include "operator.cuh"
#include "precond.cuh"

namespace stdg {

template <class T> __device__ __forceinline__ const OpArgs<T>* eng_args(const EngLaunch& L, int slot);
template <> __device__ __forceinline__ const OpArgs<double>* eng_args<double>(const EngLaunch& L, int slot) {
  return L.a64 + slot;
}
template <> __device__ __forceinline__ const OpArgs<float>* eng_args<float>(const EngLaunch& L, int slot) {
  return L.a32 + slot;
}

// Operator tiles of the slots in phase `want`; the slot's arguments are copied
// to shared memory first (they change from tick to tick).
template <int DIM, int EQ, class T, int MODE>
__global__ void __launch_bounds__(256) eng_op_kernel(const __grid_constant__ EngLaunch L, int want) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) OpArgs<T> ks;
  static_assert(sizeof(OpArgs<T>) % 4 == 0, "OpArgs copied as 32-bit words");
  const int n = *L.n_op_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const EngItem item = L.op_items[it];
    const SlotBuf& sb = L.buf[item.slot];
    const OpArgs<T>* ga = eng_args<T>(L, item.slot);
    // a slot in another phase (or past this precision's tile count: one item list serves both
    // precisions) has nothing more for this block: step past the slot's tiles at once
    if (L.ctl[item.slot].phase != want || !eng_runs(L, sb) || (long long)item.idx * ga->epb >= ga->nelem) {
      it += (sb.op0 + sb.nop - it - 1) / (int)gridDim.x * (int)gridDim.x;
      continue;
    }
    const unsigned* src = reinterpret_cast<const unsigned*>(ga);
    unsigned* dst = reinterpret_cast<unsigned*>(&ks);
    for (int i = threadIdx.x; i < (int)(sizeof(OpArgs<T>) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    st_operator_tile<DIM, EQ, T, MODE, kMaxN, kMaxS, false>(ks, item.idx, smem_raw);
  }
}

template <int DIM, int EQ>
__global__ void __launch_bounds__(128) eng_build_kernel(const __grid_constant__ EngLaunch L) {
  const int n = *L.n_chunk_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const EngItem item = L.chunk_items[it];
    if (L.ctl[item.slot].phase != kPhResid) continue;
    const SlotBuf& b = L.buf[item.slot];
    if (!eng_runs(L, b) || b.kron || b.fdm) continue;
    const long long e0 = (long long)item.idx * b.chunk_elems;
    const long long e1 = e0 + b.chunk_elems < b.nelem ? e0 + b.chunk_elems : b.nelem;
    if (b.pbtm) continue;  // temporal-mass scaling: applied directly by the update kernel
    for (long long idx = e0 * b.nd + threadIdx.x; idx < e1 * b.nd; idx += blockDim.x)
      pb_build_node<DIM, EQ, float, float>(L.a32[item.slot], b.U, b.Pinv, idx);
  }
}

template <class K>
inline cudaError_t eng_smem_attr(K kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// prepare = 1: only set the shared-memory attributes of the op kernels and report their
// resident blocks per SM at those sizes in L.occ (outside any stream capture); prepare = 0:
// launch build, residual and Jv kernels of one tick.
template <int DIM, int EQ>
cudaError_t eng_physics_inst(const EngLaunch& L, cudaStream_t st, int prepare) {
  auto k64 = eng_op_kernel<DIM, EQ, double, kModeResidual>;
  auto k32 = eng_op_kernel<DIM, EQ, float, kModeJvExact>;
  if (prepare) {
    cudaError_t e = eng_smem_attr(k64, L.op_smem64);
    if (e != cudaSuccess) return e;
    e = eng_smem_attr(k32, L.op_smem32);
    if (e != cudaSuccess || !L.occ) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.occ[0], k64, 256, L.op_smem64);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.occ[1], k32, 256, L.op_smem32);
  }
  if (L.n_active <= 0) return cudaSuccess;
  eng_build_kernel<DIM, EQ><<<L.chunk_grid, 128, 0, st>>>(L);
  k64<<<L.op_grid64, 256, L.op_smem64, st>>>(L, kPhResid);
  k32<<<L.op_grid32, 256, L.op_smem32, st>>>(L, kPhArnoldi);
  return cudaGetLastError();
}

// One launch of an op kernel alone on a slot with the given epb (autotuning): mode 0 the
// FP64 residual, 1 the FP32 Jv, with the slot's arguments overridden by `a64` / `a32`.
template <int DIM, int EQ>
cudaError_t eng_op_probe_inst(int mode, const OpArgs<double>& a64, const OpArgs<float>& a32, cudaStream_t st) {
  if (mode == 0) {
    auto kern = st_operator_kernel<DIM, EQ, double, kModeResidual, kMaxN, kMaxS, false>;
    const size_t smem = op_smem_bytes<DIM, Phys<EQ, DIM>::R, double, kModeResidual>(a64.n, a64.s, a64.epb);
    cudaError_t e = eng_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((a64.nelem + a64.epb - 1) / a64.epb), 256, smem, st>>>(a64);
  } else {
    auto kern = st_operator_kernel<DIM, EQ, float, kModeJvExact, kMaxN, kMaxS, false>;
    const size_t smem = op_smem_bytes<DIM, Phys<EQ, DIM>::R, float, kModeJvExact>(a32.n, a32.s, a32.epb);
    cudaError_t e = eng_smem_attr(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((a32.nelem + a32.epb - 1) / a32.epb), 256, smem, st>>>(a32);
  }
  return cudaGetLastError();
}

cudaError_t eng_physics_euler2(const EngLaunch& L, cudaStream_t st, int prepare);
cudaError_t eng_physics_burgers2(const EngLaunch& L, cudaStream_t st, int prepare);
cudaError_t eng_physics_advection(int dim, const EngLaunch& L, cudaStream_t st, int prepare);
cudaError_t eng_probe_euler2(int mode, const OpArgs<double>& a64, const OpArgs<float>& a32, cudaStream_t st);
cudaError_t eng_probe_burgers2(int mode, const OpArgs<double>& a64, const OpArgs<float>& a32, cudaStream_t st);
cudaError_t eng_probe_advection(int dim, int mode, const OpArgs<double>& a64, const OpArgs<float>& a32,
                                cudaStream_t st);

}  // namespace stdg
