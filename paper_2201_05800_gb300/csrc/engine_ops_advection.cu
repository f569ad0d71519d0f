// Batched engine kernels for linear advection in 1D and 2D.
#include "engine_ops.cuh"

namespace stdg {
cudaError_t eng_physics_advection(int dim, const EngLaunch& L, cudaStream_t st) {
  if (dim == 1) return eng_physics_inst<1, STDG_ADVECTION>(L, st);
  if (dim == 2) return eng_physics_inst<2, STDG_ADVECTION>(L, st);
  return cudaErrorInvalidValue;
}
}  // namespace stdg
