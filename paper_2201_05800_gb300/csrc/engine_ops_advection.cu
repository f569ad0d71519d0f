// Batched engine kernels for linear advection in 1D and 2D.
#include "engine_ops.cuh"

namespace stdg {
cudaError_t eng_physics_advection(int dim, const EngLaunch& L, cudaStream_t st, int prepare) {
  if (dim == 1) return eng_physics_inst<1, STDG_ADVECTION>(L, st, prepare);
  if (dim == 2) return eng_physics_inst<2, STDG_ADVECTION>(L, st, prepare);
  return cudaErrorInvalidValue;
}
cudaError_t eng_probe_advection(int dim, int mode, const OpArgs<double>& a64, const OpArgs<float>& a32,
                                cudaStream_t st) {
  if (dim == 1) return eng_op_probe_inst<1, STDG_ADVECTION>(mode, a64, a32, st);
  if (dim == 2) return eng_op_probe_inst<2, STDG_ADVECTION>(mode, a64, a32, st);
  return cudaErrorInvalidValue;
}
}  // namespace stdg
