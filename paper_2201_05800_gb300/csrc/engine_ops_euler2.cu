// Batched engine kernels for the 2D Euler equations.
#include "engine_ops.cuh"

namespace stdg {
cudaError_t eng_physics_euler2(const EngLaunch& L, cudaStream_t st, int prepare) {
  return eng_physics_inst<2, STDG_EULER>(L, st, prepare);
}
cudaError_t eng_probe_euler2(int mode, const OpArgs<double>& a64, const OpArgs<float>& a32, cudaStream_t st) {
  return eng_op_probe_inst<2, STDG_EULER>(mode, a64, a32, st);
}
}  // namespace stdg
