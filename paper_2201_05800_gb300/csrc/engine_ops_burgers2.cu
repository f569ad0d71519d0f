// Batched engine kernels for 2D Burgers.
#include "engine_ops.cuh"

namespace stdg {
cudaError_t eng_physics_burgers2(const EngLaunch& L, cudaStream_t st, int prepare) {
  return eng_physics_inst<2, STDG_BURGERS>(L, st, prepare);
}
cudaError_t eng_probe_burgers2(int mode, const OpArgs<double>& a64, const OpArgs<float>& a32, cudaStream_t st) {
  return eng_op_probe_inst<2, STDG_BURGERS>(mode, a64, a32, st);
}
}  // namespace stdg
