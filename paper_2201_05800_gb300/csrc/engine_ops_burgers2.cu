// Batched engine kernels for 2D Burgers.
#include "engine_ops.cuh"

namespace stdg {
cudaError_t eng_physics_burgers2(const EngLaunch& L, cudaStream_t st) {
  return eng_physics_inst<2, STDG_BURGERS>(L, st);
}
}  // namespace stdg
