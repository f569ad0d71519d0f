// Batched engine kernels for the 2D Euler equations.
#include "engine_ops.cuh"

namespace stdg {
cudaError_t eng_physics_euler2(const EngLaunch& L, cudaStream_t st) { return eng_physics_inst<2, STDG_EULER>(L, st); }
}  // namespace stdg
