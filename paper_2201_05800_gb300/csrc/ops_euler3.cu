// Instantiations of the space-time operator for the 3D Euler equations.
#include "ops_impl.cuh"

namespace stdg {

template <class T>
cudaError_t launch_euler3(int mode, const OpArgs<T>& k, cudaStream_t st) {
  if (k.n == 4 && k.s == 3) return launch_modes<3, STDG_EULER, T, 4, 3, true>(mode, k, st);
  return launch_generic<3, STDG_EULER, T>(mode, k, st);
}

template cudaError_t launch_euler3<double>(int, const OpArgs<double>&, cudaStream_t);
template cudaError_t launch_euler3<float>(int, const OpArgs<float>&, cudaStream_t);

}  // namespace stdg
