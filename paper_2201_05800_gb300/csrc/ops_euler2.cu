// Instantiations of the space-time operator for the 2D Euler equations.
#include "ops_impl.cuh"

namespace stdg {

template <class T>
cudaError_t launch_euler2(int mode, const OpArgs<T>& k, cudaStream_t st) {
  if (k.n == 5 && k.s == 4) return launch_modes<2, STDG_EULER, T, 5, 4, true>(mode, k, st);
  return launch_generic<2, STDG_EULER, T>(mode, k, st);
}

template cudaError_t launch_euler2<double>(int, const OpArgs<double>&, cudaStream_t);
template cudaError_t launch_euler2<float>(int, const OpArgs<float>&, cudaStream_t);

}  // namespace stdg
