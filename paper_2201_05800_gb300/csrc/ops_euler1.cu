// Instantiations of the space-time operator for the 1D Euler equations.
#include "ops_impl.cuh"

namespace stdg {

template <class T>
cudaError_t launch_euler1(int mode, const OpArgs<T>& k, cudaStream_t st) {

  return launch_generic<1, STDG_EULER, T>(mode, k, st);
}

template cudaError_t launch_euler1<double>(int, const OpArgs<double>&, cudaStream_t);
template cudaError_t launch_euler1<float>(int, const OpArgs<float>&, cudaStream_t);

}  // namespace stdg
