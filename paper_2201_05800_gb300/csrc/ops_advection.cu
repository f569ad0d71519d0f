// Instantiations of the space-time operator for linear advection.
#include "ops_impl.cuh"

namespace stdg {

template <class T>
cudaError_t launch_advection(int dim, int mode, const OpArgs<T>& k, cudaStream_t st) {
  switch (dim) {
    case 1:
      if (k.n == 4 && k.s == 3) return launch_modes<1, STDG_ADVECTION, T, 4, 3, true>(mode, k, st);
      return launch_generic<1, STDG_ADVECTION, T>(mode, k, st);
    case 2: return launch_generic<2, STDG_ADVECTION, T>(mode, k, st);
    case 3: return launch_generic<3, STDG_ADVECTION, T>(mode, k, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_advection<double>(int, int, const OpArgs<double>&, cudaStream_t);
template cudaError_t launch_advection<float>(int, int, const OpArgs<float>&, cudaStream_t);

}  // namespace stdg
