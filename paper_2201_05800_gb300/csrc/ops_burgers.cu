// Instantiations of the space-time operator for (inviscid) Burgers.
#include "ops_impl.cuh"

namespace stdg {

template <class T>
cudaError_t launch_burgers(int dim, int mode, const OpArgs<T>& k, cudaStream_t st) {
  switch (dim) {
    case 1: return launch_generic<1, STDG_BURGERS, T>(mode, k, st);
    case 2: return launch_generic<2, STDG_BURGERS, T>(mode, k, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_burgers<double>(int, int, const OpArgs<double>&, cudaStream_t);
template cudaError_t launch_burgers<float>(int, int, const OpArgs<float>&, cudaStream_t);

}  // namespace stdg
