// Instantiations and launcher of the tangent-only FP32 Jacobian-vector kernel
// (jv_tangent.cuh) for the Euler shapes of the 2D vortex (n = 5, s = 4) and the
// 3D density wave (n = 4, s = 3), the latter also with the volume contractions
// on the tensor cores (BF16 inputs, FP32 accumulation).
#include "jv_tangent.cuh"
#include "ops.h"

namespace stdg {

namespace {

template <int DIM, int NP, int NS, int E, bool TC = false>
cudaError_t launch_one(const OpArgs<float>& k, cudaStream_t st) {
  constexpr int ND = ipow_c(NP, DIM);
  constexpr size_t smem = jv_tangent_smem_bytes<DIM, NP, NS, E, TC>();
  auto kern = jv_tangent_kernel<DIM, NP, NS, E, TC>;
  static_assert(smem <= 227 * 1024, "tile exceeds shared memory");
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int threads = (E * NS * ND + 31) / 32 * 32;
  const long long blocks = (k.nelem + E - 1) / E;
  // CTAs resident at once on the device: the distance, in tiles, of each CTA's L2 prefetch
  static const int resident = [&] {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess)
      return 0;
    return sms * occ;
  }();
  OpArgs<float> a = k;
  a.prefetch = resident;
  kern<<<(unsigned)blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// J(U) v in FP32 by the tangent-only kernel when the shape has an instantiation and the
// slabs satisfy the bulk-copy alignment (16-byte base addresses; element tiles are whole
// multiples of 16 bytes for these shapes).  *handled = false: nothing was launched.
cudaError_t launch_jv_tangent(int dim, int eq, const OpArgs<float>& k, cudaStream_t st, bool* handled,
                              bool tensor_cores) {
  *handled = false;
  if (eq != STDG_EULER || !k.U || !k.v || !k.out || k.nelem < 1) return cudaSuccess;
  if (!aligned16(k.U) || !aligned16(k.v)) return cudaSuccess;
  if (dim == 2 && k.n == 5 && k.s == 4) {
    *handled = true;
    return launch_one<2, 5, 4, 2>(k, st);
  }
  if (dim == 3 && k.n == 4 && k.s == 3) {
    *handled = true;
    return tensor_cores ? launch_one<3, 4, 3, 2, true>(k, st) : launch_one<3, 4, 3, 1>(k, st);
  }
  return cudaSuccess;
}

}  // namespace stdg
