// Point-block preconditioner: build (P_I^-1 per spatial node) and apply.
// See precond.cuh for the derivation of P_I.
#include "precond.cuh"

namespace stdg {

namespace {

template <int DIM, int EQ, class TP>
__global__ void __launch_bounds__(128) pb_build_kernel(const __grid_constant__ OpArgs<double> k,
                                                       const double* __restrict__ U, TP* __restrict__ Pinv) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < k.nelem * k.nd) pb_build_node<DIM, EQ, TP>(k, U, Pinv, idx);
}

template <class TP> struct Acc { using type = double; };
template <> struct Acc<float> { using type = float; };

// Thread per (element, value q of one temporal node's [node][c] block): the s
// values of q across the temporal nodes are read once (coalesced per m) and
// mapped by the s x s matrix of q's node.
template <int S, class TP, class TV, class TO>
__global__ void __launch_bounds__(256) pb_apply_kernel(TO* out, const TV* __restrict__ v, double a,
                                                       const TP* __restrict__ Pinv, int accumulate, long long nelem,
                                                       int nd, int r) {
  using CT = typename Acc<TP>::type;
  const int tnode = nd * r;
  const size_t total = (size_t)nelem * tnode;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const CT ac = (CT)a;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const size_t e = idx / tnode;
    const int q = (int)(idx - e * tnode);
    const int node = q / r;
    CT x[S];
#pragma unroll
    for (int j = 0; j < S; ++j) x[j] = (CT)v[(e * S + j) * tnode + q];
    const TP* P = Pinv + (e * S * S) * nd + node;
#pragma unroll
    for (int m = 0; m < S; ++m) {
      CT z = CT(0);
#pragma unroll
      for (int j = 0; j < S; ++j) z = fma((CT)P[(size_t)(m * S + j) * nd], x[j], z);
      const size_t o = (e * S + m) * tnode + q;
      if (accumulate) out[o] = (TO)((double)out[o] + (double)(ac * z));
      else out[o] = (TO)(ac * z);
    }
  }
}

unsigned apply_grid(size_t total) {
  size_t b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <int DIM, int EQ, class TP>
cudaError_t build_inst(const OpArgs<double>& k, const double* U, TP* Pinv, cudaStream_t st) {
  const long long total = k.nelem * k.nd;
  const unsigned blocks = (unsigned)((total + 127) / 128);
  pb_build_kernel<DIM, EQ, TP><<<blocks, 128, 0, st>>>(k, U, Pinv);
  return cudaGetLastError();
}

}  // namespace

template <class TP>
cudaError_t pb_build(int dim, int eq, const OpArgs<double>& k, const double* U, TP* Pinv, cudaStream_t st) {
  if (k.s < 2 || k.s > kMaxS) return cudaErrorInvalidValue;
  switch (eq) {
    case STDG_ADVECTION:
      if (dim == 1) return build_inst<1, STDG_ADVECTION, TP>(k, U, Pinv, st);
      if (dim == 2) return build_inst<2, STDG_ADVECTION, TP>(k, U, Pinv, st);
      if (dim == 3) return build_inst<3, STDG_ADVECTION, TP>(k, U, Pinv, st);
      break;
    case STDG_BURGERS:
      if (dim == 1) return build_inst<1, STDG_BURGERS, TP>(k, U, Pinv, st);
      if (dim == 2) return build_inst<2, STDG_BURGERS, TP>(k, U, Pinv, st);
      break;
    case STDG_EULER:
      if (dim == 1) return build_inst<1, STDG_EULER, TP>(k, U, Pinv, st);
      if (dim == 2) return build_inst<2, STDG_EULER, TP>(k, U, Pinv, st);
      if (dim == 3) return build_inst<3, STDG_EULER, TP>(k, U, Pinv, st);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

template <class TP, class TV, class TO>
cudaError_t pb_apply(TO* out, const TV* v, double a, const TP* Pinv, int accumulate, long long nelem, int s,
                     int nd, int r, cudaStream_t st) {
  const unsigned g = apply_grid((size_t)nelem * nd * r);
  switch (s) {
    case 2: pb_apply_kernel<2, TP, TV, TO><<<g, 256, 0, st>>>(out, v, a, Pinv, accumulate, nelem, nd, r); break;
    case 3: pb_apply_kernel<3, TP, TV, TO><<<g, 256, 0, st>>>(out, v, a, Pinv, accumulate, nelem, nd, r); break;
    case 4: pb_apply_kernel<4, TP, TV, TO><<<g, 256, 0, st>>>(out, v, a, Pinv, accumulate, nelem, nd, r); break;
    case 5: pb_apply_kernel<5, TP, TV, TO><<<g, 256, 0, st>>>(out, v, a, Pinv, accumulate, nelem, nd, r); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t pb_build<double>(int, int, const OpArgs<double>&, const double*, double*, cudaStream_t);
template cudaError_t pb_build<float>(int, int, const OpArgs<double>&, const double*, float*, cudaStream_t);
template cudaError_t pb_apply<double, double, double>(double*, const double*, double, const double*, int, long long,
                                                      int, int, int, cudaStream_t);
template cudaError_t pb_apply<float, float, float>(float*, const float*, double, const float*, int, long long, int,
                                                   int, int, cudaStream_t);
template cudaError_t pb_apply<float, float, double>(double*, const float*, double, const float*, int, long long, int,
                                                    int, int, cudaStream_t);

}  // namespace stdg
