// Fused space-time DG-SEM operator: residual R(U), or J(U) v, of one time slab.
//
// One CTA owns `epb` consecutive elements (all s temporal nodes of each).  The
// element tiles are staged in shared memory (component-planar, padded to an
// odd node stride), then for every temporal node m:
//   1. thread per node: f_a(u) and the wave speed |v_a| + c for all
//      directions a (one reciprocal of rho, one pressure, one sound speed)
//   2. thread per node: volume term  -sum_a (2/h_a) (D f_a)      -> smem acc
//   3. thread per face point, one direction a at a time: Rusanov flux with
//      the neighbour trace (read from global memory / L2; its flux and wave
//      speed share one reciprocal and one pressure) and the strong-form face
//      correction -(2/h_a)(1/w_end)(H.n - f_a(u).n) added to acc
//   4. thread per output value (coalesced): temporal coupling
//        R_m = sum_j omega_j Dtau[j][m] U_j + [m=0] u_prev - [m=s-1] U_s
//              + dt/2 omega_m F_m
//      (Eq. DG_in_time moved to one side so that dR/dU is Eq. Jacobian_ST).
// Strong form of the spatial operator (Sec. 3.1 with the SBP property of
// Eq. SBP): F_I = -sum_a (2/h_a) [ sum_j D[i_a][j] f_a(u_(I,i_a->j))
//      + (1/w_N) [i_a = N] (H_a^+ - f_a(u_I)) - (1/w_0) [i_a = 0] (H_a^- - f_a(u_I)) ].
// The kernel is FP64-pipe bound in FP64 (ncu), so every FP64 operation it
// can avoid is avoided: 2/h_a is folded into D, 1/eps is a multiplication,
// wave speeds are computed once per node.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace stdg {

// Pointwise state that the spatial operator sees in each mode.
template <int MODE, class T>
__device__ __forceinline__ auto eval_state(T u, T v, T eps) {
  if constexpr (MODE == kModeJvExact) return Dual<T>{u, v};
  else if constexpr (MODE == kModeJvFD) return u + eps * v;
  else return u;
}
template <class T> __device__ __forceinline__ T tangent(Dual<T> x) { return x.d; }
template <class T> __device__ __forceinline__ T tangent(T x) { return T(0); }

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// Shared-memory footprint (bytes) of one CTA.
template <int DIM, int R, class T, int MODE>
__host__ __device__ inline size_t op_smem_bytes(int n, int s, int epb) {
  int nd = 1;
  for (int a = 0; a < DIM; ++a) nd *= n;
  int ndp = nd | 1;
  size_t vbytes = (MODE == kModeJvExact) ? 2 * sizeof(T) : sizeof(T);
  size_t b = (size_t)epb * s * R * ndp * sizeof(T);            // U tile
  if (MODE != kModeResidual) b += (size_t)epb * s * R * ndp * sizeof(T);  // v tile
  b += (size_t)epb * DIM * R * ndp * vbytes;                     // fluxes
  b += (size_t)epb * R * ndp * vbytes;                           // accumulators
  b += (size_t)epb * DIM * ndp * vbytes;                         // wave speeds
  b += (3 * kMaxN * kMaxN + kMaxS * kMaxS) * sizeof(T);          // scaled D per direction, C
  return b;
}

// NPX/NTX: compile-time n and s when FIXED, else upper bounds (runtime n, s).
template <int DIM, int EQ, class T, int MODE, int NPX, int NTX, bool FIXED>
__global__ void __launch_bounds__(256) st_operator_kernel(const __grid_constant__ OpArgs<T> k) {
  using P = Phys<EQ, DIM>;
  constexpr int R = P::R;
  using V = typename std::conditional<MODE == kModeJvExact, Dual<T>, T>::type;

  const int n = FIXED ? NPX : k.n;
  const int s = FIXED ? NTX : k.s;
  const int nd = FIXED ? ipow_c(NPX, DIM) : k.nd;
  const int ndp = nd | 1;
  const int nf = nd / n;  // nodes on one face
  const int epb = k.epb;

  const long long e0 = (long long)blockIdx.x * epb;
  const int nel = (int)((k.nelem - e0) < epb ? (k.nelem - e0) : epb);
  const int tid = threadIdx.x, nth = blockDim.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);                       // [epb][s][R][ndp]
  T* sv = su + (size_t)epb * s * R * ndp;                        // [epb][s][R][ndp] (Jv modes)
  V* sf = reinterpret_cast<V*>(MODE == kModeResidual ? sv : sv + (size_t)epb * s * R * ndp);  // [epb][DIM][R][ndp]
  V* sr = sf + (size_t)epb * DIM * R * ndp;                      // [epb][R][ndp]
  V* sl = sr + (size_t)epb * R * ndp;                            // [epb][DIM][ndp] wave speeds
  T* sD = reinterpret_cast<T*>(sl + (size_t)epb * DIM * ndp);    // [3][kMaxN][kMaxN]  (2/h_a) D
  T* sC = sD + 3 * kMaxN * kMaxN;                                // [kMaxS][kMaxS]  C
  for (int i = tid; i < 3 * kMaxN * kMaxN; i += nth) {
    const int a = i / (kMaxN * kMaxN), q = i % (kMaxN * kMaxN);
    sD[i] = k.ginv[a] * k.D[q / kMaxN][q % kMaxN];
  }
  for (int i = tid; i < kMaxS * kMaxS; i += nth) sC[i] = k.C[i / kMaxS][i % kMaxS];

  const size_t slab_elem = (size_t)s * nd * R;  // values of one element's slab
  // ---- stage the element tiles (coalesced global reads, planar smem writes)
  {
    const size_t total = (size_t)nel * slab_elem;
    const T* gU = k.U + (size_t)e0 * slab_elem;
    const T* gv = (MODE != kModeResidual) ? k.v + (size_t)e0 * slab_elem : nullptr;
    for (size_t idx = tid; idx < total; idx += nth) {
      int c = (int)(idx % R);
      size_t t = idx / R;
      int node = (int)(t % nd);
      t /= nd;  // = el * s + m
      size_t so = (t * R + c) * ndp + node;
      su[so] = gU[idx];
      if (MODE != kModeResidual) sv[so] = k.vscale * gv[idx];
    }
  }
  __syncthreads();

  int strides[3] = {1, n, n * n};

  for (int m = 0; m < s; ++m) {
    // ---- 1. fluxes and wave speeds at every node of the temporal node m
    for (int t = tid; t < nel * nd; t += nth) {
      int el = t / nd, node = t - el * nd;
      size_t so = ((size_t)(el * s + m) * R) * ndp + node;
      V u[R];
#pragma unroll
      for (int c = 0; c < R; ++c)
        u[c] = eval_state<MODE>(su[so + c * ndp], MODE == kModeResidual ? T(0) : sv[so + c * ndp], k.eps);
      V f[DIM][R];
      V lam[DIM];
      P::flux_all_speed(u, f, lam, k);
      V* sfe = sf + (size_t)el * DIM * R * ndp;
      V* sle = sl + (size_t)el * DIM * ndp;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        sle[a * ndp + node] = lam[a];
#pragma unroll
        for (int c = 0; c < R; ++c) sfe[(a * R + c) * ndp + node] = f[a][c];
      }
    }
    __syncthreads();
    // ---- 2. volume term
    for (int t = tid; t < nel * nd; t += nth) {
      int el = t / nd, node = t - el * nd;
      int idx[3] = {node % n, (node / n) % n, node / (n * n)};
      const V* sfe = sf + (size_t)el * DIM * R * ndp;
      V acc[R];
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] = Lift<V, T>::from(T(0));
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int ia = idx[a];
        const int base = node - ia * strides[a];
        const T* Da = sD + (a * kMaxN + ia) * kMaxN;
#pragma unroll
        for (int c = 0; c < R; ++c) {
#pragma unroll
          for (int j = 0; j < NPX; ++j) {
            if (FIXED || j < n) acc[c] = acc[c] - Da[j] * sfe[(a * R + c) * ndp + base + j * strides[a]];
          }
        }
      }
      V* sre = sr + (size_t)el * R * ndp;
#pragma unroll
      for (int c = 0; c < R; ++c) sre[c * ndp + node] = acc[c];
    }
    __syncthreads();
    // ---- 3. face corrections, one direction at a time (no two face points of a
    //         direction touch the same node when n >= 2)
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      for (int t = tid; t < nel * 2 * nf; t += nth) {
        int el = t / (2 * nf);
        int rem = t - el * 2 * nf;
        int side = rem / nf;  // 0: lower face (normal -e_a), 1: upper face (normal +e_a)
        int fidx = rem - side * nf;
        // own node: insert i_a into the face index
        int lo = fidx % strides[a];
        int hi = fidx / strides[a];
        int ia_own = side ? n - 1 : 0;
        int own = lo + ia_own * strides[a] + hi * strides[a] * n;
        int nbr_node = lo + (n - 1 - ia_own) * strides[a] + hi * strides[a] * n;
        // neighbour element (periodic)
        long long e = e0 + el;
        long long ex = e % k.K[0];
        long long ey = (e / k.K[0]) % k.K[1];
        long long ez = e / ((long long)k.K[0] * k.K[1]);
        long long ec[3] = {ex, ey, ez};
        ec[a] += side ? 1 : -1;
        if (ec[a] < 0) ec[a] += k.K[a];
        if (ec[a] >= k.K[a]) ec[a] -= k.K[a];
        long long en = (ec[2] * k.K[1] + ec[1]) * k.K[0] + ec[0];
        size_t gofs = ((size_t)en * s + m) * nd * R + (size_t)nbr_node * R;
        size_t so = ((size_t)(el * s + m) * R) * ndp + own;
        V um[R], up[R], fp[R], fm[R];
        const V* sfe = sf + (size_t)el * DIM * R * ndp;
#pragma unroll
        for (int c = 0; c < R; ++c) {
          fm[c] = sfe[(a * R + c) * ndp + own];
          const bool hasv = MODE != kModeResidual;
          um[c] = eval_state<MODE>(su[so + c * ndp], hasv ? sv[so + c * ndp] : T(0), k.eps);
          up[c] = eval_state<MODE>(k.U[gofs + c], hasv ? k.vscale * k.v[gofs + c] : T(0), k.eps);
        }
        const V lm = sl[((size_t)el * DIM + a) * ndp + own];
        const V lp = P::flux_speed(up, a, fp, k);
        V* sre = sr + (size_t)el * R * ndp;
        const T g = k.ginv[a] * k.winv_end;
        if (side) {  // uL = u-, uR = u+ ; F -= g (H - f(u-))
          V lam = dmax(lm, lp);
#pragma unroll
          for (int c = 0; c < R; ++c) {
            V H = T(0.5) * (fm[c] + fp[c]) - T(0.5) * (lam * (up[c] - um[c]));
            sre[c * ndp + own] = sre[c * ndp + own] - g * (H - fm[c]);
          }
        } else {     // uL = u+, uR = u- ; F += g (H - f(u-))
          V lam = dmax(lp, lm);
#pragma unroll
          for (int c = 0; c < R; ++c) {
            V H = T(0.5) * (fp[c] + fm[c]) - T(0.5) * (lam * (um[c] - up[c]));
            sre[c * ndp + own] = sre[c * ndp + own] + g * (H - fm[c]);
          }
        }
      }
      __syncthreads();
    }
    // ---- 4. temporal coupling and output (coalesced: consecutive threads write
    //         consecutive values of the element's [node][c] block)
    {
      const T hw = k.half_dt * k.omega[m];
      for (int t = tid; t < nel * nd * R; t += nth) {
        int c = t % R;
        int r2 = t / R;
        int node = r2 % nd;
        int el = r2 / nd;
        size_t g = ((size_t)(e0 + el) * s + m) * nd * R + (size_t)node * R + c;
        V Fv = sr[((size_t)el * R + c) * ndp + node];
        const T* tile = (MODE == kModeResidual) ? su : sv;
        T lin = T(0);
#pragma unroll
        for (int j = 0; j < NTX; ++j)
          if (FIXED || j < s) lin += sC[j * kMaxS + m] * tile[((size_t)(el * s + j) * R + c) * ndp + node];
        if (m == s - 1) lin -= tile[((size_t)(el * s + m) * R + c) * ndp + node];
        if (MODE == kModeResidual) {
          // u_prev is only read when R is written (F-only launches pass no u_prev)
          if (k.out) {
            if (m == 0) lin += k.uprev[(size_t)(e0 + el) * nd * R + (size_t)node * R + c];
            k.out[g] = lin + hw * val(Fv);
          }
          if (k.fout) k.fout[g] = val(Fv);
        } else if (MODE == kModeJvFD) {
          const T dF = (val(Fv) - k.F0[g]) * k.inv_eps;
          k.out[g] = k.lscale ? fma(k.inv_omega[m], lin, k.half_dt * dF) : fma(hw, dF, lin);
        } else {
          const T dF = tangent(Fv);
          k.out[g] = k.lscale ? fma(k.inv_omega[m], lin, k.half_dt * dF) : fma(hw, dF, lin);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace stdg
