// Exact Jacobian-vector product of the space-time residual for the Euler
// equations, tangent only (forward mode without the value of F):
//
//   J(U) v = (D_tau^T M_tau (x) I) v - e_s e_s^T v + dt/2 (M_tau (x) I) F'(U) v,
//
// Eq. Jacobian_ST, with F'(U) v the derivative of the strong-form DG-SEM
// operator (Sec. 3.1, Eqs. elementint/surfaceint, Rusanov flux Eq. flux:llf)
// in the direction v.  Only tangents are accumulated: the values of the
// fluxes and of the numerical flux H never enter J v (the values of 1/rho, p,
// c, |v_a| + c and of the face jumps are still needed for the derivatives).
//
// One CTA owns E consecutive elements and all s temporal nodes of their
// slab tiles (element-major layout, so the tiles of U and of v are each one
// contiguous block).  Both blocks are staged into shared memory with one bulk
// asynchronous copy each (cp.async.bulk completing on an mbarrier).  Then,
// with one thread per (element, temporal node, spatial node):
//   0. primitives and the flux tangents df_a for every direction a, and the
//      wave speeds |v_a| + c with their tangents            -> shared memory
//   1. the volume term -sum_a (2/h_a) D df_a along each line (registers), and,
//      by the same threads, every face point of the tile: the Rusanov
//      tangent against the neighbour's trace (read from global memory, L2)
//      and the strong-form correction of the own node, written to a slot per
//      direction (a node lies on at most one face per direction, so no two
//      items write the same slot and the final sum has a fixed order)
//   2. the temporal coupling from the staged v and the output, coalesced.
// Two barriers per tile.  Every face point is evaluated once by each of its
// two elements (the neighbour's side from global memory).
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace stdg {

constexpr long long kWaitLimit = 1ll << 22;  // try_wait polls before a bounded wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for phase `parity` of `bar`; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
  const unsigned a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Shared-memory bytes of one CTA of jv_tangent_kernel.
template <int DIM, int NP, int NS, int E>
__host__ __device__ constexpr size_t jv_tangent_smem_bytes() {
  constexpr int R = DIM + 2;
  constexpr int ND = ipow_c(NP, DIM);
  return sizeof(float) * ((size_t)2 * E * NS * ND * R       // staged U and v tiles
                          + (size_t)E * NS * DIM * R * ND   // flux tangents
                          + (size_t)2 * E * NS * DIM * ND   // wave speeds and tangents
                          + (size_t)E * NS * DIM * R * ND   // face corrections per direction
                          + (size_t)DIM * NP * NP);         // (2/h_a) D
}

// x[a] for a runtime index a without local memory (unrolled selects).
template <int N>
__device__ __forceinline__ float pick(const float (&x)[N], int a) {
  float r = x[0];
#pragma unroll
  for (int i = 1; i < N; ++i) r = a == i ? x[i] : r;
  return r;
}

// Primitives of one Euler state and its tangent: 1/rho, v_a, p (values) and their tangents.
template <int DIM>
struct EulerTangent {
  static constexpr int R = DIM + 2;
  float ir, dir, v[DIM], dv[DIM], p, dp;
  __device__ __forceinline__ void init(const float (&u)[R], const float (&du)[R], float gamma) {
    ir = 1.0f / u[0];
    dir = -du[0] * ir * ir;
    float ke = 0.f, dke = 0.f;  // |m|^2 / rho and its tangent
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      v[a] = u[1 + a] * ir;
      dv[a] = fmaf(du[1 + a], ir, u[1 + a] * dir);
      ke = fmaf(u[1 + a], v[a], ke);
      dke = fmaf(du[1 + a], v[a], fmaf(u[1 + a], dv[a], dke));
    }
    p = (gamma - 1.0f) * fmaf(-0.5f, ke, u[R - 1]);
    dp = (gamma - 1.0f) * fmaf(-0.5f, dke, du[R - 1]);
  }
  // tangent of f_a(u) (a may be a runtime index)
  __device__ __forceinline__ void flux_tangent(const float (&u)[R], const float (&du)[R], int a,
                                               float (&df)[R]) const {
    const float va = pick(v, a), dva = pick(dv, a);
    float dma = du[1];
#pragma unroll
    for (int b = 1; b < DIM; ++b) dma = a == b ? du[1 + b] : dma;
    df[0] = dma;
#pragma unroll
    for (int b = 0; b < DIM; ++b) df[1 + b] = fmaf(du[1 + b], va, u[1 + b] * dva) + (b == a ? dp : 0.f);
    df[R - 1] = fmaf(du[R - 1] + dp, va, (u[R - 1] + p) * dva);
  }
  // |v_a| + c and its tangent (|x| differentiates as x for x >= 0)
  __device__ __forceinline__ void speed(int a, float gamma, float c, float dc, float* lam, float* dlam) const {
    const float va = pick(v, a), dva = pick(dv, a);
    const bool pos = va >= 0.f;
    *lam = (pos ? va : -va) + c;
    *dlam = (pos ? dva : -dva) + dc;
  }
  __device__ __forceinline__ void sound(float gamma, float* c, float* dc) const {
    const float q = gamma * (p * ir);
    *c = sqrtf(q);
    const float dq = gamma * fmaf(dp, ir, p * dir);
    *dc = dq * (0.5f / *c);
  }
};

// out = J(U) v for elements [blockIdx.x * E, ...) of the slab.  FP32; k.U, k.v, k.out are
// FP32 slabs [e][m][node][c]; blockDim.x >= E * NS * ND.
template <int DIM, int NP, int NS, int E>
__global__ void __launch_bounds__((E * NS * ipow_c(NP, DIM) + 31) / 32 * 32)
    jv_tangent_kernel(const __grid_constant__ OpArgs<float> k) {
  constexpr int R = DIM + 2;
  constexpr int ND = ipow_c(NP, DIM);
  constexpr int NF = ND / NP;
  constexpr int TILE = NS * ND * R;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* su = reinterpret_cast<float*>(smem_raw);  // [E][NS][ND][R]
  float* sv = su + E * TILE;                       // [E][NS][ND][R]
  float* sf = sv + E * TILE;                       // [E][NS][DIM][R][ND]
  float* sl = sf + E * NS * DIM * R * ND;          // [E][NS][DIM][ND]
  float* sdl = sl + E * NS * DIM * ND;             // [E][NS][DIM][ND]
  float* sc = sdl + E * NS * DIM * ND;             // [E][NS][DIM][R][ND]
  float* sD = sc + E * NS * DIM * R * ND;          // [DIM][NP][NP]
  __shared__ __align__(8) uint64_t bar;
  __shared__ int staged;

  const int tid = threadIdx.x;
  const long long e0 = (long long)blockIdx.x * E;
  const int nel = (int)((k.nelem - e0) < E ? (k.nelem - e0) : E);
  if (tid == 0) {
    mbar_init(&bar, 1);
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned bytes = (unsigned)(nel * TILE * sizeof(float));
    mbar_expect_tx(&bar, 2 * bytes);
    bulk_g2s(su, k.U + e0 * TILE, bytes, &bar);
    bulk_g2s(sv, k.v + e0 * TILE, bytes, &bar);
  }
  for (int i = tid; i < DIM * NP * NP; i += blockDim.x) {
    const int a = i / (NP * NP), q = i % (NP * NP);
    sD[i] = k.ginv[a] * k.D[q / NP][q % NP];
  }
  if (tid == 0) {
    bool ok = mbar_wait(&bar, 0, kWaitLimit);
    if (!ok) {
      if (k.err) atomicOr(k.err, 1u);
      mbar_wait(&bar, 0, kWaitLimit);  // let the copies in flight land before the CTA exits
    }
    staged = ok ? 1 : 0;
  }
  __syncthreads();
  if (!staged) return;
  mbar_wait(&bar, 0, kWaitLimit);  // completed: acquire the staged data in every thread

  const int item = tid;
  const bool active = item < nel * NS * ND;
  const int el = item / (NS * ND);
  const int m = (item / ND) % NS;
  const int node = item % ND;
  const int q1 = node / NP, q2 = q1 / NP;
  const int idx[3] = {node % NP, DIM > 1 ? q1 % NP : 0, DIM > 2 ? q2 : 0};
  const int strides[3] = {1, NP, NP * NP};
  const float gamma = k.gamma;

  // ---- 0. primitives, flux tangents and wave speeds at (el, m, node)
  if (active) {
    const float* ue = su + ((el * NS + m) * ND + node) * R;
    const float* due = sv + ((el * NS + m) * ND + node) * R;
    float u[R], du[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
      u[c] = ue[c];
      du[c] = due[c];
    }
    EulerTangent<DIM> P;
    P.init(u, du, gamma);
    float c0, dc0;
    P.sound(gamma, &c0, &dc0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      float df[R];
      P.flux_tangent(u, du, a, df);
      float* sfa = sf + (((el * NS + m) * DIM + a) * R) * ND + node;
#pragma unroll
      for (int c = 0; c < R; ++c) sfa[c * ND] = df[c];
      float lam, dlam;
      P.speed(a, gamma, c0, dc0, &lam, &dlam);
      sl[((el * NS + m) * DIM + a) * ND + node] = lam;
      sdl[((el * NS + m) * DIM + a) * ND + node] = dlam;
    }
  }
  __syncthreads();

  // ---- 1a. volume term (tangent), kept in registers for the output phase
  float acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = 0.f;
  if (active) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int ia = idx[a];
      const int base = node - ia * strides[a];
      const float* Da = sD + (a * NP + ia) * NP;
      const float* sfa = sf + (((el * NS + m) * DIM + a) * R) * ND + base;
#pragma unroll
      for (int c = 0; c < R; ++c)
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[c] = fmaf(-Da[j], sfa[c * ND + j * strides[a]], acc[c]);
    }
  }
  // ---- 1b. face points: items (el, m, a, side, fidx), correction of the own node
  const float gh_end = 0.5f * k.winv_end;
  for (int f = tid; f < nel * NS * DIM * 2 * NF; f += blockDim.x) {
    const int fidx = f % NF;
    const int side = (f / NF) & 1;  // 1: upper face (normal +e_a)
    const int a = (f / (2 * NF)) % DIM;
    const int fm = (f / (2 * NF * DIM)) % NS;
    const int fel = f / (2 * NF * DIM * NS);
    const int sa = a == 0 ? 1 : (a == 1 ? NP : NP * NP);  // node stride along e_a
    const int hi = a == 0 ? fidx : (a == 1 ? fidx / NP : 0);
    const int lo = fidx - hi * sa;
    const int ia_own = side ? NP - 1 : 0;
    const int own = lo + ia_own * sa + hi * sa * NP;
    const int nbr = lo + (NP - 1 - ia_own) * sa + hi * sa * NP;
    // periodic neighbour element across the face (element index e = (ez K1 + ey) K0 + ex)
    const int e = (int)(e0 + fel);
    const int K0 = k.K[0], K1 = k.K[1], K2 = k.K[2];
    int ex = e % K0, ey = (e / K0) % K1, ez = e / (K0 * K1);
    const int step = side ? 1 : -1;
    if (a == 0) ex = (ex + step + K0) % K0;
    else if (a == 1) ey = (ey + step + K1) % K1;
    else ez = (ez + step + K2) % K2;
    const long long en = ((long long)ez * K1 + ey) * K0 + ex;
    // own side (staged)
    const float* uo = su + ((fel * NS + fm) * ND + own) * R;
    const float* duo = sv + ((fel * NS + fm) * ND + own) * R;
    const float* sfo = sf + (((fel * NS + fm) * DIM + a) * R) * ND + own;
    const float lo_l = sl[((fel * NS + fm) * DIM + a) * ND + own];
    const float lo_d = sdl[((fel * NS + fm) * DIM + a) * ND + own];
    // neighbour side (global memory)
    const size_t gn = (((size_t)en * NS + fm) * ND + nbr) * R;
    float un[R], dun[R], dfn[R];
#pragma unroll
    for (int c = 0; c < R; ++c) {
      un[c] = __ldg(k.U + gn + c);
      dun[c] = __ldg(k.v + gn + c);
    }
    EulerTangent<DIM> Pn;
    Pn.init(un, dun, gamma);
    float cn, dcn, ln, dln;
    Pn.sound(gamma, &cn, &dcn);
    Pn.speed(a, gamma, cn, dcn, &ln, &dln);
    Pn.flux_tangent(un, dun, a, dfn);
    // Rusanov tangent with lambda = max over the two states (ties: the state below the face)
    float lam, dlam;
    if (side) {
      const bool own_wins = lo_l >= ln;
      lam = own_wins ? lo_l : ln;
      dlam = own_wins ? lo_d : dln;
    } else {
      const bool nbr_wins = ln >= lo_l;
      lam = nbr_wins ? ln : lo_l;
      dlam = nbr_wins ? dln : lo_d;
    }
    const float g = gh_end * k.ginv[a];
    float* sco = sc + (((fel * NS + fm) * DIM + a) * R) * ND + own;
#pragma unroll
    for (int c = 0; c < R; ++c) {
      // side 1: -(g/2)(d(df) - dlam du - lam d(du)), du = u_nbr - u_own, df = f_nbr - f_own
      // side 0: +(g/2)(d(df) - dlam du - lam d(du)), du = u_own - u_nbr, df = f_nbr - f_own
      const float ddf = dfn[c] - sfo[c * ND];
      const float jv = side ? un[c] - uo[c] : uo[c] - un[c];
      const float djv = side ? dun[c] - duo[c] : duo[c] - dun[c];
      const float t = ddf - fmaf(dlam, jv, lam * djv);
      sco[c * ND] = side ? -g * t : g * t;
    }
  }
  __syncthreads();

  // ---- 2. temporal coupling and output
  if (active) {
    const float vs = k.vscale;
    const float sm = k.lscale ? k.inv_omega[m] : 1.0f;
    const float cfac = (k.lscale ? k.half_dt : k.half_dt * k.omega[m]) * vs;
    const float cv = sm * vs;
    const float* vn = sv + (el * NS * ND + node) * R;  // (el, j = 0, node)
    float* out = k.out + (((size_t)(e0 + el) * NS + m) * ND + node) * R;
#pragma unroll
    for (int c = 0; c < R; ++c) {
      float F = acc[c];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        if (idx[a] == 0 || idx[a] == NP - 1) F += sc[(((el * NS + m) * DIM + a) * R + c) * ND + node];
      float lin = 0.f;
#pragma unroll
      for (int j = 0; j < NS; ++j) lin = fmaf(k.C[j][m], vn[j * ND * R + c], lin);
      if (m == NS - 1) lin -= vn[m * ND * R + c];
      out[c] = fmaf(cfac, F, cv * lin);
    }
  }
}

}  // namespace stdg
