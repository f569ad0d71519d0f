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

#include <cuda_bf16.h>
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

// Hint: bring `bytes` (a multiple of 16, 16-byte aligned) from global memory into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bounded wait for phase `parity` of `bar`; false when the limit ran out.  A failed poll backs
// off for a few tens of nanoseconds, so that the waiting warp does not take issue slots from the
// warps of the other CTAs on the SM while the copy is in flight.
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
    __nanosleep(32);
  }
  return false;
}

// Line pitch of the flux-tangent store: a line of NP values padded to whole 16-byte words.
__host__ __device__ constexpr int jv_line_pitch(int np) { return (np + 3) / 4 * 4; }

// ---------------------------------------------------------------- tensor cores (tcgen05)
// One CTA-wide BF16 x BF16 -> FP32 MMA of M = 128, N = 16, K = 16 with the operands in shared
// memory (K-major, no swizzle: 8-row x 16-byte core matrices, K chunks kTcLbo bytes apart,
// 8-row groups kTcSbo bytes apart) and the accumulator in tensor memory (row i = TMEM lane i,
// column j = TMEM column j).
constexpr unsigned kTcLbo = 128, kTcSbo = 256;
constexpr unsigned kTcCols = 64;  // TMEM columns allocated per CTA (three 16-column accumulators)

__device__ __forceinline__ unsigned tc_offset(int row, int k) {  // byte offset of (row, k), bf16
  return (unsigned)((row >> 3) * kTcSbo + (k >> 3) * kTcLbo + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t tc_desc(const void* smem) {
  const uint64_t a = smem_u32(smem);
  return ((a >> 4) & 0x3FFFull) | ((uint64_t)(kTcLbo >> 4) << 16) | ((uint64_t)(kTcSbo >> 4) << 32) |
         (1ull << 46);  // descriptor version 1, no swizzle, base offset 0
}
// instruction descriptor: D FP32, A and B BF16, both K-major, N = 16, M = 128
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tmem_alloc(unsigned* dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(kTcCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(unsigned d_tmem, uint64_t adesc, uint64_t bdesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(0)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ..)
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory bytes of one CTA of jv_tangent_kernel (TC: plus the tensor-core operands, BF16
// A (128 x 16) and B (16 x 16) per direction at a 128-byte boundary, and the volume terms read
// back from tensor memory, one slot per direction).
template <int DIM, int NP, int NS, int E, bool TC = false>
__host__ __device__ constexpr size_t jv_tangent_smem_bytes() {
  constexpr int R = DIM + 2;
  constexpr int ND = ipow_c(NP, DIM);
  constexpr int LINES = (ND / NP) * jv_line_pitch(NP);
  constexpr size_t base = sizeof(float) * ((size_t)2 * E * NS * ND * R          // staged U and v tiles
                                           + (size_t)E * NS * DIM * R * LINES   // flux tangents, per direction
                                           + (size_t)2 * E * NS * DIM * ND      // wave speeds and tangents
                                           + (size_t)E * NS * DIM * R * ND      // face corrections per direction
                                           + (size_t)DIM * NP * jv_line_pitch(NP));  // (2/h_a) D, rows padded
  return TC ? (base + 127) / 128 * 128 + (size_t)DIM * (128 * 16 + 16 * 16) * 2 +
                  sizeof(float) * (size_t)DIM * E * NS * R * ND
            : base;
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
    ir = __fdividef(1.0f, u[0]);  // hardware reciprocal: ~2 ulp, below the FP32 rounding of J v
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
    const float rq = rsqrtf(q);  // hardware 1/sqrt: c = q / sqrt(q), dc = dq / (2 sqrt(q))
    *c = q * rq;
    const float dq = gamma * fmaf(dp, ir, p * dir);
    *dc = dq * (0.5f * rq);
  }
};

// out = J(U) v for elements [blockIdx.x * E, ...) of the slab.  FP32; k.U, k.v, k.out are
// FP32 slabs [e][m][node][c]; blockDim.x >= E * NS * ND.
// TC: the volume contractions on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation):
// per direction a one M = 128 x N = 16 x K = 16 MMA whose rows are (element, component,
// temporal node, group of four lines along e_a) and whose K index is (line in the group, node on
// the line); B = I_4 (x) (-(2/h_a) D)^T.  3D, n = 4 only (E R NS 4 <= 128 rows).
template <int DIM, int NP, int NS, int E, bool TC = false>
__global__ void __launch_bounds__((E * NS * ipow_c(NP, DIM) + 31) / 32 * 32)
    jv_tangent_kernel(const __grid_constant__ OpArgs<float> k) {
  constexpr int R = DIM + 2;
  constexpr int ND = ipow_c(NP, DIM);
  constexpr int NF = ND / NP;
  constexpr int TILE = NS * ND * R;
  constexpr int LP = jv_line_pitch(NP);  // pitch of one line of the flux-tangent store
  constexpr int LINES = NF * LP;         // one component of one direction: NF lines
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* su = reinterpret_cast<float*>(smem_raw);  // [E][NS][ND][R]
  float* sv = su + E * TILE;                       // [E][NS][ND][R]
  // flux tangents of direction a, line-major: the NP values along e_a of line q at
  // [((el NS + m) DIM + a) R + c][q LP + i_a]; the line of a face point fidx is q = fidx
  float* sf = sv + E * TILE;
  float* sl = sf + E * NS * DIM * R * LINES;       // [E][NS][DIM][ND]
  float* sdl = sl + E * NS * DIM * ND;             // [E][NS][DIM][ND]
  float* sc = sdl + E * NS * DIM * ND;             // [E][NS][DIM][R][ND]
  float* sD = sc + E * NS * DIM * R * ND;          // [DIM][NP][LP]
  static_assert(TILE % 4 == 0, "element tiles must be whole 16-byte words (bulk copy)");
  static_assert(!TC || (DIM == 3 && NP == 4 && E * R * NS * 4 <= 128 && E * NS * ND >= 128),
                "tensor-core volume: 3D, n = 4, at most 128 MMA rows and four full warps");
  constexpr size_t kBase = jv_tangent_smem_bytes<DIM, NP, NS, E, false>();
  unsigned char* tcA = smem_raw + (kBase + 127) / 128 * 128;  // [a][128 x 16] bf16, core-matrix layout
  unsigned char* tcB = tcA + DIM * 128 * 16 * 2;               // [a][16 x 16] bf16
  float* svol = reinterpret_cast<float*>(tcB + DIM * 16 * 16 * 2);  // [a][E][NS][R][ND]
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ unsigned tmem_base;
  __shared__ int mma_ok;
  static_assert((2 * E * TILE + E * NS * DIM * R * LINES + 2 * E * NS * DIM * ND + E * NS * DIM * R * ND) % 4 == 0,
                "the D rows are read as 16-byte words");
  __shared__ __align__(8) uint64_t bar;
  __shared__ int staged;
  __shared__ long long snb[E * DIM * 2];  // periodic neighbour element of (el, a, side)

  const int tid = threadIdx.x;
  const long long e0 = (long long)blockIdx.x * E;
  const int nel = (int)((k.nelem - e0) < E ? (k.nelem - e0) : E);
  if (tid == 0) {
    mbar_init(&bar, 1);
    if (TC) mbar_init(&bar_mma, 1);
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned bytes = (unsigned)(nel * TILE * sizeof(float));
    mbar_expect_tx(&bar, 2 * bytes);
    bulk_g2s(su, k.U + e0 * TILE, bytes, &bar);
    bulk_g2s(sv, k.v + e0 * TILE, bytes, &bar);
    // the tile of the CTA that starts about one residency later: its copy then comes from L2
    const long long pe = e0 + (long long)k.prefetch * E;
    if (k.prefetch > 0 && pe < k.nelem) {
      const int pn = (int)((k.nelem - pe) < E ? (k.nelem - pe) : E);
      bulk_prefetch_l2(k.U + pe * TILE, (unsigned)(pn * TILE * sizeof(float)));
      bulk_prefetch_l2(k.v + pe * TILE, (unsigned)(pn * TILE * sizeof(float)));
    }
  }
  for (int i = tid; i < DIM * NP * LP; i += blockDim.x) {
    const int a = i / (NP * LP), r = (i / LP) % NP, j = i % LP;
    sD[i] = j < NP ? k.ginv[a] * k.D[r][j] : 0.f;
  }
  // neighbour table of the tile (element index e = (ez K1 + ey) K0 + ex, periodic)
  if (tid < nel * DIM * 2) {
    const int side = tid & 1, a = (tid >> 1) % DIM, fel = (tid >> 1) / DIM;
    const long long e = e0 + fel;
    const long long K0 = k.K[0], K1 = k.K[1], K2 = k.K[2];
    long long ex = e % K0, ey = (e / K0) % K1, ez = e / (K0 * K1);
    const long long step = side ? 1 : -1;
    if (a == 0) ex = (ex + step + K0) % K0;
    else if (a == 1) ey = (ey + step + K1) % K1;
    else ez = (ez + step + K2) % K2;
    snb[tid] = (ez * K1 + ey) * K0 + ex;
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
  if constexpr (TC) {
    if (tid < 32) {  // one warp allocates (and later frees) the accumulators
      tmem_alloc(&tmem_base);
      tc_fence_before();
    }
    // B_a = I_4 (x) (-(2/h_a) D)^T: B[n = 4 l' + i][kk = 4 l + j] = [l = l'] (-(2/h_a) D[i][j])
    for (int t = tid; t < DIM * 256; t += blockDim.x) {
      const int a = t >> 8, n = (t >> 4) & 15, kk = t & 15;
      const float b = (n >> 2) == (kk >> 2) ? -k.ginv[a] * k.D[n & 3][kk & 3] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(tcB + a * 512 + tc_offset(n, kk)) = __float2bfloat16_rn(b);
    }
    // rows past the CTA's elements are zero
    for (int t = tid; t < DIM * 128 * 16; t += blockDim.x) {
      const int a = t / 2048, row = (t / 16) % 128, kk = t % 16;
      if (row >= nel * R * NS * 4)
        *reinterpret_cast<__nv_bfloat16*>(tcA + a * 4096 + tc_offset(row, kk)) = __float2bfloat16_rn(0.f);
    }
  }

  const int item = tid;
  const bool active = item < nel * NS * ND;
  const int el = item / (NS * ND);
  const int m = (item / ND) % NS;
  const int node = item % ND;
  const int q1 = node / NP, q2 = q1 / NP;
  const int idx[3] = {node % NP, DIM > 1 ? q1 % NP : 0, DIM > 2 ? q2 : 0};
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
      // line q of node along e_a and position i_a on it
      const int ia = idx[a];
      const int q = a == 0 ? idx[1] + NP * idx[2] : (a == 1 ? idx[0] + NP * idx[2] : idx[0] + NP * idx[1]);
      float* sfa = sf + (((el * NS + m) * DIM + a) * R) * LINES + q * LP + ia;
#pragma unroll
      for (int c = 0; c < R; ++c) sfa[c * LINES] = df[c];
      if constexpr (TC) {  // the MMA operand: row (el, c, m, q / 4), column 4 (q % 4) + i_a
#pragma unroll
        for (int c = 0; c < R; ++c) {
          const int row = ((el * R + c) * NS + m) * 4 + (q >> 2);
          *reinterpret_cast<__nv_bfloat16*>(tcA + a * 4096 + tc_offset(row, 4 * (q & 3) + ia)) =
              __float2bfloat16_rn(df[c]);
        }
      }
      float lam, dlam;
      P.speed(a, gamma, c0, dc0, &lam, &dlam);
      sl[((el * NS + m) * DIM + a) * ND + node] = lam;
      sdl[((el * NS + m) * DIM + a) * ND + node] = dlam;
    }
  }
  if constexpr (TC) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands -> tensor cores
  __syncthreads();

  // ---- 1a. volume term (tangent), kept in registers for the output phase (TC: three MMAs,
  //          issued here and read back after the face points)
  float acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = 0.f;
  if constexpr (TC) {
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int a = 0; a < DIM; ++a) tc_mma(tmem_base + 16 * a, tc_desc(tcA + a * 4096), tc_desc(tcB + a * 512));
      tc_commit(&bar_mma);
    }
  }
  if (!TC && active) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int ia = idx[a];
      const int q = a == 0 ? idx[1] + NP * idx[2] : (a == 1 ? idx[0] + NP * idx[2] : idx[0] + NP * idx[1]);
      float Da[LP];
      const float4* Dv = reinterpret_cast<const float4*>(sD + (a * NP + ia) * LP);
#pragma unroll
      for (int w = 0; w < LP / 4; ++w) {
        const float4 d4 = Dv[w];
        Da[4 * w] = d4.x, Da[4 * w + 1] = d4.y, Da[4 * w + 2] = d4.z, Da[4 * w + 3] = d4.w;
      }
      const float* sfa = sf + (((el * NS + m) * DIM + a) * R) * LINES + q * LP;
#pragma unroll
      for (int c = 0; c < R; ++c) {
        const float4* fv = reinterpret_cast<const float4*>(sfa + c * LINES);
#pragma unroll
        for (int w = 0; w < LP / 4; ++w) {
          const float4 f4 = fv[w];
          const float f[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            if (4 * w + jj < NP) acc[c] = fmaf(-Da[4 * w + jj], f[jj], acc[c]);
        }
      }
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
    const long long en = snb[(fel * DIM + a) * 2 + side];
    // own side (staged)
    const float* uo = su + ((fel * NS + fm) * ND + own) * R;
    const float* duo = sv + ((fel * NS + fm) * ND + own) * R;
    const float* sfo = sf + (((fel * NS + fm) * DIM + a) * R) * LINES + fidx * LP + ia_own;
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
      const float ddf = dfn[c] - sfo[c * LINES];
      const float jv = side ? un[c] - uo[c] : uo[c] - un[c];
      const float djv = side ? dun[c] - duo[c] : duo[c] - dun[c];
      const float t = ddf - fmaf(dlam, jv, lam * djv);
      sco[c * ND] = side ? -g * t : g * t;
    }
  }
  if constexpr (TC) {
    // accumulators complete (bounded wait), then warps 0-3 read lanes 0-127 back to shared memory
    if (tid == 0) {
      bool ok = mbar_wait(&bar_mma, 0, kWaitLimit);
      if (!ok) {
        if (k.err) atomicOr(k.err, 1u);
        mbar_wait(&bar_mma, 0, kWaitLimit);
      }
      mma_ok = ok ? 1 : 0;
    }
    __syncthreads();
    tc_fence_after();
    if (tid < 128 && mma_ok) {
      const int row = tid;
      const int g = row & 3, rm = (row >> 2) % NS, rc = (row / (4 * NS)) % R, rel = row / (4 * NS * R);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        float v[16];
        tmem_ld16(tmem_base + ((unsigned)(tid & ~31) << 16) + 16 * a, v);
        if (rel < nel) {
#pragma unroll
          for (int nn = 0; nn < 16; ++nn) {
            const int q = 4 * g + (nn >> 2), i = nn & 3;
            const int node = a == 0 ? i + 4 * q : (a == 1 ? (q & 3) + 4 * i + 16 * (q >> 2) : q + 16 * i);
            svol[(((a * E + rel) * NS + rm) * R + rc) * ND + node] = v[nn];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 32) tmem_dealloc(tmem_base);
    if (!mma_ok) return;
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
      if constexpr (TC) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) F += svol[(((a * E + el) * NS + m) * R + c) * ND + node];
      }
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
