// Physics-independent kernels of the batched engine (engine.cuh): the dot
// pass, the per-slot controller and the vector update.
#include <math.h>

#include "engine.cuh"
#include "warp_scatter.cuh"

namespace stdg {

namespace {

// element range of a chunk item
__device__ __forceinline__ void chunk_range(const SlotBuf& b, int idx, long long* e0, long long* e1) {
  *e0 = (long long)idx * b.chunk_elems;
  long long hi = *e0 + b.chunk_elems;
  *e1 = hi < b.nelem ? hi : b.nelem;
}

// Block sum of k per-thread FP64 values into partials[0..k) (fixed order).
template <int KB>
__device__ __forceinline__ void block_reduce_store(const double (&accd)[KB], int k, double (*red)[kEngRows],
                                                   double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KB; ++i) {
    if (i < k) {
      double v = accd[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][i] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[q][threadIdx.x];
    out[threadIdx.x] = v;
  }
  __syncthreads();
}

// V_i . w over [v0, v1) for i < k, in passes over groups of G rows (w is re-read from L1/L2
// once per group).  The pass is bound by memory latency, so each thread keeps one 16-byte
// load of every row of the group in flight.  When the rows start on 16 bytes the aligned
// body of the range is read in 16-byte words (four values per load), the at most three
// values before and after it one by one.  Per-warp sums of each row go to red[warp][row];
// then one fixed-order sum.
template <int G>
__device__ __forceinline__ void dot_rows(const SlotBuf& b, size_t v0, size_t v1, int j, int k,
                                         double (*red)[kEngRows], double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float* w = b.V + (size_t)(j + 1) * b.L;
  size_t a0 = v0, a1 = v0;  // 16-byte body [a0, a1)
  if (b.vec4) {
    a0 = (v0 + 3) & ~(size_t)3;
    if (a0 > v1) a0 = v1;
    a1 = a0 + ((v1 - a0) & ~(size_t)3);
  }
  for (int g0 = 0; g0 < k; g0 += G) {
    float acc[G];
#pragma unroll
    for (int i = 0; i < G; ++i) acc[i] = 0.f;
    const float4* w4 = reinterpret_cast<const float4*>(w);
    for (size_t q = a0 / 4 + threadIdx.x; q < a1 / 4; q += blockDim.x) {
      const float4 wv = w4[q];
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (g0 + i < k) {
          const float4 x = reinterpret_cast<const float4*>(b.V + (size_t)(g0 + i) * b.L)[q];
          acc[i] = fmaf(x.w, wv.w, fmaf(x.z, wv.z, fmaf(x.y, wv.y, fmaf(x.x, wv.x, acc[i]))));
        }
    }
    for (size_t v = threadIdx.x; v < (a0 - v0) + (v1 - a1); v += blockDim.x) {  // head, then tail
      const size_t vv = v < a0 - v0 ? v0 + v : a1 + (v - (a0 - v0));
      const float w0 = w[vv];
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (g0 + i < k) acc[i] = fmaf(b.V[(size_t)(g0 + i) * b.L + vv], w0, acc[i]);
    }
    // warp sums of the group's rows by a reduce-scatter (rows past k are zeros)
    double d[G];
#pragma unroll
    for (int i = 0; i < G; ++i) d[i] = g0 + i < k ? (double)acc[i] : 0.0;
    int row = 0;
    WarpScatter<G, 16>::run(d, lane, row);
    if ((lane & (32 / G - 1)) == 0 && g0 + row < k) red[wid][g0 + row] = d[0];
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double d = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) d += red[q][threadIdx.x];
    out[threadIdx.x] = d;
  }
  __syncthreads();
}

// partials[item][i], i < k: |R|^2 over the chunk (kPhResid) or V_i . w with
// w = V_{j+1} (kPhArnoldi, kPhReorth; k = j + 2, per-thread sums in FP32 as in
// the single-slab mixed path, cross-thread sums in FP64 in a fixed order).
// WIDE = 0: 8 rows per pass, four resident blocks per SM, for the slots below
// kDotWideLen values; WIDE = 1: 16 rows per pass (twice the loads in flight per
// thread, two resident blocks per SM) for the longer slots, whose chunks are long
// streams.  A slot always takes the same kernel, so its sums do not depend on the
// other slots.
template <int WIDE>
__global__ void __launch_bounds__(kEngThreads, WIDE ? 2 : 4) eng_dot_kernel(const __grid_constant__ EngLaunch L) {
  __shared__ double red[kEngThreads / 32][kEngRows];
  const int n = *L.n_chunk_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const EngItem item = L.chunk_items[it];
    const int ph = L.ctl[item.slot].phase;
    if (ph != kPhResid && ph != kPhArnoldi && ph != kPhReorth) continue;
    const SlotBuf b = L.buf[item.slot];
    if ((b.L >= kDotWideLen) != (WIDE != 0) || !eng_runs(L, b)) continue;
    long long e0, e1;
    chunk_range(b, item.idx, &e0, &e1);
    const size_t blockvals = (size_t)b.s * b.nd * b.r;
    const size_t v0 = (size_t)e0 * blockvals, v1 = (size_t)e1 * blockvals;
    double* out = L.partials + (size_t)it * kEngRows;
    if (ph == kPhResid) {
      double a[1] = {0.0};
      for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) a[0] = fma(b.R[v], b.R[v], a[0]);
      block_reduce_store<1>(a, 1, red, out);
    } else {
      const int j = L.ctl[item.slot].j;
      dot_rows<WIDE ? 16 : 8>(b, v0, v1, j, j + 2, red, out);
    }
  }
}

// Shared-memory copy of what the controller of one slot touches in a tick.
struct CtlShared {
  double red[kCtlWideWarps][kEngRows];  // per-warp sums of each row
  double P[kEngRows];                      // the tick's reduced dot products
  double h[kEngRows + 1];                  // column j of H
  double cs[kEngRows], sn[kEngRows], sig[kEngRows + 1];
  double g[kEngRows + 1], y[kEngRows];
  double T[kEngRows * kEngRows];  // leading kd x kd block of H at the end of a cycle
  int kd;                         // > 0 when the cycle ended (the triangular solve follows)
};

// Givens column update and the end-of-cycle test (thread 0): column j of H in S.h, the
// earlier rotations in S.cs / S.sn.  Returns the number of basis vectors of the
// correction when the cycle ends, else 0.
__device__ int finish_column(SlotCtl& c, const SlotBuf& b, OpArgs<float>& a32, double r2, CtlShared& S) {
  const int j = c.j;
  if (!isfinite(r2)) {
    c.status = STDG_ERR_NAN;
    c.phase = kPhDone;
    c.upd = kUpdNone;
    return 0;
  }
  const double hn = sqrt(r2 > 0.0 ? r2 : 0.0);
  double* h = S.h;
  for (int i = 0; i < j; ++i) {
    const double t0 = S.cs[i] * h[i] + S.sn[i] * h[i + 1];
    h[i + 1] = -S.sn[i] * h[i] + S.cs[i] * h[i + 1];
    h[i] = t0;
  }
  double den = hypot(h[j], hn);
  if (den == 0.0) den = 1e-300;
  const double csj = h[j] / den, snj = hn / den;
  h[j] = den;
  c.cs[j] = csj;
  c.sn[j] = snj;
  for (int i = 0; i <= j; ++i) c.H[i * kEngRows + j] = h[i];
  const double gj = c.g[j];
  const double gj1 = -snj * gj;
  c.g[j + 1] = gj1;
  c.g[j] = csj * gj;
  c.gmres_its += 1;
  c.sig[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
  const bool done = fabs(gj1) <= c.tol || j + 1 >= c.m || hn <= 1e-300 * c.beta;
  if (done) {
    c.upd = kUpdSolve;
    c.upd_k = j + 1;
    c.newton_its += 1;
    c.phase = kPhResid;
    return j + 1;
  }
  // w -= V c (coefficients of this pass), z_{j+1} = P^-1 (w / |w|)
  c.upd = kUpdGSZ;
  c.upd_row = j + 1;
  c.upd_k = j + 1;
  c.zscale = c.sig[j + 1];
  c.j = j + 1;
  c.phase = kPhArnoldi;
  a32.v = b.Z + (size_t)(j + 1) * b.L;
  a32.out = b.V + (size_t)(j + 2) * b.L;
  return 0;
}

// One block per active slot (grid = number of active slots).  The block reduces the
// slot's per-item partial sums: warp w < W takes the groups of kA consecutive items
// w, w + W, w + 2W, ... (kA loads in flight per lane, lane = row), each warp combines its
// kA running sums in a fixed tree and the warps' sums are added in warp order, so the
// result does not depend on timing; W depends on the slot's item count only (not on the
// block size, which follows the largest slot of the batch).  Thread 0 then runs the
// Newton / Arnoldi logic on a shared-memory copy of the Givens data; at the end of a
// cycle the block stages H's leading block for the triangular solve.
__global__ void __launch_bounds__(32 * kCtlWideWarps) eng_control_kernel(const __grid_constant__ EngLaunch L) {
  constexpr int kA = 8;
  __shared__ CtlShared S;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int slot = L.active[blockIdx.x];
  SlotCtl& c = L.ctl[slot];
  const SlotBuf& b = L.buf[slot];
  const int W = b.nitems > kCtlWideItems ? kCtlWideWarps : kEngThreads / 32;
  const int ph = c.phase;
  if ((ph != kPhResid && ph != kPhArnoldi && ph != kPhReorth) || !eng_runs(L, b)) {
    if (threadIdx.x == 0) c.upd = kUpdNone;
    return;
  }
  const int k = ph == kPhResid ? 1 : c.j + 2;
  const int j = c.j;
  if (lane < k && wid < W) {
    const double* pp = L.partials + (size_t)b.item0 * kEngRows + lane;
    const int nit = b.nitems;
    double acc[kA];
#pragma unroll
    for (int a = 0; a < kA; ++a) acc[a] = 0.0;
    int q0 = wid * kA;
    for (; q0 + kA <= nit; q0 += W * kA) {
#pragma unroll
      for (int a = 0; a < kA; ++a) acc[a] += pp[(size_t)(q0 + a) * kEngRows];
    }
#pragma unroll
    for (int a = 0; a < kA; ++a)
      if (q0 + a < nit) acc[a] += pp[(size_t)(q0 + a) * kEngRows];
    S.red[wid][lane] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
  if (ph != kPhResid) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      S.cs[i] = c.cs[i];
      S.sn[i] = c.sn[i];
    }
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      S.sig[i] = c.sig[i];
      if (ph == kPhReorth) S.h[i] = c.H[i * kEngRows + j];
    }
  }
  if (threadIdx.x == 0) S.kd = 0;
  __syncthreads();
  if (threadIdx.x < k) {
    double d = 0.0;
    for (int q = 0; q < W; ++q) d += S.red[q][threadIdx.x];
    S.P[threadIdx.x] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* P = S.P;
    OpArgs<float>& a32 = L.a32[slot];
    if (ph == kPhResid) {
      const double res = sqrt(P[0]);
      c.resid_evals += 1;
      c.res = res;
      if (c.resid_evals == 1) {
        c.res0 = res;
        c.target = fmax(c.rtol * res, c.atol);
      }
      if (!isfinite(res)) {
        c.status = STDG_ERR_NAN;
        c.phase = kPhDone;
        c.upd = kUpdNone;
      } else if (res <= c.target) {
        c.status = STDG_OK;
        c.phase = kPhDone;
        c.upd = kUpdExtract;
      } else if (c.newton_its >= c.newton_maxit) {
        c.status = STDG_ERR_NOT_CONVERGED;
        c.phase = kPhDone;
        c.upd = kUpdExtract;
      } else {
        c.beta = res;
        c.tol = c.gmres_rtol * res;
        c.sig[0] = -1.0 / res;  // V_0 holds R, v_0 = -R / |R|
        for (int i = 0; i <= kEngRows; ++i) c.g[i] = 0.0;
        c.g[0] = res;
        c.j = 0;
        c.upd = kUpdInit;
        c.zscale = c.sig[0];
        c.phase = kPhArnoldi;
        a32.v = b.Z;
        a32.out = b.V + b.L;
      }
    } else if (ph == kPhArnoldi) {
      c.jv_evals += 1;
      const double w2 = P[j + 1];
      double h2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        const double h = S.sig[i] * P[i];
        S.h[i] = h;
        h2 += h * h;
        c.coef[i] = S.sig[i] * h;
      }
      const double r2 = w2 - h2;
      if (!(r2 > 0.01 * w2) && isfinite(r2)) {
        // strong cancellation: apply this projection, then project once more
        for (int i = 0; i <= j; ++i) c.H[i * kEngRows + j] = S.h[i];
        c.phase = kPhReorth;
        c.upd = kUpdGS;
        c.upd_row = j + 1;
        c.upd_k = j + 1;
      } else {
        S.kd = finish_column(c, b, a32, r2, S);
      }
    } else {
      double e2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        const double h = S.sig[i] * P[i];
        S.h[i] += h;
        e2 += h * h;
        c.coef[i] = S.sig[i] * h;
      }
      S.kd = finish_column(c, b, a32, P[j + 1] - e2, S);
    }
  }
  __syncthreads();
  const int kd = S.kd;
  if (kd == 0) return;
  // end of the cycle: y = H^-1 g (upper triangular), the update is U += sum_i y_i z_i
  for (int t = threadIdx.x; t < kd * kd; t += blockDim.x) {
    const int i = t / kd, q = t % kd;
    if (q >= i) S.T[i * kEngRows + q] = q == kd - 1 ? S.h[i] : c.H[i * kEngRows + q];
  }
  for (int i = threadIdx.x; i < kd; i += blockDim.x) S.g[i] = c.g[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = kd - 1; i >= 0; --i) {
      double acc = S.g[i];
      for (int q = i + 1; q < kd; ++q) acc -= S.T[i * kEngRows + q] * S.y[q];
      S.y[i] = acc / S.T[i * kEngRows + i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kd; i += blockDim.x) c.coef[i] = S.y[i];
}

// sum_{i<k} c_i X[i * ld] with four independent partial sums (loads of four rows in
// flight), combined as (s0 + s1) + (s2 + s3).
__device__ __forceinline__ float rows_sum(const float* c, const float* X, size_t ld, int k) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int i = 0;
  for (; i + 8 <= k; i += 8) {  // eight rows in flight
    const float x0 = X[(size_t)i * ld], x1 = X[(size_t)(i + 1) * ld], x2 = X[(size_t)(i + 2) * ld],
                x3 = X[(size_t)(i + 3) * ld], x4 = X[(size_t)(i + 4) * ld], x5 = X[(size_t)(i + 5) * ld],
                x6 = X[(size_t)(i + 6) * ld], x7 = X[(size_t)(i + 7) * ld];
    s0 = fmaf(c[i + 4], x4, fmaf(c[i], x0, s0));
    s1 = fmaf(c[i + 5], x5, fmaf(c[i + 1], x1, s1));
    s2 = fmaf(c[i + 6], x6, fmaf(c[i + 2], x2, s2));
    s3 = fmaf(c[i + 7], x7, fmaf(c[i + 3], x3, s3));
  }
  for (; i + 4 <= k; i += 4) {
    s0 = fmaf(c[i], X[(size_t)i * ld], s0);
    s1 = fmaf(c[i + 1], X[(size_t)(i + 1) * ld], s1);
    s2 = fmaf(c[i + 2], X[(size_t)(i + 2) * ld], s2);
    s3 = fmaf(c[i + 3], X[(size_t)(i + 3) * ld], s3);
  }
  for (; i < k; ++i) s0 = fmaf(c[i], X[(size_t)i * ld], s0);
  return (s0 + s1) + (s2 + s3);
}

// rows_sum for four consecutive values (16-byte loads of each row), the same association per value.
__device__ __forceinline__ float4 rows_sum4(const float* c, const float* X, size_t ld, int k) {
  float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
  auto f4 = [&](int i) { return *reinterpret_cast<const float4*>(X + (size_t)i * ld); };
  auto acc = [](float4& s, float ci, const float4& x) {
    s.x = fmaf(ci, x.x, s.x);
    s.y = fmaf(ci, x.y, s.y);
    s.z = fmaf(ci, x.z, s.z);
    s.w = fmaf(ci, x.w, s.w);
  };
  int i = 0;
  for (; i + 8 <= k; i += 8) {
    const float4 x0 = f4(i), x1 = f4(i + 1), x2 = f4(i + 2), x3 = f4(i + 3), x4 = f4(i + 4), x5 = f4(i + 5),
                 x6 = f4(i + 6), x7 = f4(i + 7);
    acc(s0, c[i], x0);
    acc(s0, c[i + 4], x4);
    acc(s1, c[i + 1], x1);
    acc(s1, c[i + 5], x5);
    acc(s2, c[i + 2], x2);
    acc(s2, c[i + 6], x6);
    acc(s3, c[i + 3], x3);
    acc(s3, c[i + 7], x7);
  }
  for (; i + 4 <= k; i += 4) {
    acc(s0, c[i], f4(i));
    acc(s1, c[i + 1], f4(i + 1));
    acc(s2, c[i + 2], f4(i + 2));
    acc(s3, c[i + 3], f4(i + 3));
  }
  for (; i < k; ++i) acc(s0, c[i], f4(i));
  return make_float4((s0.x + s1.x) + (s2.x + s3.x), (s0.y + s1.y) + (s2.y + s3.y), (s0.z + s1.z) + (s2.z + s3.z),
                     (s0.w + s1.w) + (s2.w + s3.w));
}

// Updates that need no per-node s x s block (Init, GS, GSZ of slots without point blocks, and the
// Newton update): value by value over the chunk's range [v0, v1), in 16-byte words over the
// aligned body when the rows start on 16 bytes (and, with the temporal-mass scaling, each word
// lies in one temporal node: nd r % 4 == 0).  z_m = zscale x_m / omega_m for temporal-mass slots.
__device__ __forceinline__ void linear_update(const EngLaunch& L, const SlotBuf& b, int slot, int mode, int k,
                                              int row, float zs, const float* cf, long long e0, long long e1) {
  const int tnode = b.nd * b.r;
  const size_t blockvals = (size_t)b.s * tnode;
  const size_t v0 = (size_t)e0 * blockvals, v1 = (size_t)e1 * blockvals;
  const bool scale = b.pbtm && (mode == kUpdInit || mode == kUpdGSZ);
  const float* iw = L.a32[slot].inv_omega;
  float* w = mode == kUpdInit ? b.V : b.V + (size_t)row * b.L;
  float* z = mode == kUpdInit ? b.Z : b.Z + (size_t)row * b.L;
  const bool vec = b.vec4 && (!scale || tnode % 4 == 0);
  size_t a0 = v0, a1 = v0;
  if (vec) {
    a0 = (v0 + 3) & ~(size_t)3;
    if (a0 > v1) a0 = v1;
    a1 = a0 + ((v1 - a0) & ~(size_t)3);
  }
  // temporal node of value v (v0 starts an element block; a chunk holds at most 65,536 values or
  // one element block)
  auto tnode_of = [&](size_t v) { return ((int)(v - v0) / tnode) % b.s; };
  for (size_t q = a0 / 4 + threadIdx.x; q < a1 / 4; q += blockDim.x) {
    const size_t v = 4 * q;
    if (mode == kUpdSolve) {
      const float4 acc = rows_sum4(cf, b.Z + v, b.L, k);
      double2* U2 = reinterpret_cast<double2*>(b.U + v);
      double2 u01 = U2[0], u23 = U2[1];
      u01.x += (double)acc.x;
      u01.y += (double)acc.y;
      u23.x += (double)acc.z;
      u23.y += (double)acc.w;
      U2[0] = u01;
      U2[1] = u23;
      *reinterpret_cast<float4*>(b.U32 + v) = make_float4((float)u01.x, (float)u01.y, (float)u23.x, (float)u23.y);
      continue;
    }
    float4 x;
    if (mode == kUpdInit) {
      const double2* R2 = reinterpret_cast<const double2*>(b.R + v);
      const double2 r01 = R2[0], r23 = R2[1];
      x = make_float4((float)r01.x, (float)r01.y, (float)r23.x, (float)r23.y);
    } else {
      const float4 acc = rows_sum4(cf, b.V + v, b.L, k);
      const float4 wv = *reinterpret_cast<const float4*>(w + v);
      x = make_float4(wv.x - acc.x, wv.y - acc.y, wv.z - acc.z, wv.w - acc.w);
    }
    *reinterpret_cast<float4*>(w + v) = x;
    if (scale) {
      const float f = iw[tnode_of(v)];
      *reinterpret_cast<float4*>(z + v) =
          make_float4(zs * x.x * f, zs * x.y * f, zs * x.z * f, zs * x.w * f);
    }
  }
  for (size_t t = threadIdx.x; t < (a0 - v0) + (v1 - a1); t += blockDim.x) {  // head, then tail
    const size_t v = t < a0 - v0 ? v0 + t : a1 + (t - (a0 - v0));
    if (mode == kUpdSolve) {
      const double u = b.U[v] + (double)rows_sum(cf, b.Z + v, b.L, k);
      b.U[v] = u;
      b.U32[v] = (float)u;
      continue;
    }
    const float x = mode == kUpdInit ? (float)b.R[v] : w[v] - rows_sum(cf, b.V + v, b.L, k);
    w[v] = x;
    if (scale) z[v] = zs * x * iw[tnode_of(v)];
  }
}

// Vector update of one tick.  Point-block slots (Init, GSZ) and the extraction of u^{n+1}:
// thread per (element, value q of a temporal node's block) of the chunk; the s temporal values
// of q are handled together so that z = (P^-1 (x) I_r) x is formed in registers.  Everything
// else: linear_update.
__global__ void __launch_bounds__(kEngThreads) eng_update_kernel(const __grid_constant__ EngLaunch L) {
  __shared__ float cf[kEngRows];
  const int n = *L.n_chunk_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const EngItem item = L.chunk_items[it];
    const SlotCtl& c = L.ctl[item.slot];
    const int mode = c.upd;
    if (mode == kUpdNone) continue;
    const SlotBuf b = L.buf[item.slot];
    const int k = c.upd_k;
    if ((mode == kUpdGS || mode == kUpdGSZ || mode == kUpdSolve) && threadIdx.x < k)
      cf[threadIdx.x] = (float)c.coef[threadIdx.x];
    __syncthreads();
    const int row = c.upd_row;
    const float zs = (float)c.zscale;
    long long e0, e1;
    chunk_range(b, item.idx, &e0, &e1);
    const bool pb_apply = (mode == kUpdInit || mode == kUpdGSZ) && !b.pbtm && !b.kron && !b.fdm;
    if (mode != kUpdExtract && !pb_apply) {
      linear_update(L, b, item.slot, mode, k, row, zs, cf, e0, e1);
      __syncthreads();
      continue;
    }
    const int s = b.s, nd = b.nd, r = b.r;
    const int tnode = nd * r;
    const int total = (int)(e1 - e0) * tnode;  // a chunk holds at most 65,536 values or one element block
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const size_t e = (size_t)e0 + t / tnode;
      const int q = t % tnode;
      const int node = q / r;
      const size_t base = e * s * tnode + q;  // (e, m = 0, q)
      if (mode == kUpdExtract) {
        b.uprev[e * tnode + q] = b.U[base + (size_t)(s - 1) * tnode];
        continue;
      }
      float x[kMaxS];
      float* zout;
      if (mode == kUpdInit) {
        for (int m = 0; m < s; ++m) {
          const float v = (float)b.R[base + (size_t)m * tnode];
          b.V[base + (size_t)m * tnode] = v;
          x[m] = zs * v;
        }
        zout = b.Z;
      } else {
        float* w = b.V + (size_t)row * b.L;
        for (int m = 0; m < s; ++m) {
          const size_t o = base + (size_t)m * tnode;
          const float acc = w[o] - rows_sum(cf, b.V + o, b.L, k);
          w[o] = acc;
          x[m] = zs * acc;
        }
        zout = b.Z + (size_t)row * b.L;
      }
      const float* P = b.Pinv + (e * s * s) * nd + node;
      for (int m = 0; m < s; ++m) {
        float zv = 0.f;
        for (int jj = 0; jj < s; ++jj) zv = fmaf(P[(size_t)(m * s + jj) * nd], x[jj], zv);
        zout[base + (size_t)m * tnode] = zv;
      }
    }
    __syncthreads();
  }
}

// z = P^-1 (zscale w) with the element tensor-product preconditioner of scalar
// equations.  Per element, with A_a the element-local 1D operator along e_a (the
// interior penalty form with the neighbours set to zero, plus the upwind
// dissipation lambda/(h_a w_end) at the end nodes), A_a = V_a Lambda_a V_a^-1:
//   P = T (x) I - dt/2 M_tau (x) (A_x (+) A_y)
//     = (I (x) V_y (x) V_x) [block-diag over modes k: P_k = T - dt/2 Lambda_k M_tau]
//       (I (x) V_y^-1 (x) V_x^-1),
// so z is three contractions: V^-1 along x and y, P_k^-1 (s x s) per mode, V back.
// The elements of a chunk are processed in groups held in shared memory.
__global__ void __launch_bounds__(kEngThreads) eng_kron_kernel(const __grid_constant__ EngLaunch L) {
  constexpr int kBuf = 2048;  // floats per ping-pong buffer
  constexpr int kKd = 4 * kMaxN * kMaxN + kMaxN * kMaxN * kMaxS * kMaxS;  // 2D data of the largest class
  __shared__ float sa[kBuf], sb2[kBuf];
  __shared__ float skd[kKd];
  const int nitems = *L.n_chunk_items;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const EngItem item = L.chunk_items[it];
    const SlotBuf b = L.buf[item.slot];
    if (!b.kron) continue;
    const SlotCtl& c = L.ctl[item.slot];
    const int mode = c.upd;
    if (mode != kUpdInit && mode != kUpdGSZ) continue;
    const int row = mode == kUpdInit ? 0 : c.upd_row;
    const float zs = (float)c.zscale;
    const float* src = b.V + (size_t)row * b.L;
    float* dst = b.Z + (size_t)row * b.L;
    const int n = b.n, s = b.s, nd = b.nd, dim = b.dim;
    const int per = s * nd;  // values of one element (r = 1)
    const int E = kBuf / per > 0 ? kBuf / per : 1;
    const int nkd = 4 * n * n + nd * s * s;
    for (int i = threadIdx.x; i < nkd; i += blockDim.x) skd[i] = b.kdat[i];
    __syncthreads();
    const float* Vxi = skd;
    const float* Vx = Vxi + n * n;
    const float* Vyi = Vx + n * n;
    const float* Vy = Vyi + n * n;
    const float* Pk = Vy + n * n;
    long long e0, e1;
    chunk_range(b, item.idx, &e0, &e1);
    for (long long eg = e0; eg < e1; eg += E) {
      const int ne = (int)((e1 - eg) < E ? (e1 - eg) : E);
      const int tot = ne * per;
      for (int t = threadIdx.x; t < tot; t += blockDim.x) sa[t] = zs * src[(size_t)eg * per + t];
      __syncthreads();
      // forward along x: sb2[., iy, kx] = sum_ix Vx^-1[kx][ix] sa[., iy, ix]
      for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int kx = t % n, base = t - kx;
        float acc = 0.f;
        for (int ix = 0; ix < n; ++ix) acc = fmaf(Vxi[kx * n + ix], sa[base + ix], acc);
        sb2[t] = acc;
      }
      __syncthreads();
      const float* cur = sb2;
      float* nxt = sa;
      if (dim == 2) {  // forward along y
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
          const int kx = t % n, ky = (t / n) % n, base = t - (t % nd);
          float acc = 0.f;
          for (int iy = 0; iy < n; ++iy) acc = fmaf(Vyi[ky * n + iy], cur[base + iy * n + kx], acc);
          nxt[t] = acc;
        }
        __syncthreads();
        cur = sa;
        nxt = sb2;
      }
      // per mode k: z_m = sum_j (P_k^-1)[m][j] y_j
      for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int k = t % nd, m = (t / nd) % s, el = t / per;
        const float* P = Pk + ((size_t)k * s + m) * s;
        float acc = 0.f;
        for (int j = 0; j < s; ++j) acc = fmaf(P[j], cur[el * per + j * nd + k], acc);
        nxt[t] = acc;
      }
      __syncthreads();
      {
        const float* c2 = nxt;
        float* n2 = const_cast<float*>(cur);
        if (dim == 2) {  // back along y: n2[., iy, kx] = sum_ky Vy[iy][ky] c2[., ky, kx]
          for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            const int kx = t % n, iy = (t / n) % n, base = t - (t % nd);
            float acc = 0.f;
            for (int ky = 0; ky < n; ++ky) acc = fmaf(Vy[iy * n + ky], c2[base + ky * n + kx], acc);
            n2[t] = acc;
          }
          __syncthreads();
          const float* tmp = c2;
          c2 = n2;
          n2 = const_cast<float*>(tmp);
        }
        // back along x, straight to global memory
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
          const int ix = t % n, base = t - ix;
          float acc = 0.f;
          for (int kx = 0; kx < n; ++kx) acc = fmaf(Vx[ix * n + kx], c2[base + kx], acc);
          dst[(size_t)eg * per + t] = acc;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void eng_tick_kernel(int* tick) { *tick += 1; }

__global__ void eng_fill_kernel(double* U, float* U32, size_t L, int r, Fill5 st) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += stride) {
    const double v = st.v[i % r];
    U[i] = v;
    U32[i] = (float)v;
  }
}

__global__ void eng_init_kernel(const SlotBuf b) {
  const int tnode = b.nd * b.r;
  const size_t total = (size_t)b.nelem * b.s * tnode;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const size_t e = idx / ((size_t)b.s * tnode);
    const size_t q = idx % tnode;
    const double u = b.uprev[e * tnode + q];
    b.U[idx] = u;
    b.U32[idx] = (float)u;
  }
}

}  // namespace

cudaError_t eng_tick_tail(const EngLaunch& L, cudaStream_t st) {
  if (L.n_active <= 0) return cudaSuccess;
  eng_dot_kernel<0><<<L.chunk_grid, kEngThreads, 0, st>>>(L);
  if (L.any_wide) eng_dot_kernel<1><<<L.chunk_grid, kEngThreads, 0, st>>>(L);
  eng_control_kernel<<<L.n_active, L.ctl_threads, 0, st>>>(L);
  eng_update_kernel<<<L.chunk_grid, kEngThreads, 0, st>>>(L);
  if (L.any_kron) eng_kron_kernel<<<L.chunk_grid, kEngThreads, 0, st>>>(L);
  if (L.any_fdm) {
    const cudaError_t e = eng_fdm_apply(L, st);
    if (e != cudaSuccess) return e;
  }
  eng_tick_kernel<<<1, 1, 0, st>>>(L.tick);
  return cudaGetLastError();
}

cudaError_t eng_fill_state(double* U, float* U32, size_t L, int r, const Fill5& state, cudaStream_t st) {
  size_t blocks = (L + 255) / 256;
  if (blocks > 2432) blocks = 2432;
  eng_fill_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, st>>>(U, U32, L, r, state);
  return cudaGetLastError();
}

cudaError_t eng_init_slot(const SlotBuf& b, cudaStream_t st) {
  size_t total = (size_t)b.nelem * b.s * b.nd * b.r;
  size_t blocks = (total + 255) / 256;
  if (blocks > 2432) blocks = 2432;
  eng_init_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, st>>>(b);
  return cudaGetLastError();
}

}  // namespace stdg
