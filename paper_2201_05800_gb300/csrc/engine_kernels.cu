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

// V_i . w over [v0, v1) for i < k, in passes over groups of 8 rows (few registers, so many
// blocks stay resident; w is re-read from L1/L2 once per group), two values per thread and
// iteration.  Per-warp sums of each row go to red[warp][row]; then one fixed-order sum.
__device__ __forceinline__ void dot_rows(const SlotBuf& b, size_t v0, size_t v1, int j, int k,
                                         double (*red)[kEngRows], double* out) {
  constexpr int G = 8;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float* w = b.V + (size_t)(j + 1) * b.L;
  for (int g0 = 0; g0 < k; g0 += G) {
    float acc[G];
#pragma unroll
    for (int i = 0; i < G; ++i) acc[i] = 0.f;
    const size_t step = (size_t)2 * blockDim.x;
    size_t v = v0 + threadIdx.x;
    for (; v + blockDim.x < v1; v += step) {
      const float w0 = w[v], w1 = w[v + blockDim.x];
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (g0 + i < k) {
          const float* Vi = b.V + (size_t)(g0 + i) * b.L;
          acc[i] = fmaf(Vi[v + blockDim.x], w1, fmaf(Vi[v], w0, acc[i]));
        }
    }
    if (v < v1) {
      const float w0 = w[v];
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (g0 + i < k) acc[i] = fmaf(b.V[(size_t)(g0 + i) * b.L + v], w0, acc[i]);
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
__global__ void __launch_bounds__(kEngThreads, 4) eng_dot_kernel(const __grid_constant__ EngLaunch L) {
  __shared__ double red[kEngThreads / 32][kEngRows];
  const int n = *L.n_chunk_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const EngItem item = L.chunk_items[it];
    const int ph = L.ctl[item.slot].phase;
    if (ph != kPhResid && ph != kPhArnoldi && ph != kPhReorth) continue;
    const SlotBuf b = L.buf[item.slot];
    if (!eng_runs(L, b)) continue;
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
      dot_rows(b, v0, v1, j, j + 2, red, out);
    }
  }
}

// Givens column update and the end-of-cycle test (lane 0 of the slot's warp).
__device__ void finish_column(SlotCtl& c, const SlotBuf& b, OpArgs<float>& a32, double r2) {
  const int j = c.j;
  if (!isfinite(r2)) {
    c.status = STDG_ERR_NAN;
    c.phase = kPhDone;
    c.upd = kUpdNone;
    return;
  }
  const double hn = sqrt(r2 > 0.0 ? r2 : 0.0);
  double* H = c.H;
  for (int i = 0; i < j; ++i) {
    const double t0 = c.cs[i] * H[i * kEngRows + j] + c.sn[i] * H[(i + 1) * kEngRows + j];
    H[(i + 1) * kEngRows + j] = -c.sn[i] * H[i * kEngRows + j] + c.cs[i] * H[(i + 1) * kEngRows + j];
    H[i * kEngRows + j] = t0;
  }
  double den = hypot(H[j * kEngRows + j], hn);
  if (den == 0.0) den = 1e-300;
  c.cs[j] = H[j * kEngRows + j] / den;
  c.sn[j] = hn / den;
  H[j * kEngRows + j] = den;
  c.g[j + 1] = -c.sn[j] * c.g[j];
  c.g[j] = c.cs[j] * c.g[j];
  c.gmres_its += 1;
  c.sig[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
  const bool done = fabs(c.g[j + 1]) <= c.tol || j + 1 >= c.m || hn <= 1e-300 * c.beta;
  if (done) {
    // y = H^-1 g (upper triangular), U += sum_i y_i z_i
    const int kd = j + 1;
    double y[kEngRows];
    for (int i = kd - 1; i >= 0; --i) {
      double acc = c.g[i];
      for (int q = i + 1; q < kd; ++q) acc -= H[i * kEngRows + q] * y[q];
      y[i] = acc / H[i * kEngRows + i];
    }
    for (int i = 0; i < kd; ++i) c.coef[i] = y[i];
    c.upd = kUpdSolve;
    c.upd_k = kd;
    c.newton_its += 1;
    c.phase = kPhResid;
  } else {
    // w -= V c (coefficients of this pass), z_{j+1} = P^-1 (w / |w|)
    c.upd = kUpdGSZ;
    c.upd_row = j + 1;
    c.upd_k = j + 1;
    c.zscale = c.sig[j + 1];
    c.j = j + 1;
    c.phase = kPhArnoldi;
    a32.v = b.Z + (size_t)(j + 1) * b.L;
    a32.out = b.V + (size_t)(j + 2) * b.L;
  }
}

// One warp per active slot.
__global__ void __launch_bounds__(kEngThreads) eng_control_kernel(const __grid_constant__ EngLaunch L) {
  __shared__ double sp[kEngThreads / 32][kEngRows];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= L.n_active) return;
  const int slot = L.active[g];
  SlotCtl& c = L.ctl[slot];
  const SlotBuf& b = L.buf[slot];
  const int ph = c.phase;
  if ((ph != kPhResid && ph != kPhArnoldi && ph != kPhReorth) || !eng_runs(L, b)) {
    if (lane == 0) c.upd = kUpdNone;
    return;
  }
  // lane i sums row i over the slot's work items in a fixed order (four interleaved partial
  // sums, combined as (s0 + s1) + (s2 + s3)); rows are consecutive in memory per item
  const int k = ph == kPhResid ? 1 : c.j + 2;
  if (lane < k) {
    const double* pp = L.partials + (size_t)b.item0 * kEngRows + lane;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int q = 0;
    for (; q + 4 <= b.nitems; q += 4) {
      s0 += pp[(size_t)q * kEngRows];
      s1 += pp[(size_t)(q + 1) * kEngRows];
      s2 += pp[(size_t)(q + 2) * kEngRows];
      s3 += pp[(size_t)(q + 3) * kEngRows];
    }
    for (; q < b.nitems; ++q) s0 += pp[(size_t)q * kEngRows];
    sp[wid][lane] = (s0 + s1) + (s2 + s3);
  }
  __syncwarp();
  if (lane != 0) return;
  const double* P = sp[wid];
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
    return;
  }
  const int j = c.j;
  double* H = c.H;
  if (ph == kPhArnoldi) {
    c.jv_evals += 1;
    const double w2 = P[j + 1];
    double h2 = 0.0;
    for (int i = 0; i <= j; ++i) {
      const double h = c.sig[i] * P[i];
      H[i * kEngRows + j] = h;
      h2 += h * h;
      c.coef[i] = c.sig[i] * h;
    }
    const double r2 = w2 - h2;
    if (!(r2 > 0.01 * w2) && isfinite(r2)) {
      // strong cancellation: apply this projection, then project once more
      c.phase = kPhReorth;
      c.upd = kUpdGS;
      c.upd_row = j + 1;
      c.upd_k = j + 1;
      return;
    }
    finish_column(c, b, a32, r2);
  } else {
    double e2 = 0.0;
    for (int i = 0; i <= j; ++i) {
      const double h = c.sig[i] * P[i];
      H[i * kEngRows + j] += h;
      e2 += h * h;
      c.coef[i] = c.sig[i] * h;
    }
    finish_column(c, b, a32, P[j + 1] - e2);
  }
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

// Vector update of one tick.  Thread per (element, value q of a temporal
// node's block) of the chunk; the s temporal values of q are handled together
// so that z = (P^-1 (x) I_r) x is formed in registers.
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
    const int s = b.s, nd = b.nd, r = b.r;
    const int tnode = nd * r;
    const size_t total = (size_t)(e1 - e0) * tnode;
    for (size_t t = threadIdx.x; t < total; t += blockDim.x) {
      const size_t e = (size_t)e0 + t / tnode;
      const int q = (int)(t % tnode);
      const int node = q / r;
      const size_t base = e * s * tnode + q;  // (e, m = 0, q)
      float x[kMaxS];
      bool apply_z = false;
      float* zout = nullptr;
      if (mode == kUpdInit) {
        for (int m = 0; m < s; ++m) {
          const float v = (float)b.R[base + (size_t)m * tnode];
          b.V[base + (size_t)m * tnode] = v;
          x[m] = zs * v;
        }
        apply_z = true;
        zout = b.Z;
      } else if (mode == kUpdGS || mode == kUpdGSZ) {
        float* w = b.V + (size_t)row * b.L;
        for (int m = 0; m < s; ++m) {
          const size_t o = base + (size_t)m * tnode;
          const float acc = w[o] - rows_sum(cf, b.V + o, b.L, k);
          w[o] = acc;
          x[m] = zs * acc;
        }
        apply_z = mode == kUpdGSZ;
        zout = b.Z + (size_t)row * b.L;
      } else if (mode == kUpdSolve) {
        for (int m = 0; m < s; ++m) {
          const size_t o = base + (size_t)m * tnode;
          const float acc = rows_sum(cf, b.Z + o, b.L, k);
          const double u = b.U[o] + (double)acc;
          b.U[o] = u;
          b.U32[o] = (float)u;
        }
      } else if (mode == kUpdExtract) {
        b.uprev[e * tnode + q] = b.U[base + (size_t)(s - 1) * tnode];
      }
      if (apply_z && b.pbtm) {  // temporal-mass scaling: z_m = x_m / omega_m
        const OpArgs<float>& a = L.a32[item.slot];
        for (int m = 0; m < s; ++m) zout[base + (size_t)m * tnode] = x[m] * a.inv_omega[m];
      } else if (apply_z && !b.kron && !b.fdm) {  // Kron / fdm slots: z is formed by their own kernels
        const float* P = b.Pinv + (e * s * s) * nd + node;
        for (int m = 0; m < s; ++m) {
          float z = 0.f;
          for (int jj = 0; jj < s; ++jj) z = fmaf(P[(size_t)(m * s + jj) * nd], x[jj], z);
          zout[base + (size_t)m * tnode] = z;
        }
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
  eng_dot_kernel<<<L.chunk_grid, kEngThreads, 0, st>>>(L);
  const int warps_per_block = kEngThreads / 32;
  eng_control_kernel<<<(L.n_active + warps_per_block - 1) / warps_per_block, kEngThreads, 0, st>>>(L);
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
