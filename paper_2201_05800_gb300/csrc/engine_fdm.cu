// Global fast-diagonalisation preconditioner of the batch engine for scalar
// slots on periodic grids (host data: fdm_host.h).  With W the temporal LGL
// weights, C = D_tau^T M_tau - e_s e_s^T and A_x, A_y the periodic 1D operators
// of the interior penalty form plus the upwind dissipation (the linear part of
// the spatial Jacobian that the preconditioner keeps),
//   P = C (x) I - dt/2 M_tau (x) (A_x (+) A_y),
// whose inverse is applied exactly by diagonalising both 1D operators:
//   x pass      along every x-line: FFT over the elements (radix 2), then the
//               per-mode eigenvector transform F_x (n x n)       -> scratch X
//   y pass      per x-mode (kx, jx): the same along y, then per spatial mode
//               the s x s solve (C - dt/2 (lam_x + lam_y) M_tau) z = x with
//               partial pivoting, and the inverse y transform        (in place)
//   x^-1 pass   inverse eigenvector transform and inverse FFT along x -> z
// z = P^-1 (zscale w) is written to the slot's preconditioned direction.  All
// arithmetic is FP32 (complex); flexible GMRES uses the stored z as it is.
#include <math.h>

#include "engine.cuh"

namespace stdg {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ int bitrev(int i, int logk) {
  return logk ? (int)(__brev((unsigned)i) >> (32 - logk)) : 0;
}

// In-place radix-2 FFT of nb batches of K = 2^logk values held in bit-reversed order,
// A[b * K + k]; tw[t] = exp(-2 pi i t / K); inverse: conjugate twiddles (no scaling).
__device__ void fft_batched(float2* A, int nb, int logk, const float2* tw, bool inverse) {
  const int K = 1 << logk;
  for (int len = 2; len <= K; len <<= 1) {
    const int half = len >> 1, step = K / len;
    const int nbf = nb * (K >> 1);
    for (int t = threadIdx.x; t < nbf; t += blockDim.x) {
      const int b = t / (K >> 1), r = t % (K >> 1);
      const int blk = r / half, j = r % half;
      const int i0 = b * K + blk * len + j, i1 = i0 + half;
      const float2 w = tw[j * step];
      const float2 v = inverse ? cmulc(A[i1], w) : cmul(A[i1], w);
      const float2 u = A[i0];
      A[i0] = cadd(u, v);
      A[i1] = csub(u, v);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool fdm_wants(const EngLaunch& L, const EngItem& it, int* row, float* zs) {
  const SlotBuf& b = L.buf[it.slot];
  if (!b.fdm) return false;
  const SlotCtl& c = L.ctl[it.slot];
  if (c.upd != kUpdInit && c.upd != kUpdGSZ) return false;
  *row = c.upd == kUpdInit ? 0 : c.upd_row;
  *zs = (float)c.zscale;
  return true;
}

// x pass: item (slot, ey * s + m); A[(iy n + ix) Kx + k] in shared memory.
__global__ void __launch_bounds__(256) eng_fdm_x_kernel(const __grid_constant__ EngLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* A = reinterpret_cast<float2*>(smem_raw);
  const int nitems = *L.n_fdm_rows;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const EngItem item = L.fdm_rows[it];
    int row;
    float zs;
    if (!fdm_wants(L, item, &row, &zs)) continue;
    const SlotBuf& b = L.buf[item.slot];
    const int n = b.n, ny = b.fny, Kx = b.fkx, Ky = b.fky, s = b.s, nd = b.nd;
    const int ey = item.idx / s, m = item.idx % s;
    const int nb = ny * n;
    const float* src = b.V + (size_t)row * b.L;
    const float2* tw = reinterpret_cast<const float2*>(b.fdat + b.f_twx);
    const float2* F = reinterpret_cast<const float2*>(b.fdat + b.f_Fx);
    for (int t = threadIdx.x; t < nb * Kx; t += blockDim.x) {
      const int node = t % nd, ex = t / nd;  // coalesced along the element's node block
      const float x = zs * src[((size_t)(ey * Kx + ex) * s + m) * nd + node];
      A[node * Kx + bitrev(ex, b.flogx)] = make_float2(x, 0.f);
    }
    __syncthreads();
    fft_batched(A, nb, b.flogx, tw, false);
    // per mode k: c[k][jx][iy] = (1/Kx) sum_ix F_k[jx][ix] A[iy n + ix][k]
    const float inv = 1.0f / Kx;
    for (int t = threadIdx.x; t < Kx * n * ny; t += blockDim.x) {
      const int iy = t % ny, jx = (t / ny) % n, k = t / (ny * n);
      float2 acc = make_float2(0.f, 0.f);
      const float2* Fk = F + ((size_t)k * n + jx) * n;
      for (int ix = 0; ix < n; ++ix) acc = cadd(acc, cmul(Fk[ix], A[(iy * n + ix) * Kx + k]));
      b.fx[(((size_t)k * n + jx) * s + m) * Ky * ny + ey * ny + iy] = make_float2(acc.x * inv, acc.y * inv);
    }
    __syncthreads();
  }
}

// y pass and temporal solves: item (slot, kx n + jx); A[(m ny + iy) Ky + k], Bf[(ky ny + jy) s + m].
__global__ void __launch_bounds__(256) eng_fdm_y_kernel(const __grid_constant__ EngLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nitems = *L.n_fdm_cols;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const EngItem item = L.fdm_cols[it];
    int row;
    float zs;
    if (!fdm_wants(L, item, &row, &zs)) continue;
    const SlotBuf& b = L.buf[item.slot];
    const OpArgs<float>& a = L.a32[item.slot];
    const int n = b.n, ny = b.fny, Ky = b.fky, s = b.s;
    const int kx = item.idx / n, jx = item.idx % n;
    const int nbv = s * ny * Ky;
    float2* A = reinterpret_cast<float2*>(smem_raw);
    float2* Bf = A + nbv;
    float2* base = b.fx + ((size_t)(kx * n + jx) * s) * Ky * ny;
    const float2* tw = reinterpret_cast<const float2*>(b.fdat + b.f_twy);
    const float2* F = reinterpret_cast<const float2*>(b.fdat + b.f_Fy);
    const float2* Bk = reinterpret_cast<const float2*>(b.fdat + b.f_By);
    const float lx = b.fdat[b.f_lx + kx * n + jx];
    const float* ly = b.fdat + b.f_ly;
    for (int t = threadIdx.x; t < nbv; t += blockDim.x) {
      const int iy = t % ny, ey = (t / ny) % Ky, m = t / (ny * Ky);
      A[(m * ny + iy) * Ky + bitrev(ey, b.flogy)] = base[t];
    }
    __syncthreads();
    fft_batched(A, s * ny, b.flogy, tw, false);
    const float inv = 1.0f / Ky;
    for (int t = threadIdx.x; t < nbv; t += blockDim.x) {
      const int m = t % s, jy = (t / s) % ny, ky = t / (s * ny);
      float2 acc = make_float2(0.f, 0.f);
      const float2* Fk = F + ((size_t)ky * ny + jy) * ny;
      for (int iy = 0; iy < ny; ++iy) acc = cadd(acc, cmul(Fk[iy], A[(m * ny + iy) * Ky + ky]));
      Bf[t] = make_float2(acc.x * inv, acc.y * inv);  // t = (ky ny + jy) s + m
    }
    __syncthreads();
    // (C - mu M_tau) z = c per spatial mode, C[m][j] = (D_tau^T M_tau)[m][j] - [m = j = s-1]
    for (int t = threadIdx.x; t < Ky * ny; t += blockDim.x) {
      const float mu = a.half_dt * (lx + ly[t]);
      float M[kMaxS][kMaxS];
      float2 r[kMaxS];
      for (int m = 0; m < s; ++m) {
        for (int j = 0; j < s; ++j) M[m][j] = a.C[j][m] - (m == s - 1 && j == s - 1 ? 1.f : 0.f);
        M[m][m] -= mu * a.omega[m];
        r[m] = Bf[t * s + m];
      }
      for (int c = 0; c < s; ++c) {  // elimination with partial pivoting
        int p = c;
        for (int q = c + 1; q < s; ++q)
          if (fabsf(M[q][c]) > fabsf(M[p][c])) p = q;
        if (p != c) {
          for (int j = 0; j < s; ++j) {
            const float tmp = M[c][j];
            M[c][j] = M[p][j];
            M[p][j] = tmp;
          }
          const float2 tr = r[c];
          r[c] = r[p];
          r[p] = tr;
        }
        const float ip = 1.0f / M[c][c];
        for (int q = c + 1; q < s; ++q) {
          const float f = M[q][c] * ip;
          for (int j = c; j < s; ++j) M[q][j] -= f * M[c][j];
          r[q] = make_float2(fmaf(-f, r[c].x, r[q].x), fmaf(-f, r[c].y, r[q].y));
        }
      }
      for (int c = s - 1; c >= 0; --c) {
        float2 acc = r[c];
        for (int j = c + 1; j < s; ++j) acc = make_float2(fmaf(-M[c][j], r[j].x, acc.x), fmaf(-M[c][j], r[j].y, acc.y));
        const float ip = 1.0f / M[c][c];
        r[c] = make_float2(acc.x * ip, acc.y * ip);
      }
      for (int m = 0; m < s; ++m) Bf[t * s + m] = r[m];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nbv; t += blockDim.x) {
      const int iy = t % ny, ky = (t / ny) % Ky, m = t / (ny * Ky);
      float2 acc = make_float2(0.f, 0.f);
      const float2* Bq = Bk + ((size_t)ky * ny + iy) * ny;
      for (int jy = 0; jy < ny; ++jy) acc = cadd(acc, cmul(Bq[jy], Bf[(ky * ny + jy) * s + m]));
      A[(m * ny + iy) * Ky + bitrev(ky, b.flogy)] = acc;
    }
    __syncthreads();
    fft_batched(A, s * ny, b.flogy, tw, true);
    for (int t = threadIdx.x; t < nbv; t += blockDim.x) {
      const int iy = t % ny, ey = (t / ny) % Ky, m = t / (ny * Ky);
      base[t] = A[(m * ny + iy) * Ky + ey];
    }
    __syncthreads();
  }
}

// inverse x pass: item (slot, ey * s + m); writes z = P^-1 (zscale w) to the Z row.
__global__ void __launch_bounds__(256) eng_fdm_xinv_kernel(const __grid_constant__ EngLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nitems = *L.n_fdm_rows;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const EngItem item = L.fdm_rows[it];
    int row;
    float zs;
    if (!fdm_wants(L, item, &row, &zs)) continue;
    const SlotBuf& b = L.buf[item.slot];
    const int n = b.n, ny = b.fny, Kx = b.fkx, Ky = b.fky, s = b.s, nd = b.nd;
    const int ey = item.idx / s, m = item.idx % s;
    const int nb = ny * n;
    float2* X = reinterpret_cast<float2*>(smem_raw);  // [(k n + jx) ny + iy]
    float2* A = X + nb * Kx;                           // [(iy n + ix) Kx + k]
    const float2* tw = reinterpret_cast<const float2*>(b.fdat + b.f_twx);
    const float2* Bk = reinterpret_cast<const float2*>(b.fdat + b.f_Bx);
    for (int t = threadIdx.x; t < nb * Kx; t += blockDim.x) {
      const int iy = t % ny, kj = t / ny;  // kj = k n + jx
      X[t] = b.fx[((size_t)kj * s + m) * Ky * ny + ey * ny + iy];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb * Kx; t += blockDim.x) {
      const int k = t % Kx, ix = (t / Kx) % n, iy = t / (Kx * n);
      float2 acc = make_float2(0.f, 0.f);
      const float2* Bq = Bk + ((size_t)k * n + ix) * n;
      for (int jx = 0; jx < n; ++jx) acc = cadd(acc, cmul(Bq[jx], X[(k * n + jx) * ny + iy]));
      A[(iy * n + ix) * Kx + bitrev(k, b.flogx)] = acc;
    }
    __syncthreads();
    fft_batched(A, nb, b.flogx, tw, true);
    float* dst = b.Z + (size_t)row * b.L;
    for (int t = threadIdx.x; t < nb * Kx; t += blockDim.x) {
      const int node = t % nd, ex = t / nd;
      dst[((size_t)(ey * Kx + ex) * s + m) * nd + node] = A[node * Kx + ex].x;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t eng_fdm_prepare(const EngLaunch& L) {
  const size_t cap = 99 * 1024;
  if (L.fdm_smem_a > cap || L.fdm_smem_b > cap || L.fdm_smem_c > cap) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(eng_fdm_x_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(eng_fdm_y_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(eng_fdm_xinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

cudaError_t eng_fdm_apply(const EngLaunch& L, cudaStream_t st) {
  if (!L.any_fdm) return cudaSuccess;
  eng_fdm_x_kernel<<<L.fdm_grid_rows, 256, L.fdm_smem_a, st>>>(L);
  eng_fdm_y_kernel<<<L.fdm_grid_cols, 256, L.fdm_smem_b, st>>>(L);
  eng_fdm_xinv_kernel<<<L.fdm_grid_rows, 256, L.fdm_smem_c, st>>>(L);
  return cudaGetLastError();
}

}  // namespace stdg
