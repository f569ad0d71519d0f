// Point-block preconditioner of the slab Jacobian (right preconditioning of
// GMRES, J P^-1 y = -R, dU = P^-1 y).
//
// J = (D_tau^T M_tau - e_s e_s^T) (x) I + dt/2 (M_tau (x) I) J_F   (Eq. Jacobian_ST).
// The block of J that couples the s temporal nodes and r components of one
// spatial node I keeps the temporal part exactly and, of the spatial part,
// the diagonal of J_F at I.  In the strong form with the Rusanov flux
// (Eq. flux:llf) that diagonal is, up to the derivative of the wave speed,
//   dF_I/du_I = -sigma_I I,   sigma_I = sum over the element faces through I
//               of (2/h_a) (1/w_end) lambda_face / 2
// (the flux Jacobians of the volume term D[i][i] f'(u_I) and of the face
// correction cancel at the end nodes, where D[N][N] = -D[0][0] = 1/(2 w_end)
// by the SBP property, Eq. SBP; D[i][i] = 0 at the interior nodes).  So the
// block is P_I (x) I_r with the s x s matrix
//   P_I[m][j] = (D_tau^T M_tau)[m][j] - [m = j = s-1] - [m = j] dt/2 omega_m sigma_{I,m},
// (with a viscous term, sigma also holds the diagonal of the interior-penalty
// operator at I, which does not depend on U),
// one per spatial node, the same for all r components.  Its inverse is stored
// per node as Pinv[e][m][j][node] (node fastest, so that consecutive threads
// of the apply kernel read consecutive addresses).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace stdg {

// One (element, spatial node) idx = e * nd + node:  sigma_{I,m} from the wave speeds
// lambda = max(|v_a| + c) over the two traces of every face through I, then
// P_I by Gauss-Jordan elimination with partial pivoting (s <= 5).
// CT: the arithmetic type (double for the FP64 solver; float for the FP32 Krylov solves,
// where P^-1 is stored in FP32 anyway and FP64 operations are 64x slower).
template <int DIM, int EQ, class TP, class CT = double>
__device__ __forceinline__ void pb_build_node(const OpArgs<CT>& k, const double* __restrict__ U,
                                              TP* __restrict__ Pinv, long long idx) {
  using P = Phys<EQ, DIM>;
  constexpr int R = P::R;
  const int n = k.n, s = k.s, nd = k.nd;
  const long long e = idx / nd;
  const int node = (int)(idx - e * nd);
  const int strides[3] = {1, n, n * n};
  const int ia[3] = {node % n, (node / n) % n, node / (n * n)};
  const long long ec[3] = {e % k.K[0], (e / k.K[0]) % k.K[1], e / ((long long)k.K[0] * k.K[1])};
  CT sig[kMaxS];
  for (int m = 0; m < s; ++m) {
    CT uo[R];
    const size_t go = (((size_t)e * s + m) * nd + node) * R;
#pragma unroll
    for (int c = 0; c < R; ++c) uo[c] = (CT)U[go + c];
    CT acc = CT(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const bool up = ia[a] == n - 1, lo = ia[a] == 0;
      if (!up && !lo) continue;
      long long en[3] = {ec[0], ec[1], ec[2]};
      en[a] += up ? 1 : -1;
      if (en[a] < 0) en[a] += k.K[a];
      if (en[a] >= k.K[a]) en[a] -= k.K[a];
      const long long enb = (en[2] * k.K[1] + en[1]) * k.K[0] + en[0];
      const int nb_node = node + ((up ? 0 : n - 1) - ia[a]) * strides[a];
      const size_t gn = (((size_t)enb * s + m) * nd + nb_node) * R;
      CT un[R];
#pragma unroll
      for (int c = 0; c < R; ++c) un[c] = (CT)U[gn + c];
      const CT lo_s = P::template speed<CT, CT>(uo, a, k);
      const CT nb_s = P::template speed<CT, CT>(un, a, k);
      acc += CT(0.5) * k.ginv[a] * k.winv_end * (lo_s >= nb_s ? lo_s : nb_s);
    }
    // viscous term: its diagonal is independent of U
    if (k.nu != CT(0))
      for (int a = 0; a < DIM; ++a) acc += k.vdiag[a][ia[a]];
    sig[m] = acc;
  }
  // augmented [P | I], row m = temporal node m
  CT A[kMaxS][2 * kMaxS];
  for (int m = 0; m < s; ++m) {
    for (int j = 0; j < s; ++j) {
      CT v = k.C[j][m];
      if (m == j) v -= k.half_dt * k.omega[m] * sig[m];
      if (m == s - 1 && j == s - 1) v -= CT(1);
      A[m][j] = v;
      A[m][s + j] = (m == j) ? CT(1) : CT(0);
    }
  }
  for (int col = 0; col < s; ++col) {
    int piv = col;
    for (int q = col + 1; q < s; ++q)
      if (fabs(A[q][col]) > fabs(A[piv][col])) piv = q;
    if (piv != col)
      for (int j = 0; j < 2 * s; ++j) {
        const CT t = A[col][j];
        A[col][j] = A[piv][j];
        A[piv][j] = t;
      }
    const CT inv = CT(1) / A[col][col];
    for (int j = 0; j < 2 * s; ++j) A[col][j] *= inv;
    for (int q = 0; q < s; ++q) {
      if (q == col) continue;
      const CT f = A[q][col];
      if (f != CT(0))
        for (int j = 0; j < 2 * s; ++j) A[q][j] -= f * A[col][j];
    }
  }
  for (int m = 0; m < s; ++m)
    for (int j = 0; j < s; ++j) Pinv[(((size_t)e * s + m) * s + j) * nd + node] = (TP)A[m][s + j];
}

// Pinv of every spatial node from the wave speeds of the slab U (FP64 layout
// [e][m][node][c]); Pinv in TP (double or float).
template <class TP>
cudaError_t pb_build(int dim, int eq, const OpArgs<double>& k, const double* U, TP* Pinv, cudaStream_t st);

// out = a * (P^-1 (x) I_r) v (accumulate = 0) or out += a * (P^-1 (x) I_r) v
// (accumulate = 1), v and out in slab layout.
template <class TP, class TV, class TO>
cudaError_t pb_apply(TO* out, const TV* v, double a, const TP* Pinv, int accumulate, long long nelem, int s,
                     int nd, int r, cudaStream_t st);

}  // namespace stdg
