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
// one per spatial node, the same for all r components.  Its inverse is stored
// per node as Pinv[e][m][j][node] (node fastest, so that consecutive threads
// of the apply kernel read consecutive addresses).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace stdg {

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
