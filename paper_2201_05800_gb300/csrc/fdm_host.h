// Host construction of the global fast-diagonalisation (FDM) preconditioner of
// the batch engine for scalar equations on periodic uniform grids.
//
// The linear part of the spatial operator that the preconditioner keeps, per
// direction a, is the periodic 1D operator A_a = -dF/du of the symmetric
// interior penalty form (Sec. 3.1, H_v^IP with penalty eta and h_e = h_a) plus
// the upwind dissipation lambda/2 [[u]] of the Rusanov flux (Eq. flux:llf) with
// a constant wave-speed bound lambda; the central part of the convective flux
// is left out.  On a periodic row of identical elements A_a is block circulant:
//   (A_a u)_e = A0 u_e + Ap u_{e+1} + Am u_{e-1},
// so its eigenvectors are e^{i theta e} v with theta = 2 pi k / K and v an
// eigenvector of the symbol A(theta) = A0 + Ap e^{i theta} + Am e^{-i theta}.
// A(theta) is self-adjoint in the inner product of the LGL weights W, so
// S = W^{1/2} A(theta) W^{-1/2} is Hermitian: S = U diag(lambda) U^H.
#pragma once

#include <complex>

namespace stdg {

using cplx = std::complex<double>;

// A0, Ap, Am (n x n, row-major) of the 1D operator on elements of width h with n
// LGL nodes, viscosity nu, penalty eta (<= 0: 10 N^2) and dissipation speed lam.
void fdm_blocks_1d(int n, double h, double nu, double eta, double lam, double* A0, double* Ap, double* Am);

// Eigenvalues and eigenvectors of A(theta_k), theta_k = 2 pi k / K, k = 0..K-1:
// lambda[k n + j]; B[(k n + i) n + j] = (W^{-1/2} U_k)[i][j] (columns: eigenvectors);
// F[(k n + j) n + i] = (U_k^H W^{1/2})[j][i] (so that F_k B_k = I and
// A(theta_k) = B_k diag(lambda_k) F_k).  Returns false if the Jacobi sweeps did not converge.
bool fdm_symbol_eig(int n, int K, const double* A0, const double* Ap, const double* Am, const double* w,
                    double* lambda, cplx* B, cplx* F);

}  // namespace stdg
