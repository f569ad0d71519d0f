// Host construction of the global fast-diagonalisation preconditioner (fdm_host.h).
#include "fdm_host.h"

#include <cmath>
#include <vector>

#include "lgl_host.h"
#include "stdg.h"

namespace stdg {

void fdm_blocks_1d(int n, double h, double nu, double eta, double lam, double* A0, double* Ap, double* Am) {
  const int N = n - 1;
  double xi[16], w[16], D[256];
  lgl_rule(n, xi, w);
  diff_matrix(n, xi, D);  // D[i n + j] = l_j'(xi_i)
  const double g = 2.0 / h;
  const double pen = eta > 0.0 ? eta : 10.0 * N * N;
  const double sig = nu * pen / h;
  double vup[16], vlo[16];
  for (int i = 0; i < n; ++i) {
    vup[i] = nu * 0.5 * g * g * D[N * n + i] / w[i];  // lift of the upper-face jump
    vlo[i] = nu * 0.5 * g * g * D[i] / w[i];          // lift of the lower-face jump
  }
  // column j: the response F of the operator (dF/du, F = -A u) to the unit vector e_j placed in
  // the own element (A0), in the right neighbour (Ap) or in the left neighbour (Am)
  for (int j = 0; j < n; ++j) {
    double q[16], F0[16], Fp[16], Fm[16];
    for (int k = 0; k < n; ++k) q[k] = g * D[k * n + j];  // gradient of e_j at node k
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += w[k] * D[k * n + i] * q[k];
      F0[i] = -nu * g / w[i] * acc;  // volume term
      Fp[i] = Fm[i] = 0.0;
    }
    const double jN = j == N ? 1.0 : 0.0, j0 = j == 0 ? 1.0 : 0.0;
    // own element: upper face (average gradient, penalty), lower face, lifts, dissipation
    F0[N] += g / w[N] * (nu * 0.5 * q[N] - sig * jN);
    F0[0] -= g / w[0] * (nu * 0.5 * q[0] + sig * j0);
    for (int i = 0; i < n; ++i) F0[i] += vup[i] * jN - vlo[i] * j0;
    F0[N] -= g * lam / (2.0 * w[N]) * jN;
    F0[0] -= g * lam / (2.0 * w[0]) * j0;
    // right neighbour: its node 0 and its gradient there enter the own upper face
    Fp[N] += g / w[N] * (nu * 0.5 * q[0] + sig * j0);
    for (int i = 0; i < n; ++i) Fp[i] -= vup[i] * j0;
    Fp[N] += g * lam / (2.0 * w[N]) * j0;
    // left neighbour: its node N and its gradient there enter the own lower face
    Fm[0] -= g / w[0] * (nu * 0.5 * q[N] - sig * jN);
    for (int i = 0; i < n; ++i) Fm[i] += vlo[i] * jN;
    Fm[0] += g * lam / (2.0 * w[0]) * jN;
    for (int i = 0; i < n; ++i) {
      A0[i * n + j] = -F0[i];
      Ap[i * n + j] = -Fp[i];
      Am[i * n + j] = -Fm[i];
    }
  }
}

namespace {

// Cyclic Jacobi for a Hermitian n x n matrix H (row-major, overwritten): on return the
// diagonal holds the eigenvalues and V (unitary, columns) the eigenvectors.  Each rotation
// first turns H[p][q] real by a phase on column q, then applies the real Jacobi rotation
// that zeroes it (Golub & Van Loan, Sec. 8.5, with the phase step for complex entries).
bool hermitian_jacobi(int n, cplx* H, cplx* V) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = i == j ? 1.0 : 0.0;
  double scale = 0.0;
  for (int i = 0; i < n * n; ++i) scale = std::fmax(scale, std::abs(H[i]));
  if (scale == 0.0) return true;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off = std::fmax(off, std::abs(H[p * n + q]));
    if (off <= 1e-15 * scale) return true;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cplx c = H[p * n + q];
        const double r = std::abs(c);
        if (r <= 1e-300) continue;
        const cplx ph = c / r;  // e^{i phi}
        const double a = H[p * n + p].real(), b = H[q * n + q].real();
        const double tau = (b - a) / (2.0 * r);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        // G = diag(1, conj(ph)) on (p, q) times the real rotation [[cs, sn], [-sn, cs]]
        const cplx gpp = cs, gpq = sn, gqp = -sn * std::conj(ph), gqq = cs * std::conj(ph);
        for (int k = 0; k < n; ++k) {  // H <- H G
          const cplx hp = H[k * n + p], hq = H[k * n + q];
          H[k * n + p] = hp * gpp + hq * gqp;
          H[k * n + q] = hp * gpq + hq * gqq;
        }
        for (int k = 0; k < n; ++k) {  // H <- G^H H
          const cplx hp = H[p * n + k], hq = H[q * n + k];
          H[p * n + k] = std::conj(gpp) * hp + std::conj(gqp) * hq;
          H[q * n + k] = std::conj(gpq) * hp + std::conj(gqq) * hq;
        }
        H[p * n + q] = H[q * n + p] = 0.0;
        H[p * n + p] = H[p * n + p].real();
        H[q * n + q] = H[q * n + q].real();
        for (int k = 0; k < n; ++k) {  // V <- V G
          const cplx vp = V[k * n + p], vq = V[k * n + q];
          V[k * n + p] = vp * gpp + vq * gqp;
          V[k * n + q] = vp * gpq + vq * gqq;
        }
      }
  }
  return false;
}

}  // namespace

bool fdm_symbol_eig(int n, int K, const double* A0, const double* Ap, const double* Am, const double* w,
                    double* lambda, cplx* B, cplx* F) {
  const double pi = 3.14159265358979323846;
  std::vector<cplx> S(n * n), V(n * n);
  bool ok = true;
  for (int k = 0; k < K; ++k) {
    const double th = 2.0 * pi * k / K;
    const cplx ep(std::cos(th), std::sin(th));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const cplx a = A0[i * n + j] + Ap[i * n + j] * ep + Am[i * n + j] * std::conj(ep);
        S[i * n + j] = std::sqrt(w[i]) * a / std::sqrt(w[j]);
      }
    for (int i = 0; i < n; ++i)  // exact Hermitian part (equal to S up to rounding)
      for (int j = i; j < n; ++j) {
        const cplx h = 0.5 * (S[i * n + j] + std::conj(S[j * n + i]));
        S[i * n + j] = h;
        S[j * n + i] = std::conj(h);
      }
    ok = hermitian_jacobi(n, S.data(), V.data()) && ok;
    for (int j = 0; j < n; ++j) lambda[k * n + j] = S[j * n + j].real();
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        B[(k * n + i) * n + j] = V[i * n + j] / std::sqrt(w[i]);
        F[(k * n + j) * n + i] = std::conj(V[i * n + j]) * std::sqrt(w[i]);
      }
  }
  return ok;
}

}  // namespace stdg

extern "C" stdg_status stdg_fdm_symbol(int N, int K, double h, double nu, double eta, double lam, double* lambda,
                                       double* Vre, double* Vim) {
  if (N < 1 || N > 7 || K < 1 || !(h > 0.0) || !(nu >= 0.0) || !(lam >= 0.0) || !lambda || !Vre || !Vim)
    return STDG_ERR_INVALID_ARG;
  const int n = N + 1;
  double xi[16], w[16];
  stdg::lgl_rule(n, xi, w);
  std::vector<double> A0(n * n), Ap(n * n), Am(n * n);
  stdg::fdm_blocks_1d(n, h, nu, eta, lam, A0.data(), Ap.data(), Am.data());
  std::vector<stdg::cplx> B((size_t)K * n * n), F((size_t)K * n * n);
  if (!stdg::fdm_symbol_eig(n, K, A0.data(), Ap.data(), Am.data(), w, lambda, B.data(), F.data()))
    return STDG_ERR_NOT_CONVERGED;
  for (size_t i = 0; i < B.size(); ++i) {
    Vre[i] = B[i].real();
    Vim[i] = B[i].imag();
  }
  return STDG_OK;
}
