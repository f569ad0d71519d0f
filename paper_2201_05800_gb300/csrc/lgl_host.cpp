// Host-side LGL constants for the CUDA path (FP64).
//
// The DG-SEM basis lives on the Legendre-Gauss-Lobatto nodes in space
// (Sec. 3.1) and time (Sec. 4).  Interior LGL nodes of the n = N+1 point rule
// are the zeros of P_N', i.e. of the Jacobi polynomial P^(1,1)_{N-1}; they are
// found by Newton's method on the Jacobi three-term recurrence (differentiated
// alongside), starting from Chebyshev-Gauss-Lobatto points.  Weights are
// w_j = 2 / (N (N+1) P_N(x_j)^2).  The differentiation matrix D[i][j] = l_j'(x_i)
// uses the barycentric form: D[i][j] = (lambda_j / lambda_i) / (x_i - x_j) for
// i != j, lambda_j = 1 / prod_{k != j} (x_j - x_k), and D[i][i] = -sum_{j != i} D[i][j].
#include "lgl_host.h"

#include <cmath>

namespace stdg {

namespace {

// P^(1,1)_k(x) and its derivative by the Jacobi recurrence
// 2(k+1)(k+a+b+1)(2k+a+b) P_{k+1} = (2k+a+b+1)[(2k+a+b+2)(2k+a+b) x + a^2-b^2] P_k
//                                   - 2(k+a)(k+b)(2k+a+b+2) P_{k-1},   a = b = 1.
void jacobi11(int deg, double x, double* p, double* dp) {
  const double a = 1.0, b = 1.0;
  double pm = 1.0, dpm = 0.0;  // P_0
  if (deg == 0) { *p = pm; *dp = dpm; return; }
  double pc = 0.5 * ((a + b + 2.0) * x + (a - b)), dpc = 0.5 * (a + b + 2.0);  // P_1
  for (int k = 1; k < deg; ++k) {
    double c1 = 2.0 * (k + 1) * (k + a + b + 1) * (2 * k + a + b);
    double c2 = (2 * k + a + b + 1) * (2 * k + a + b + 2) * (2 * k + a + b);
    double c3 = (2 * k + a + b + 1) * (a * a - b * b);
    double c4 = 2.0 * (k + a) * (k + b) * (2 * k + a + b + 2);
    double pn = ((c2 * x + c3) * pc - c4 * pm) / c1;
    double dpn = ((c2 * x + c3) * dpc + c2 * pc - c4 * dpm) / c1;
    pm = pc; dpm = dpc; pc = pn; dpc = dpn;
  }
  *p = pc; *dp = dpc;
}

double legendre_p(int N, double x) {
  double pm = 1.0;
  if (N == 0) return pm;
  double pc = x;
  for (int k = 1; k < N; ++k) {
    double pn = ((2.0 * k + 1.0) * x * pc - k * pm) / (k + 1.0);
    pm = pc; pc = pn;
  }
  return pc;
}

}  // namespace

void lgl_rule(int n, double* x, double* w) {
  const int N = n - 1;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      jacobi11(N - 1, t, &p, &dp);
      double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[j] = t;
  }
  for (int j = 0; j <= N; ++j) {
    double p = legendre_p(N, x[j]);
    w[j] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

void diff_matrix(int n, const double* x, double* D) {
  double lam[16];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0 / prod;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double v = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * n + j] = v;
      diag -= v;
    }
    D[i * n + i] = diag;
  }
}

void lagrange_shift_matrix(int s, double shift, double* E) {
  double tau[16], w[16];
  lgl_rule(s, tau, w);
  for (int m = 0; m < s; ++m)
    for (int j = 0; j < s; ++j) {
      double l = 1.0;
      for (int q = 0; q < s; ++q)
        if (q != j) l *= (tau[m] + shift - tau[q]) / (tau[j] - tau[q]);
      E[m * s + j] = l;
    }
}

}  // namespace stdg
