// Host-side construction of the operator constants (OpArgs) of one slab
// problem: LGL nodes, weights and differentiation matrices in space and time
// (lgl_host.cpp), the strong-form scalings 2/h_a and 1/w_end, dt/2.
#pragma once

#include <cstring>

#include "common.cuh"
#include "lgl_host.h"

namespace stdg {

// nu > 0: constants of the symmetric interior penalty form of -nu Laplace(u)
// (F_v = nu grad u in Eq. general, H_v^IP of Sec. 3.1 with penalty eta,
// eta <= 0 meaning the paper's 10 N^2, and h_e = h_a on faces normal to e_a).
template <class T>
inline void fill_op_args(OpArgs<T>& k, int dim, int n, int s, const int cells[3], const double h[3], double dt,
                         double gamma, const double adv[3], double nu = 0.0, double eta = 0.0) {
  std::memset(&k, 0, sizeof(k));
  k.n = n;
  k.s = s;
  int nd = 1;
  long long nelem = 1;
  for (int a = 0; a < dim; ++a) {
    nd *= n;
    nelem *= cells[a];
  }
  k.nd = nd;
  k.K[0] = cells[0];
  k.K[1] = dim > 1 ? cells[1] : 1;
  k.K[2] = dim > 2 ? cells[2] : 1;
  k.nelem = nelem;
  double xi[16], w[16], D[256];
  lgl_rule(n, xi, w);
  diff_matrix(n, xi, D);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) k.D[i][j] = (T)D[i * n + j];
  double tau[16], om[16], Dt[256];
  lgl_rule(s, tau, om);
  diff_matrix(s, tau, Dt);
  // (D_tau^T M_tau)[m][j] = Dtau[j][m] omega_j  with Dtau[j][m] = l_m'(tau_j)
  for (int j = 0; j < s; ++j)
    for (int m = 0; m < s; ++m) k.C[j][m] = (T)(om[j] * Dt[j * s + m]);
  for (int m = 0; m < s; ++m) k.omega[m] = (T)om[m];
  for (int a = 0; a < 3; ++a) k.ginv[a] = (T)(a < dim ? 2.0 / h[a] : 0.0);
  k.winv_end = (T)(1.0 / w[0]);
  k.half_dt = (T)(0.5 * dt);
  k.gamma = (T)gamma;
  for (int a = 0; a < 3; ++a) k.adv[a] = (T)adv[a];
  k.vscale = (T)1;
  for (int m = 0; m < s; ++m) k.inv_omega[m] = (T)(1.0 / om[m]);
  k.mg_n = fast_div_magic((unsigned)n);
  k.mg_n2 = fast_div_magic((unsigned)(n * n));
  k.mg_nd = fast_div_magic((unsigned)nd);
  k.nu = (T)nu;
  if (nu > 0.0) {
    const int N = n - 1;
    const double pen_eta = eta > 0.0 ? eta : 10.0 * N * N;
    for (int a = 0; a < dim; ++a) {
      const double g = 2.0 / h[a];
      const double sig = nu * pen_eta / h[a];
      k.pen[a] = (T)sig;
      for (int i = 0; i < n; ++i) {
        for (int q = 0; q < n; ++q) k.vDW[a][i][q] = (T)(nu * g * (w[q] / w[i]) * D[q * n + i]);
        k.vup[a][i] = (T)(0.5 * nu * g * g * D[N * n + i] / w[i]);
        k.vlo[a][i] = (T)(0.5 * nu * g * g * D[0 * n + i] / w[i]);
        // diagonal of B(e_i, e_i) / (J w_i) on one line (neighbours zero): volume part plus the
        // face terms at the end nodes (penalty, averaged gradient, lifted jump)
        double dg = 0.0;
        for (int q = 0; q < n; ++q) dg += w[q] * D[q * n + i] * D[q * n + i];
        dg *= nu * g * g / w[i];
        if (i == N) dg += g * sig / w[N] - nu * g * g * D[N * n + N] / w[N];
        if (i == 0) dg += g * sig / w[0] + nu * g * g * D[0] / w[0];
        k.vdiag[a][i] = (T)dg;
      }
    }
  }
}

}  // namespace stdg
