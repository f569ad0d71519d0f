// Host-side construction of the operator constants (OpArgs) of one slab
// problem: LGL nodes, weights and differentiation matrices in space and time
// (lgl_host.cpp), the strong-form scalings 2/h_a and 1/w_end, dt/2.
#pragma once

#include <cstring>

#include "common.cuh"
#include "lgl_host.h"

namespace stdg {

template <class T>
inline void fill_op_args(OpArgs<T>& k, int dim, int n, int s, const int cells[3], const double h[3], double dt,
                         double gamma, const double adv[3]) {
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
}

}  // namespace stdg
