// Host-side LGL constants for the CUDA path (see lgl_host.cpp).
#pragma once

namespace stdg {

// n-point Legendre-Gauss-Lobatto nodes (ascending on [-1, 1]) and weights, 2 <= n <= 16.
void lgl_rule(int n, double* x, double* w);
// D[i*n + j] = l_j'(x_i) for the Lagrange basis on the nodes x.
void diff_matrix(int n, const double* x, double* D);
// E[m*s + j] = l_j(tau_m + shift): the Lagrange basis of the s-point LGL rule on [-1, 1]
// evaluated at the nodes moved by shift (shift = 2: the same nodes one slab later).
void lagrange_shift_matrix(int s, double shift, double* E);

}  // namespace stdg
