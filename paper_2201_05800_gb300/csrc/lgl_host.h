// Host-side LGL constants for the CUDA path (see lgl_host.cpp).
#pragma once

namespace stdg {

// n-point Legendre-Gauss-Lobatto nodes (ascending on [-1, 1]) and weights, 2 <= n <= 16.
void lgl_rule(int n, double* x, double* w);
// D[i*n + j] = l_j'(x_i) for the Lagrange basis on the nodes x.
void diff_matrix(int n, const double* x, double* D);

}  // namespace stdg
