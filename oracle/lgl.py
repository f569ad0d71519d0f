"""LGL nodes, weights, differentiation matrices and the Lobatto IIIC tableau.

Oracle (test infrastructure only).  FP64, NumPy.

* Nodes/weights: the Legendre-Gauss-Lobatto rule used for the DG-SEM basis
  and quadrature in space (Sec. 3.1) and in time (Sec. 4, derivation of
  Eq. DGSEM_time_component).  Interior nodes are the roots of
  q(x) = P_{N+1}(x) - P_{N-1}(x) (proportional to (1-x^2) P_N'(x)), found by
  Newton's method from Chebyshev-Gauss-Lobatto guesses (Kopriva 2009, Ch. 3).
  Weights w_j = 2 / (N (N+1) P_N(x_j)^2).
* Differentiation matrix (D)_{ji} = l_i'(x_j), the definition used in Sec. 4
  for D_tau, evaluated with the derivative of the Lagrange product formula.
* Temporal matrices B_tau, M_tau, D_tau (Sec. 4, just before Eq. DG_in_time).
* Lobatto IIIC tableau from the DG-SEM matrices, Eq. SBP_to_RK:
  A = 1/2 (D + M^-1 e_1 e_1^T)^-1,  b = 1/2 M 1,  c = (1 + tau)/2.
"""
import numpy as np


def legendre(N, x):
    """P_N(x) by the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev
    p = x.copy()
    for k in range(1, N):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    return p


def lgl_nodes_weights(n):
    """n-point Legendre-Gauss-Lobatto nodes (ascending, on [-1, 1]) and weights."""
    if n < 2:
        raise ValueError("LGL rule needs at least 2 points")
    N = n - 1
    x = -np.cos(np.pi * np.arange(n) / N)  # Chebyshev-Gauss-Lobatto start
    x[0], x[-1] = -1.0, 1.0
    for j in range(1, N):
        xj = x[j]
        for _ in range(100):
            q = legendre(N + 1, xj) - legendre(N - 1, xj)
            dq = (2 * N + 1) * legendre(N, xj)  # d/dx (P_{N+1} - P_{N-1})
            step = q / dq
            xj -= step
            if abs(step) < 1e-16:
                break
        x[j] = xj
    w = 2.0 / (N * (N + 1) * legendre(N, x) ** 2)
    return x, w


def lagrange_derivative_matrix(x):
    """(D)_{ji} = l_i'(x_j) for the Lagrange basis on nodes x.

    l_i(x) = prod_{k != i} (x - x_k)/(x_i - x_k); its derivative at a node x_j is
      j != i:  1/(x_i - x_j) * prod_{k != i, j} (x_j - x_k)/(x_i - x_k)
      j == i:  sum_{k != i} 1/(x_i - x_k).
    """
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                D[j, i] = sum(1.0 / (x[i] - x[k]) for k in range(n) if k != i)
            else:
                prod = 1.0 / (x[i] - x[j])
                for k in range(n):
                    if k != i and k != j:
                        prod *= (x[j] - x[k]) / (x[i] - x[k])
                D[j, i] = prod
    return D


def lagrange_interpolation_matrix(x_nodes, x_eval):
    """(P)_{qi} = l_i(x_eval[q]) with the Lagrange product formula."""
    x_eval = np.asarray(x_eval, dtype=np.float64)
    n = len(x_nodes)
    P = np.ones((len(x_eval), n))
    for i in range(n):
        for k in range(n):
            if k != i:
                P[:, i] *= (x_eval - x_nodes[k]) / (x_nodes[i] - x_nodes[k])
    return P


def temporal_matrices(s):
    """B_tau, M_tau, D_tau and the nodes tau for N_tau = s temporal LGL nodes (Sec. 4)."""
    tau, omega = lgl_nodes_weights(s)
    B = np.zeros((s, s))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    M = np.diag(omega)
    D = lagrange_derivative_matrix(tau)
    return B, M, D, tau


def lobatto_iiic_from_dgsem(s):
    """Butcher tableau (A, b, c) from the DG-SEM matrices, Eq. SBP_to_RK."""
    B, M, D, tau = temporal_matrices(s)
    e1 = np.zeros(s)
    e1[0] = 1.0
    Dtilde = D + np.linalg.inv(M) @ np.outer(e1, e1)
    A = 0.5 * np.linalg.inv(Dtilde)
    b = 0.5 * M @ np.ones(s)
    c = 0.5 * (1.0 + tau)
    return A, b, c
