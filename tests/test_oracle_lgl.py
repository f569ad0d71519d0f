"""Pins of oracle.lgl: LGL rule, differentiation matrix, temporal SBP matrices, Lobatto IIIC.

Each check compares the oracle with something it does not compute itself:
values printed in the paper (Appendix B, Appendix D), library routines
(numpy Legendre roots), closed forms (exact polynomial integrals/derivatives,
Pade approximants of exp) and the order conditions of Sec. 5.2."""
import json
import math
import os

import numpy as np
import pytest

from oracle import lgl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ev(expr):
    return float(eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _mat(rows):
    return np.array([[_ev(e) for e in row] for row in rows])


@pytest.mark.parametrize("n", range(2, 10))
def test_nodes_are_legendre_derivative_roots(n):
    """Interior LGL nodes are the roots of P_N' (numpy's Legendre class), ends are -1, 1."""
    x, _ = lgl.lgl_nodes_weights(n)
    N = n - 1
    ref = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real) if N > 1 else np.array([])
    np.testing.assert_allclose(x[1:-1], ref, atol=1e-14)
    assert x[0] == -1.0 and x[-1] == 1.0


@pytest.mark.parametrize("n", range(2, 10))
def test_quadrature_exact_to_degree_2N_minus_1(n):
    x, w = lgl.lgl_nodes_weights(n)
    N = n - 1
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * N):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13, k
    # degree 2N is not integrated exactly (the rule is Lobatto, not Gauss)
    k = 2 * N
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n", range(2, 10))
def test_differentiation_sbp_consistency_order(n):
    """SBP (Eq. SBP), D 1 = 0 and D x^q = q x^{q-1} for q <= N (order of the operator, Sec. 5.2)."""
    x, w = lgl.lgl_nodes_weights(n)
    D = lgl.lagrange_derivative_matrix(x)
    M = np.diag(w)
    B = np.zeros((n, n))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(M @ D + (M @ D).T, B, atol=1e-13)
    np.testing.assert_allclose(D @ np.ones(n), 0.0, atol=1e-12)
    for q in range(1, n):
        np.testing.assert_allclose(D @ x ** q, q * x ** (q - 1), atol=1e-11)
    # degree n is not differentiated exactly
    assert np.max(np.abs(D @ x ** n - n * x ** (n - 1))) > 1e-6


@pytest.mark.parametrize("s", [2, 3, 4])
def test_appendix_d_matrices(s):
    g = json.load(open(os.path.join(GOLDEN, "appendix_d_dgsem_matrices.json")))["matrices"][str(s)]
    B, M, D, _ = lgl.temporal_matrices(s)
    np.testing.assert_allclose(B, _mat(g["B"]), atol=0)
    np.testing.assert_allclose(M, _mat(g["M"]), atol=1e-15)
    np.testing.assert_allclose(D, _mat(g["D"]), atol=1e-14)


def test_appendix_d_printed_typo_is_inconsistent():
    """The printed row 2 of D_tau (N_tau = 4) violates D 1 = 0; the corrected reading satisfies it."""
    g = json.load(open(os.path.join(GOLDEN, "appendix_d_dgsem_matrices.json")))["matrices"]["4"]
    printed = np.array([_ev(e) for e in g["D_printed_row2"]])
    assert abs(printed.sum() + math.sqrt(5.0)) < 1e-14
    assert abs(_mat(g["D"])[1].sum()) < 1e-14


@pytest.mark.parametrize("s", [2, 3, 4])
def test_appendix_b_tableaus(s):
    g = json.load(open(os.path.join(GOLDEN, "appendix_b_lobatto_iiic.json")))["tableaus"][str(s)]
    A, b, c = lgl.lobatto_iiic_from_dgsem(s)
    np.testing.assert_allclose(A, _mat(g["A"]), atol=1e-15)
    np.testing.assert_allclose(b, [_ev(e) for e in g["b"]], atol=1e-15)
    np.testing.assert_allclose(c, [_ev(e) for e in g["c"]], atol=1e-15)


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6])
def test_order_conditions(s):
    """Theorem (Lobatto IIIC order): B(2s-2), C(s-1), D(s-1); C(s) fails (stage order exactly s-1)."""
    A, b, c = lgl.lobatto_iiic_from_dgsem(s)
    for j in range(1, 2 * s - 1):
        assert abs(b @ c ** (j - 1) - 1.0 / j) < 1e-14, ("B", j)
    for j in range(1, s):
        np.testing.assert_allclose(A @ c ** (j - 1), c ** j / j, atol=1e-14)
        np.testing.assert_allclose(A.T @ (b * c ** (j - 1)), b * (1.0 - c ** j) / j, atol=1e-14)
    assert abs(b @ c ** (2 * s - 2) - 1.0 / (2 * s - 1)) > 1e-8
    assert np.max(np.abs(A @ c ** (s - 1) - c ** s / s)) > 1e-8


def _pade_exp(k, j, z):
    """(k, j) Pade approximant of e^z (Hairer & Wanner II, Thm IV.3.11 closed form)."""
    P = sum(math.factorial(k + j - i) * math.factorial(k) /
            (math.factorial(k + j) * math.factorial(i) * math.factorial(k - i)) * z ** i for i in range(k + 1))
    Q = sum(math.factorial(k + j - i) * math.factorial(j) /
            (math.factorial(k + j) * math.factorial(i) * math.factorial(j - i)) * (-z) ** i for i in range(j + 1))
    return P / Q


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_stability_function_is_pade(s):
    """R(z) = 1 + z b^T (I - z A)^-1 1 equals the (s-2, s) Pade approximant of exp (Lobatto IIIC)."""
    A, b, _ = lgl.lobatto_iiic_from_dgsem(s)
    for z in [-0.3, -2.0, 0.7, -1.0 + 2.0j, -5.0 - 1.5j, -40.0]:
        R = 1.0 + z * (b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s)))
        assert abs(R - _pade_exp(s - 2, s, z)) <= 1e-13 * max(1.0, abs(R)), z


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_dtilde_identities(s):
    """Sec. 5.1: Dtilde^-1 M^-1 e_1 = 1 and e_s^T Dtilde^-1 = 1^T M (so b = M 1 / 2)."""
    _, M, D, _ = lgl.temporal_matrices(s)
    e1 = np.eye(s)[0]
    Dt = D + np.linalg.inv(M) @ np.outer(e1, e1)
    np.testing.assert_allclose(np.linalg.solve(Dt, np.linalg.inv(M) @ e1), np.ones(s), atol=1e-13)
    np.testing.assert_allclose(np.linalg.inv(Dt)[-1], np.diag(M), atol=1e-13)


def test_interpolation_matrix_reproduces_polynomials():
    x, _ = lgl.lgl_nodes_weights(5)
    xe = np.linspace(-1, 1, 17)
    P = lgl.lagrange_interpolation_matrix(x, xe)
    for q in range(5):
        np.testing.assert_allclose(P @ x ** q, xe ** q, atol=1e-13)
