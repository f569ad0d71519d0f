"""Host-side constants of the CUDA path, on the CPU (no GPU involved).

* stdg_lgl_constants: the LGL nodes, weights and differentiation matrix the CUDA path is built
  from (Jacobi-polynomial Newton iteration and barycentric D) against the oracle's independent
  construction (Legendre Newton iteration, Lagrange product D) for n = 2..16, against the
  Appendix D matrices (with the printed D_tau typo read as in the golden file), and against
  exactness, SBP (Eq. SBP) and D 1 = 0.
* stdg_predictor_matrix: E[m, j] = l_j(tau_m + 2), the previous slab's temporal polynomial (the
  Lagrange basis on the s temporal LGL nodes of the space-time expansion, Eq. StCoeff) evaluated
  at the next slab's nodes, tau in [-1, 1] on each slab.  Pins: exact continuation of every
  polynomial of degree < s; the first row picks the previous slab's last node
  (tau_0 + 2 = 1 = tau_{s-1}); rows sum to one; agreement with the oracle's Lagrange
  interpolation matrix (an independent construction)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import lgl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def S():
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


def _golden_value(expr):
    """Exact entries of the golden file: rationals and sqrt(5) expressions."""
    return float(eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt}))


@pytest.mark.parametrize("n", list(range(2, 17)))
def test_lgl_constants_match_the_oracle(S, n):
    x, w, D = S.lgl_constants(n)
    xo, wo = lgl.lgl_nodes_weights(n)
    Do = lgl.lagrange_derivative_matrix(xo)
    assert np.max(np.abs(x - xo)) <= 1e-14
    assert np.max(np.abs(w - wo)) <= 1e-14
    assert np.max(np.abs(D - Do)) <= 1e-12 * max(1.0, np.max(np.abs(Do)))


@pytest.mark.parametrize("n", list(range(2, 17)))
def test_lgl_constants_exactness_and_sbp(S, n):
    x, w, D = S.lgl_constants(n)
    N = n - 1
    # quadrature exact to degree 2N - 1; D exact on degree <= N; D 1 = 0
    for q in range(2 * N):
        exact = (1.0 - (-1.0) ** (q + 1)) / (q + 1)
        assert abs(w @ x ** q - exact) <= 1e-13, q
    for q in range(1, N + 1):
        assert np.max(np.abs(D @ x ** q - q * x ** (q - 1))) <= 1e-10 * q * q, q
    assert np.max(np.abs(D.sum(axis=1))) <= 1e-11 * n * n
    # SBP: W D + (W D)^T = diag(-1, 0, ..., 0, 1)
    Q = np.diag(w) @ D
    B = np.zeros((n, n))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.max(np.abs(Q + Q.T - B)) <= 1e-11 * n * n


@pytest.mark.parametrize("s", [2, 3, 4])
def test_lgl_constants_reproduce_appendix_d(S, s):
    g = json.load(open(os.path.join(GOLDEN, "appendix_d_dgsem_matrices.json")))["matrices"][str(s)]
    x, w, D = S.lgl_constants(s)
    Dg = np.array([[_golden_value(e) for e in row] for row in g["D"]])
    Mg = np.array([[_golden_value(e) for e in row] for row in g["M"]])
    assert np.max(np.abs(D - Dg)) <= 1e-14
    assert np.max(np.abs(np.diag(w) - Mg)) <= 1e-15


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_polynomials_below_degree_s_continue_exactly(S, s):
    E = S.predictor_matrix(s)
    tau, _ = lgl.lgl_nodes_weights(s)
    for q in range(s):
        err = np.max(np.abs(E @ tau ** q - (tau + 2.0) ** q))
        assert err <= 1e-12 * 3.0 ** q, (q, err)
    # degree s is not reproduced (the continuation is the degree s-1 interpolant)
    assert np.max(np.abs(E @ tau ** s - (tau + 2.0) ** s)) > 1e-3


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_first_row_is_previous_end_node_and_rows_sum_to_one(S, s):
    E = S.predictor_matrix(s)
    e_last = np.zeros(s)
    e_last[-1] = 1.0
    assert np.max(np.abs(E[0] - e_last)) <= 1e-13
    assert np.max(np.abs(E.sum(axis=1) - 1.0)) <= 1e-12


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_matches_oracle_interpolation_matrix(S, s):
    tau, _ = lgl.lgl_nodes_weights(s)
    ref = lgl.lagrange_interpolation_matrix(tau, tau + 2.0)
    assert np.max(np.abs(S.predictor_matrix(s) - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("s", [1, 6])
def test_out_of_range_s_is_rejected(S, s):
    with pytest.raises(S.StdgError):
        S.predictor_matrix(s)
