"""The matrix of the extrapolated initial Newton iterate (stdg_predictor_matrix), on the CPU.

E[m, j] = l_j(tau_m + 2): the previous slab's temporal polynomial (the Lagrange basis on the s
temporal LGL nodes of the space-time expansion, Eq. StCoeff) evaluated at the next slab's nodes,
tau in [-1, 1] on each slab.  Pins: exact continuation of every polynomial of degree < s; the
first row picks the previous slab's last node (tau_0 + 2 = 1 = tau_{s-1}); rows sum to one;
agreement with the oracle's Lagrange interpolation matrix (an independent construction)."""
import numpy as np
import pytest

from oracle import lgl


@pytest.fixture(scope="module")
def S():
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


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
