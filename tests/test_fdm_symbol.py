"""The spectral data of the batch engine's global preconditioner (stdg_fdm_symbol, host only)
against the oracle.

The engine preconditions a scalar slot on a periodic grid by the exact inverse of
  P = (D_tau^T M_tau - e_s e_s^T) (x) I - dt/2 M_tau (x) (A_x (+) A_y),
with A_a the periodic 1D operator of the interior penalty form of -nu d^2/dx^2 (Sec. 3.1)
plus the upwind dissipation lambda/2 [[u]] of the Rusanov flux (Eq. flux:llf).  Here A is
assembled from the oracle: the viscous part from oracle.dgsem.sipg_form, the dissipation as
the part of the oracle's upwind advection operator that is symmetric in the LGL mass inner
product.  Every returned pair (lambda, phi) with phi[e][i] = exp(2 pi i k e / K) V_k[i][j]
must satisfy A phi = lambda phi, and the eigenvalues must be those of A."""
import numpy as np
import pytest

from oracle import dgsem


def _global_operator(K, N, nu, lam):
    n = N + 1
    L = 1.0
    gv = dgsem.Grid(1, (K,), (0.0,), (L,), N, "burgers", {"viscosity": nu})
    W = (gv.jacobian() * gv.node_weights()[..., None])
    A = np.zeros((K * n, K * n))
    for k in range(K * n):
        e = np.zeros((K, n, 1))
        e.ravel()[k] = 1.0
        A[:, k] = (dgsem.sipg_form(gv, e, nu) / W).ravel() if nu else 0.0
    if lam:
        ga = dgsem.Grid(1, (K,), (0.0,), (L,), N, "advection", {"adv_vel": (lam,)})
        Ja = np.zeros((K * n, K * n))
        for k in range(K * n):
            e = np.zeros((K, n, 1))
            e.ravel()[k] = 1.0
            Ja[:, k] = -dgsem.spatial_operator(ga, e).ravel()
        w = np.tile(W.ravel(), K)
        S = 0.5 * (np.diag(w) @ Ja + (np.diag(w) @ Ja).T)
        A += S / w[:, None]
    return A


@pytest.mark.parametrize("K,N,nu,lam", [(8, 3, 0.05, 0.0), (6, 6, 0.3, 0.7), (5, 2, 0.0, 1.3), (1, 4, 0.02, 0.4),
                                        (16, 5, 1e-3, 0.5)])
def test_fdm_modes_are_eigenpairs_of_the_oracle_operator(K, N, nu, lam):
    from paper_2201_05800_gb300 import stdg
    n = N + 1
    A = _global_operator(K, N, nu, lam)
    lam_k, V = stdg.fdm_symbol(N, K, 1.0 / K, nu, 0.0, lam)
    scale = np.max(np.abs(A))
    e = np.arange(K)
    for k in range(K):
        ph = np.exp(2j * np.pi * k * e / K)
        for j in range(n):
            phi = (ph[:, None] * V[k, :, j][None, :]).ravel()
            r = A @ phi - lam_k[k, j] * phi
            assert np.linalg.norm(r) <= 1e-11 * scale * np.linalg.norm(phi), (k, j)
    ev = np.sort(np.real(np.linalg.eigvals(A)))
    assert np.max(np.abs(np.sort(lam_k.ravel()) - ev)) <= 1e-10 * scale
    # the eigenvector blocks are W-orthonormal: V_k^H W V_k = I
    from oracle import lgl
    _, w = lgl.lgl_nodes_weights(n)
    for k in range(K):
        G = V[k].conj().T @ np.diag(w) @ V[k]
        assert np.allclose(G, np.eye(n), atol=1e-12)


def test_fdm_symbol_rejects_bad_arguments():
    from paper_2201_05800_gb300 import stdg
    for args in ((0, 4, 0.25, 0.1, 0.0, 0.0), (8, 4, 0.25, 0.1, 0.0, 0.0), (3, 0, 0.25, 0.1, 0.0, 0.0),
                 (3, 4, 0.0, 0.1, 0.0, 0.0), (3, 4, 0.25, -0.1, 0.0, 0.0), (3, 4, 0.25, 0.1, 0.0, -1.0)):
        with pytest.raises(stdg.StdgError):
            stdg.fdm_symbol(*args)
