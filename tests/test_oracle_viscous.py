"""Pins of the oracle's interior-penalty viscous term (oracle.dgsem.sipg_form).

Independent checks of the symmetric interior penalty form B(u, psi) of
-nu Laplace(u): as a matrix it must be symmetric (a dropped or mis-signed
consistency/symmetry term breaks this) and positive semi-definite for the
paper's penalty eta = 10 p^2 (a wrong penalty sign breaks this), constants are
its null space, it conserves the cell sums, and heat-equation solves converge
to exp(-nu k^2 t) sin(...) at the optimal order p+1."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dgsem, stdg

NU = 0.05


def _grid(dim, cells, N, nu=NU, eq="advection"):
    return dgsem.Grid(dim, cells, (0.0,) * dim, (1.0,) * dim, N, eq,
                      {"adv_vel": (0.0, 0.0, 0.0), "viscosity": nu, "gamma": 1.4})


def _form_matrix(g):
    n = int(np.prod(g.state_shape))
    A = np.empty((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[k] = 1.0
        A[:, k] = dgsem.sipg_form(g, e.reshape(g.state_shape), g.params["viscosity"]).ravel()
        e[k] = 0.0
    return A


@pytest.mark.parametrize("dim,cells,N", [(1, (5,), 1), (1, (4,), 3), (2, (3, 2), 2), (2, (2, 3), 4), (3, (2, 2, 2), 1)])
def test_symmetric_positive_semidefinite(dim, cells, N):
    g = _grid(dim, cells, N)
    A = _form_matrix(g)
    scale = np.max(np.abs(A))
    np.testing.assert_allclose(A, A.T, atol=1e-12 * scale)
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() >= -1e-11 * scale
    # exactly one zero eigenvalue (the constants) on a connected periodic grid
    assert np.sum(ev < 1e-9 * scale) == 1


@pytest.mark.parametrize("dim,cells,N", [(1, (6,), 3), (2, (3, 3), 2)])
def test_constants_and_conservation(dim, cells, N):
    g = _grid(dim, cells, N)
    c = np.full(g.state_shape, 0.7)
    assert np.max(np.abs(dgsem.sipg_form(g, c, NU))) < 1e-12
    u = np.random.default_rng(0).standard_normal(g.state_shape)
    assert abs(np.sum(dgsem.sipg_form(g, u, NU))) < 1e-11 * np.max(np.abs(dgsem.sipg_form(g, u, NU)))
    # the full operator (advection a = 0 plus viscosity) conserves the cell sums
    assert abs(dgsem.integrate(g, dgsem.spatial_operator(g, u))[0]) < 1e-11


def test_zero_penalty_breaks_coercivity():
    """With eta = 0 the symmetric form is not positive semi-definite (the penalty is needed)."""
    g = dgsem.Grid(1, (4,), (0.0,), (1.0,), 3, "advection",
                   {"adv_vel": (0.0,), "viscosity": NU, "penalty": 0.0})
    ev = np.linalg.eigvalsh(_form_matrix(g))
    assert ev.min() < -1e-6


def _march_linear(g, u, dt, s, nslabs):
    """Slabs of a linear problem: one dense Jacobian (exact, complex step) and one LU,
    then U = U0 - J^-1 R(U0) per slab (one exact Newton step solves a linear slab)."""
    F = lambda v: dgsem.spatial_operator(g, v)
    U0 = np.stack([u] * s)
    lu = sla.lu_factor(stdg.jacobian_dense("stdg", F, U0, u, dt))
    for _ in range(nslabs):
        U0 = np.stack([u] * s)
        R = stdg.residual("stdg", F, U0, u, dt)
        u = (U0 - sla.lu_solve(lu, R.ravel()).reshape(U0.shape))[s - 1]
    return u


@pytest.mark.parametrize("N,Ks", [(1, [8, 16, 32]), (2, [4, 8, 16]), (3, [4, 8, 16])])
def test_heat_equation_order(N, Ks):
    """u_t = nu u_xx, u0 = sin(2 pi x): error at T against exp(-4 pi^2 nu T) sin(2 pi x)
    decreases at the optimal SIPG order p+1 (time error made negligible: s = 5)."""
    T, dt, s = 0.05, 0.0125, 5
    errs = []
    for K in Ks:
        g = _grid(1, (K,), N)
        (x,) = g.coordinates()
        u = _march_linear(g, np.sin(2 * np.pi * x)[..., None], dt, s, int(round(T / dt)))
        exact = lambda xx: (np.exp(-4 * np.pi ** 2 * NU * T) * np.sin(2 * np.pi * xx))[..., None]
        errs.append(stdg.l2_error_overintegrated(g, u, exact))
    eoc = np.log2(errs[-2] / errs[-1])
    assert eoc > N + 1 - 0.3, (errs, eoc)


def test_heat_equation_2d_order():
    """2D: sin(2 pi x) sin(2 pi y) decays like exp(-8 pi^2 nu t); the error at T converges at
    order p+1 = 4 from 4^2 to 8^2 elements (p = 3)."""
    errs = []
    T, dt, s = 0.04, 0.02, 4
    for K in (4, 8):
        g = _grid(2, (K, K), 3)
        X = g.coordinates()
        u = (np.sin(2 * np.pi * X[0]) * np.sin(2 * np.pi * X[1]))[..., None]
        u = _march_linear(g, u, dt, s, 2)
        exact = lambda x, y: (np.exp(-8 * np.pi ** 2 * NU * T) * np.sin(2 * np.pi * x)
                              * np.sin(2 * np.pi * y))[..., None]
        errs.append(stdg.l2_error_overintegrated(g, u, exact))
    assert np.log2(errs[0] / errs[1]) > 4 - 0.3, errs
