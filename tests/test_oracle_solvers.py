"""Pins of oracle.stdg: Jacobians, solvers, the STDG = LoDG theorem on PDEs, conservation.

Independent references: numpy.linalg.solve, central finite differences, the
printed Jacobian formulas (Eqs. Jacobian_ST, Jacobian_A, Jacobian_Ainv), the
sparsity comparison of Sec. 6.3 (Fig. SparsityD1), the closed-form slab map
R(dt L_h) with R the (s-2, s) Pade approximant of exp, and brute-force dense
Newton against Newton-GMRES."""
import math

import numpy as np
import pytest

from oracle import dgsem, lgl, physics, stdg
from paper_2201_05800_gb300 import inputs

GAMMA = 1.4


def _grid(dim, cells, N, eq, lo=None, hi=None, adv=(1.0, 0.5, -0.75)):
    lo = lo or (0.0,) * dim
    hi = hi or (1.0,) * dim
    return dgsem.Grid(dim, cells, lo, hi, N, eq, {"adv_vel": adv, "gamma": GAMMA})


def _op(g):
    return lambda v: dgsem.spatial_operator(g, v)


def _spatial_jacobian(g, u):
    n = u.size
    J = np.zeros((n, n))
    h = 1e-30
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        J[:, k] = np.imag(dgsem.spatial_operator(g, u + 1j * h * e.reshape(u.shape))).ravel() / h
    return J


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    for m in (5, 20, 80):
        x, its, rel = stdg.gmres(lambda v: A @ v, b, 1e-12, m, 2000)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-10)
        assert rel <= 1e-12 and its > 0


def test_complex_step_jv_matches_central_differences():
    g = _grid(2, (2, 3), 2, physics.EULER)
    u_n = inputs.perturbed(inputs.density_wave(*g.coordinates(), gamma=GAMMA), 1, 0.05)
    s, dt = 3, 0.01
    U = np.stack([inputs.perturbed(u_n, 10 + m, 0.01) for m in range(s)])
    v = inputs.random_array(U.shape, 7)
    for form in ("stdg", "lodg"):
        Jv = stdg.jv_exact(form, _op(g), U, u_n, dt, v)
        eps = 1e-6
        fd = (stdg.residual(form, _op(g), U + eps * v, u_n, dt) -
              stdg.residual(form, _op(g), U - eps * v, u_n, dt)) / (2 * eps)
        np.testing.assert_allclose(Jv, fd, atol=1e-7 * np.max(np.abs(Jv)))


@pytest.mark.parametrize("eq", [physics.EULER, physics.ADVECTION])
def test_jacobian_matches_printed_forms(eq):
    """dR_ST/dU = (D^T M - e_s e_s^T) (x) I + dt/2 (M (x) I) J_F   (Eq. Jacobian_ST)
       dR_RK/dU = I - dt (A (x) I) J_F                              (Eq. Jacobian_A),
    with J_F block diagonal over the time nodes."""
    g = _grid(1, (3,), 2, eq)
    u_n = inputs.perturbed(inputs.density_wave(*g.coordinates(), gamma=GAMMA), 2, 0.05) \
        if eq == physics.EULER else np.sin(2 * np.pi * g.coordinates()[0])[..., None]
    s, dt = 3, 0.05
    U = np.stack([u_n * (1.0 + 0.01 * m) for m in range(s)])
    _, M, D, _ = lgl.temporal_matrices(s)
    A, _, _ = lgl.lobatto_iiic_from_dgsem(s)
    nx = u_n.size
    JF = [_spatial_jacobian(g, U[m]) for m in range(s)]
    es = np.eye(s)[-1]
    J_st = np.kron(D.T @ M - np.outer(es, es), np.eye(nx))
    J_rk = np.eye(s * nx)
    for i in range(s):
        J_st[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx] += 0.5 * dt * M[i, i] * JF[i]
        for j in range(s):
            J_rk[i * nx:(i + 1) * nx, j * nx:(j + 1) * nx] -= dt * A[i, j] * JF[j]
    np.testing.assert_allclose(stdg.jacobian_dense("stdg", _op(g), U, u_n, dt), J_st, atol=1e-12)
    np.testing.assert_allclose(stdg.jacobian_dense("lodg", _op(g), U, u_n, dt), J_rk, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_sparsity_claims(p):
    """Sec. 6.3 / Fig. SparsityD1 (1D advection, one element, order p in space and time):
    the LoDG Jacobian with A is dense-by-blocks, the A^-1 form (Eq. Jacobian_Ainv) has
    exactly as many nonzeros as the STDG Jacobian (Eq. Jacobian_ST), and fewer."""
    s = p + 1
    g = _grid(1, (1,), p, physics.ADVECTION, adv=(1.0,))
    u = np.zeros(g.state_shape)
    JF = _spatial_jacobian(g, u)
    dt = 0.1
    A, _, _ = lgl.lobatto_iiic_from_dgsem(s)
    U = np.stack([u] * s)
    J_st = stdg.jacobian_dense("stdg", _op(g), U, u, dt)
    J_a = stdg.jacobian_dense("lodg", _op(g), U, u, dt)
    J_ainv = np.kron(np.linalg.inv(dt * A), np.eye(u.size)) - np.kron(np.eye(s), JF)
    nnz = lambda X: int(np.sum(np.abs(X) > 1e-12))
    assert nnz(J_st) == nnz(J_ainv)
    assert nnz(J_st) < nnz(J_a)
    # off-diagonal temporal blocks: diagonal for STDG, full spatial blocks dt A_ij J_F for LoDG
    nx = u.size
    for i in range(s):
        for j in range(s):
            if i != j:
                blk = J_st[i * nx:(i + 1) * nx, j * nx:(j + 1) * nx]
                assert nnz(blk - np.diag(np.diag(blk))) == 0
                assert nnz(J_a[i * nx:(i + 1) * nx, j * nx:(j + 1) * nx]) == nnz(JF)


def test_stdg_equals_lodg_config1_direct():
    """1D advection, K = 16, N = 3, s = 3, dt = 0.01, 100 slabs: STDG and LoDG agree to round-off
    (Sec. 5.1 theorem), and match the closed form u^100 = R(dt L_h)^100 u^0, R = Pade(1, 3)."""
    g = _grid(1, (16,), 3, physics.ADVECTION, adv=(1.0,))
    u0 = inputs.sine(g.coordinates()[0])
    s, dt, ns = 3, 0.01, 100
    us = stdg.march("stdg", _op(g), u0, dt, s, ns)
    ul = stdg.march("lodg", _op(g), u0, dt, s, ns)
    nrm = stdg.lgl_weighted_norm(g, us[-1])
    assert stdg.lgl_weighted_norm(g, us[-1] - ul[-1]) <= 1e-12 * nrm
    L = _spatial_jacobian(g, np.zeros_like(u0))
    Z = dt * L
    # (1, 3) Pade approximant of exp: P(z) = 1 + z/4, Q(z) = 1 - 3z/4 + z^2/4 - z^3/24
    P = np.eye(len(L)) + Z / 4
    Q = np.eye(len(L)) - 3 * Z / 4 + Z @ Z / 4 - Z @ Z @ Z / 24
    Rm = np.linalg.solve(Q, P)
    u = u0.ravel()
    for _ in range(ns):
        u = Rm @ u
    assert stdg.lgl_weighted_norm(g, us[-1] - u.reshape(u0.shape)) <= 1e-12 * nrm
    # conservation of the cell sum (periodic, exact solves)
    assert abs(dgsem.integrate(g, us[-1])[0] - dgsem.integrate(g, u0)[0]) < 1e-14
    # accuracy against the exact solution sin(2 pi (x - 1)) after t = 1
    err = stdg.l2_error_overintegrated(g, us[-1], lambda x: inputs.sine(x, t=1.0))
    assert err < 5e-5


def _euler_tiny(dim):
    if dim == 2:
        g = _grid(2, (2, 2), 2, physics.EULER)
    else:
        g = _grid(3, (2, 2, 2), 1, physics.EULER)
    u_n = inputs.perturbed(inputs.density_wave(*g.coordinates(), gamma=GAMMA), 4, 0.02)
    return g, u_n


@pytest.mark.parametrize("dim", [2, 3])
def test_newton_gmres_matches_dense_newton(dim):
    """Brute force (dense Jacobian + LU Newton) vs matrix-free Newton-GMRES on tiny Euler grids;
    also STDG = LoDG on this nonlinear problem, conservation, free-stream (0 Newton steps)."""
    g, u_n = _euler_tiny(dim)
    s, dt = 2, 0.02
    U_direct, its = stdg.solve_slab_direct("stdg", _op(g), u_n, dt, s)
    assert its >= 2
    st = {}
    U_gm = stdg.solve_slab_newton_gmres("stdg", _op(g), u_n, dt, s, rtol=1e-14, atol=1e-15,
                                        gmres_tol=1e-12, gmres_m=60, stats=st)
    nrm = stdg.lgl_weighted_norm(g, U_direct)
    assert stdg.lgl_weighted_norm(g, U_gm - U_direct) <= 1e-12 * nrm
    # the left temporal-mass scaling changes the Krylov iteration, not the Newton solution
    st_w = {}
    U_w = stdg.solve_slab_newton_gmres("stdg", _op(g), u_n, dt, s, rtol=1e-14, atol=1e-15,
                                       gmres_tol=1e-12, gmres_m=60, stats=st_w, scaling="temporal_mass")
    assert stdg.lgl_weighted_norm(g, U_w - U_direct) <= 1e-12 * nrm
    U_lodg, _ = stdg.solve_slab_direct("lodg", _op(g), u_n, dt, s)
    assert stdg.lgl_weighted_norm(g, U_lodg - U_direct) <= 1e-12 * nrm
    cons = dgsem.integrate(g, U_direct[s - 1]) - dgsem.integrate(g, u_n)
    assert np.max(np.abs(cons)) < 1e-13
    const = np.broadcast_to(np.array([1.0] + [0.5] * dim + [3.0]), g.state_shape).copy()
    st = {}
    U_c = stdg.solve_slab_newton_gmres("stdg", _op(g), const, dt, s, rtol=1e-12, atol=1e-14, stats=st)
    assert st["newton_its"] == 0 and np.max(np.abs(U_c - const)) == 0.0


def test_temporal_mass_scaling_is_row_scaling_by_one_over_omega():
    """The scaled system of scaling="temporal_mass" is exactly diag(1/omega_m) J: its GMRES solution
    equals the dense solve of the unscaled Newton system (s = 3, one Newton step, tiny 2D Euler)."""
    g, u_n = _euler_tiny(2)
    s, dt = 3, 0.02
    U0 = np.stack([u_n] * s)
    R = stdg.residual("stdg", _op(g), U0, u_n, dt)
    J = stdg.jacobian_dense("stdg", _op(g), U0, u_n, dt)
    d_direct = np.linalg.solve(J, -R.ravel())
    st = {}
    U1 = stdg.solve_slab_newton_gmres("stdg", _op(g), u_n, dt, s, rtol=0.0, maxit=1, gmres_tol=1e-13,
                                      gmres_m=200, stats=st, scaling="temporal_mass")
    assert st["newton_its"] == 1
    d_gm = (U1 - U0).ravel()
    assert np.linalg.norm(d_gm - d_direct) <= 1e-11 * np.linalg.norm(d_direct)
    # the three temporal weights of s = 3 on [-1, 1]: 1/3, 4/3, 1/3 (Simpson)
    from oracle import lgl
    assert np.allclose(lgl.lgl_nodes_weights(3)[1], [1 / 3, 4 / 3, 1 / 3], atol=1e-15)


def test_newton_converges_quadratically_with_exact_solves():
    g, u_n = _euler_tiny(2)
    st = {}
    stdg.solve_slab_newton_gmres("stdg", _op(g), u_n, 0.05, 3, rtol=1e-15, atol=1e-15,
                                 gmres_tol=1e-13, gmres_m=200, stats=st)
    h = st["history"]
    # once in the asymptotic regime, each step roughly squares the relative residual
    rel = [x / h[0] for x in h]
    k = next(i for i, r in enumerate(rel) if r < 1e-3)
    if k + 1 < len(rel) and rel[k + 1] > 1e-15:
        assert rel[k + 1] < 10 * rel[k] ** 1.8
