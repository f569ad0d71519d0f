"""Pins of oracle.physics and oracle.dgsem (spatial DG-SEM operator, weak form).

Independent checks: the strong form of the same scheme written element by
element with explicit loops (equal to the weak form by SBP, Eq. SBP), closed
forms for 1D upwind advection, free-stream preservation, discrete
conservation, flux identities (consistency, homogeneity, Euler's theorem,
rotational symmetry) and the spatial convergence order N+1 on smooth
solutions."""
import itertools

import numpy as np
import pytest

from oracle import dgsem, lgl, physics, stdg
from paper_2201_05800_gb300 import inputs

GAMMA = 1.4


def _grid(dim, cells, N, eq, lo=None, hi=None, adv=(1.0, 0.5, -0.75)):
    lo = lo or (0.0,) * dim
    hi = hi or (1.0,) * dim
    return dgsem.Grid(dim, cells, lo, hi, N, eq, {"adv_vel": adv, "gamma": GAMMA})


def _state(g, seed, kind="smooth"):
    X = g.coordinates()
    if g.eq == physics.EULER:
        base = inputs.density_wave(*X, gamma=GAMMA)
        return inputs.perturbed(base, seed, 0.05) if kind == "rough" else base
    u = np.sin(2 * np.pi * sum(X))[..., None]
    return u + (inputs.random_array(u.shape, seed, 0.3) if kind == "rough" else 0.0)


def _strong_form_loops(g, u):
    """F written per element and node in strong form:
    F_I = -sum_a (2/h_a) [ sum_j D[i_a, j] f_a(u_(I, i_a -> j))
                         + (1/w_{i_a}) (delta_{i_a, N} (H_a^+ - f_a(u_I)) - delta_{i_a, 0} (H_a^- - f_a(u_I))) ]."""
    d, n, N = g.dim, g.n, g.N
    K = g.cells
    F = np.zeros_like(u)
    for e in itertools.product(*[range(k) for k in reversed(K)]):  # (ez, ey, ex)[-d:]
        for I in itertools.product(range(n), repeat=d):  # (iz, iy, ix)[-d:]
            acc = np.zeros(g.r)
            uI = u[e + I]
            for a in range(d):
                pa = d - 1 - a  # position of direction a in the reversed tuples
                ia = I[pa]
                vol = np.zeros(g.r)
                for j in range(n):
                    J = list(I)
                    J[pa] = j
                    vol += g.D[ia, j] * physics.flux(g.eq, u[e + tuple(J)], a, g.params)
                surf = np.zeros(g.r)
                fI = physics.flux(g.eq, uI, a, g.params)
                if ia == N:
                    en = list(e)
                    en[pa] = (e[pa] + 1) % K[a]
                    J = list(I)
                    J[pa] = 0
                    H = physics.rusanov(g.eq, uI, u[tuple(en) + tuple(J)], a, g.params)
                    surf += (H - fI) / g.w[N]
                if ia == 0:
                    en = list(e)
                    en[pa] = (e[pa] - 1) % K[a]
                    J = list(I)
                    J[pa] = N
                    H = physics.rusanov(g.eq, u[tuple(en) + tuple(J)], uI, a, g.params)
                    surf -= (H - fI) / g.w[0]
                acc -= (2.0 / g.h[a]) * (vol + surf)
            F[e + I] = acc
    return F


CASES = [(1, (5,), 3, physics.ADVECTION), (1, (4,), 2, physics.EULER),
         (2, (3, 2), 2, physics.ADVECTION), (2, (2, 3), 3, physics.EULER),
         (3, (2, 2, 2), 1, physics.EULER), (3, (2, 1, 2), 2, physics.ADVECTION),
         (2, (2, 2), 2, physics.BURGERS)]


@pytest.mark.parametrize("dim,cells,N,eq", CASES)
def test_weak_form_equals_strong_form(dim, cells, N, eq):
    g = _grid(dim, cells, N, eq)
    u = _state(g, 3, "rough")
    Fw = dgsem.spatial_operator(g, u)
    Fs = _strong_form_loops(g, u)
    scale = np.max(np.abs(Fs))
    np.testing.assert_allclose(Fw, Fs, atol=1e-13 * scale)


@pytest.mark.parametrize("dim,cells,N,eq", CASES)
def test_free_stream_and_conservation(dim, cells, N, eq):
    g = _grid(dim, cells, N, eq)
    if eq == physics.EULER:
        const = np.array([1.2] + [0.3, -0.2, 0.1][:dim] + [2.5])
    else:
        const = np.array([0.7])
    u = np.broadcast_to(const, g.state_shape).copy()
    assert np.max(np.abs(dgsem.spatial_operator(g, u))) < 1e-13
    u = _state(g, 5, "rough")
    tot = dgsem.integrate(g, dgsem.spatial_operator(g, u))
    assert np.max(np.abs(tot)) < 1e-13 * np.max(np.abs(u))


def test_advection_continuous_polynomial_is_exact():
    """u continuous, degree <= N per element, zero at element ends: F = -a u' at every node."""
    for N in (2, 3, 5):
        for a in (1.3, -0.6):
            g = _grid(1, (4,), N, physics.ADVECTION, adv=(a,))
            (x,) = g.coordinates()
            xl = g.lo[0] + g.h[0] * np.floor((x - g.lo[0]) / g.h[0] + 1e-12)
            xl = np.minimum(xl, g.lo[0] + g.h[0] * np.arange(4)[:, None])
            xr = xl + g.h[0]
            c = np.array([1.0, -2.0, 0.5, 3.0])[:, None]
            u = c * (x - xl) * (xr - x) * (1.0 + x)  # degree 3 <= N when N >= 3
            du = c * ((xr - x) * (1 + x) - (x - xl) * (1 + x) + (x - xl) * (xr - x))
            if N < 3:
                u = c * (x - xl) * (xr - x)
                du = c * ((xr - x) - (x - xl))
            F = dgsem.spatial_operator(g, u[..., None])[..., 0]
            np.testing.assert_allclose(F, -a * du, atol=1e-11)


def test_advection_piecewise_constant_closed_form():
    """Piecewise constant u = c_e, a > 0: F = (2 a / (h w_0)) (c_{e-1} - c_e) at the left node, 0 elsewhere."""
    N, a = 3, 0.8
    g = _grid(1, (5,), N, physics.ADVECTION, adv=(a,))
    c = np.array([1.0, 2.5, -1.0, 0.25, 4.0])
    u = np.broadcast_to(c[:, None, None], g.state_shape).copy()
    F = dgsem.spatial_operator(g, u)[..., 0]
    expect = np.zeros((5, N + 1))
    expect[:, 0] = 2 * a / (g.h[0] * g.w[0]) * (np.roll(c, 1) - c)
    np.testing.assert_allclose(F, expect, atol=1e-12)


def test_rusanov_consistency_and_upwind():
    rng = np.random.default_rng(0)
    for dim in (1, 2, 3):
        u = inputs.perturbed(inputs.density_wave(*[rng.uniform(size=7) for _ in range(dim)]), 1, 0.1)
        for a in range(dim):
            H = physics.rusanov(physics.EULER, u, u, a, {"gamma": GAMMA})
            np.testing.assert_allclose(H, physics.euler_flux(u, a, GAMMA), rtol=1e-14, atol=1e-15)
    uL, uR = rng.standard_normal((6, 1)), rng.standard_normal((6, 1))
    for vel in (0.7, -1.3):
        H = physics.rusanov(physics.ADVECTION, uL, uR, 0, {"adv_vel": (vel,)})
        np.testing.assert_allclose(H, vel * (uL if vel > 0 else uR), rtol=1e-14, atol=1e-15)


def test_euler_flux_identities():
    """Homogeneity f(l u) = l f(u); Euler's theorem (df/du) u = f(u) via the complex step;
    at rest f_a = p e_{a+1}; 2D rotation by 90 degrees maps f_1 to f_2."""
    rng = np.random.default_rng(1)
    for dim in (1, 2, 3):
        X = [rng.uniform(size=9) for _ in range(dim)]
        u = inputs.perturbed(inputs.density_wave(*X, gamma=GAMMA), 2, 0.1)
        for a in range(dim):
            f = physics.euler_flux(u, a, GAMMA)
            np.testing.assert_allclose(physics.euler_flux(2.5 * u, a, GAMMA), 2.5 * f, rtol=1e-14)
            h = 1e-30
            Ju = np.imag(physics.euler_flux(u + 1j * h * u, a, GAMMA)) / h
            np.testing.assert_allclose(Ju, f, rtol=1e-13)
        rest = u.copy()
        rest[..., 1:1 + dim] = 0.0
        p = physics.pressure(rest, GAMMA)
        for a in range(dim):
            f = physics.euler_flux(rest, a, GAMMA)
            expect = np.zeros_like(rest)
            expect[..., 1 + a] = p
            np.testing.assert_allclose(f, expect, atol=1e-15)
    u = inputs.perturbed(inputs.density_wave(rng.uniform(size=5), rng.uniform(size=5)), 3, 0.1)
    rot = u.copy()
    rot[..., 1], rot[..., 2] = -u[..., 2], u[..., 1]  # velocity rotated by +90 degrees
    f1, f2r = physics.euler_flux(u, 0, GAMMA), physics.euler_flux(rot, 1, GAMMA)
    np.testing.assert_allclose(f2r[..., 0], f1[..., 0], rtol=1e-14)
    np.testing.assert_allclose(f2r[..., 2], f1[..., 1], rtol=1e-14)
    np.testing.assert_allclose(f2r[..., 1], -f1[..., 2], rtol=1e-14)
    np.testing.assert_allclose(f2r[..., 3], f1[..., 3], rtol=1e-14)


def _convergence(dim, eq, N, Ks, T, dt, s):
    errs = []
    for K in Ks:
        g = _grid(dim, (K,) * dim, N, eq, adv=(1.0, 1.0, 1.0))
        X = g.coordinates()
        if eq == physics.EULER:
            u = inputs.density_wave(*X, gamma=GAMMA)
            exact = lambda *c: inputs.density_wave(*c, t=T, gamma=GAMMA)
        else:
            u = np.sin(2 * np.pi * sum(X))[..., None]
            exact = lambda *c: np.sin(2 * np.pi * (sum(c) - dim * T))[..., None]
        F = lambda v: dgsem.spatial_operator(g, v)
        for _ in range(int(round(T / dt))):
            U = stdg.solve_slab_newton_gmres("stdg", F, u, dt, s, rtol=1e-12, gmres_tol=1e-10, gmres_m=40)
            u = U[s - 1]
        errs.append(stdg.l2_error_overintegrated(g, u, exact))
    return [np.log2(errs[i - 1] / errs[i]) for i in range(1, len(errs))]


@pytest.mark.parametrize("N,Ks", [(1, [8, 16, 32]), (2, [16, 32, 64]), (3, [8, 16, 32])])
def test_spatial_order_euler_1d(N, Ks):
    eocs = _convergence(1, physics.EULER, N, Ks, T=0.05, dt=0.0125, s=5)
    assert eocs[-1] > N + 1 - 0.25, eocs


def test_spatial_order_advection_2d():
    """Sec. 5.2 states the DG-SEM L2 order as p+1 or p+1/2 depending on problem and flux;
    the diagonal 2D upwind case reaches p+1/2 here."""
    eocs = _convergence(2, physics.ADVECTION, 2, [4, 8, 16, 32], T=0.02, dt=0.01, s=5)
    assert eocs[-1] > 2 + 0.5 - 0.1, eocs


def test_euler_wave_speed_is_spectral_radius_of_flux_jacobian():
    """lambda_a(u) = |v_a| + c equals max |eig(d f_a / d u)| (eigenvalues v_a - c, v_a, v_a + c)."""
    rng = np.random.default_rng(4)
    for dim in (1, 2, 3):
        X = [rng.uniform(size=4) for _ in range(dim)]
        U = inputs.perturbed(inputs.density_wave(*X, gamma=GAMMA), 5, 0.2)
        U[..., 1] *= -1.0  # include negative velocities (pressure unchanged)
        for u in U:
            for a in range(dim):
                r = u.size
                J = np.empty((r, r))
                for k in range(r):
                    e = np.zeros(r)
                    e[k] = 1e-30
                    J[:, k] = np.imag(physics.euler_flux(u + 1j * e, a, GAMMA)) / 1e-30
                rho_sp = np.max(np.abs(np.linalg.eigvals(J)))
                assert abs(physics.euler_wave_speed(u, a, GAMMA) - rho_sp) < 1e-12 * rho_sp
