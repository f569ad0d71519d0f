"""Pins of the oracle's Burgers branch (physics.flux / physics.wave_speed) and of
stdg.lgl_weighted_norm, each against something other than the oracle itself.

Burgers (the convective part of the batched viscous Burgers workload, with the
Rusanov flux of Eq. flux:llf):
* the flux derivative f'(u) = u, by a central difference of physics.flux in the
  test, and the Rusanov speed equal to max(|f'(u-)|, |f'(u+)|) of those
  differences (the largest characteristic speed of the two states);
* slab solves of smooth 1D inviscid Burgers before the shock time against the
  characteristic solution u(x, t) = u0(x - u t), solved pointwise here by
  Newton's method on the scalar equation (nothing from physics), with the
  spatial order N+1 (Sec. 5.2) at a time step small enough that the Lobatto
  IIIC error (order 2s-2) is negligible.  A factor 2 in f (u^2 instead of
  u^2/2) moves every characteristic twice as fast and fails by O(1).

Norm (Eq. DG_norm read as the square root of the summed quadratic forms):
* a constant c in every component over a box of volume V: |c| sqrt(2 V r) for a
  slab (temporal weights sum to 2 on [-1, 1]) and |c| sqrt(V r) for one level;
* products of polynomials of degree <= N-1 per direction and <= s-2 in time,
  whose squares the LGL rules integrate exactly: the norm equals the exact
  integral computed with numpy.polynomial in the test.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from oracle import dgsem, physics, stdg


# ------------------------------------------------------------------ Burgers flux


def test_burgers_flux_derivative_and_rusanov_speed():
    rng = np.random.default_rng(11)
    u = rng.uniform(-2.0, 2.0, size=(64, 1))
    h = 1e-6
    for a in range(2):
        df = (physics.flux("burgers", u + h, a, {}) - physics.flux("burgers", u - h, a, {})) / (2 * h)
        # f'(u) = u (the flux of u_t + div(u^2/2 (1, 1)) = 0)
        np.testing.assert_allclose(df, u, rtol=0, atol=1e-9)
        # largest characteristic speed = |f'(u)|
        np.testing.assert_allclose(physics.wave_speed("burgers", u, a, {}), np.abs(df[:, 0]), rtol=0, atol=1e-9)
    f0 = physics.flux("burgers", np.zeros((1, 1)), 0, {})
    assert f0[0, 0] == 0.0
    # Rusanov: central average minus lambda/2 (uR - uL), lambda = max(|f'(uL)|, |f'(uR)|)
    uL = rng.uniform(-2.0, 2.0, size=(64, 1))
    uR = rng.uniform(-2.0, 2.0, size=(64, 1))
    H = physics.rusanov("burgers", uL, uR, 0, {})
    fL = physics.flux("burgers", uL, 0, {})
    fR = physics.flux("burgers", uR, 0, {})
    dL = (physics.flux("burgers", uL + h, 0, {}) - physics.flux("burgers", uL - h, 0, {})) / (2 * h)
    dR = (physics.flux("burgers", uR + h, 0, {}) - physics.flux("burgers", uR - h, 0, {})) / (2 * h)
    lam = np.maximum(np.abs(dL), np.abs(dR))
    np.testing.assert_allclose(H, 0.5 * (fL + fR) - 0.5 * lam * (uR - uL), rtol=0, atol=1e-8)


def _u0(x):
    return 0.5 + 0.25 * np.sin(2 * np.pi * x)


def _du0(x):
    return 0.25 * 2 * np.pi * np.cos(2 * np.pi * x)


def _characteristic(x, t):
    """u(x, t) solving u = u0(x - u t) by Newton on g(u) = u - u0(x - u t)."""
    u = _u0(x)
    for _ in range(60):
        g = u - _u0(x - u * t)
        dg = 1.0 + t * _du0(x - u * t)
        step = g / dg
        u = u - step
        if np.max(np.abs(step)) < 1e-15:
            break
    return u


def _burgers_error(K, N, s, dt, nslabs):
    g = dgsem.Grid(1, (K,), (0.0,), (1.0,), N, "burgers", {})
    X = g.coordinates()[0]
    u = _u0(X)[..., None]
    F = lambda v: dgsem.spatial_operator(g, v)
    for _ in range(nslabs):
        U = stdg.solve_slab_newton_gmres("stdg", F, u, dt, s, rtol=1e-13, atol=1e-14, gmres_tol=1e-12,
                                         gmres_m=40)
        u = U[s - 1]
    T = dt * nslabs
    return stdg.l2_error_overintegrated(g, u, lambda x: _characteristic(x, T)[..., None])


def test_burgers_characteristic_solution_and_spatial_order():
    # shock time 1 / max(-u0') = 1 / (0.5 pi) ~ 0.64; march to t = 0.2
    N, s, dt, nslabs = 3, 4, 0.02, 10
    errs = [_burgers_error(K, N, s, dt, nslabs) for K in (8, 16, 32)]
    assert errs[-1] < 2e-6, errs
    eoc = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    # order N+1 = 4 (Sec. 5.2: p+1 for smooth solutions)
    assert eoc[-1] > N + 1 - 0.5, (errs, eoc)


def test_burgers_double_speed_flux_would_fail():
    """The characteristic check separates u^2/2 from u^2: with the solution of a
    flux twice as large (u_t + (u^2)_x = 0, characteristic speed 2u) the error is O(1)."""
    N, s, dt, nslabs, K = 3, 4, 0.02, 10, 16
    g = dgsem.Grid(1, (K,), (0.0,), (1.0,), N, "burgers", {})
    X = g.coordinates()[0]
    u = _u0(X)[..., None]
    F = lambda v: dgsem.spatial_operator(g, v)
    for _ in range(nslabs):
        u = stdg.solve_slab_newton_gmres("stdg", F, u, dt, s, rtol=1e-12, gmres_tol=1e-11)[s - 1]
    T = dt * nslabs
    wrong = stdg.l2_error_overintegrated(g, u, lambda x: _characteristic(x, 2 * T)[..., None])
    right = stdg.l2_error_overintegrated(g, u, lambda x: _characteristic(x, T)[..., None])
    assert right < 1e-4 and wrong > 1e-2, (right, wrong)


# ------------------------------------------------------------------ LGL-weighted norm


def _lgl_nodes(n):
    """LGL nodes on [-1, 1]: the end points and the roots of P_{n-1}' (numpy Legendre)."""
    c = np.zeros(n)
    c[-1] = 1.0
    inner = np.polynomial.legendre.Legendre(c).deriv().roots()
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


@pytest.mark.parametrize("dim,cells,N,s,r", [(1, (5,), 3, 3, 1), (2, (3, 2), 2, 4, 4), (3, (2, 1, 2), 2, 2, 5)])
def test_norm_of_constant(dim, cells, N, s, r):
    eq = "euler" if r > 1 else "advection"
    lo, hi = (-0.5, 0.0, 1.0)[:dim], (1.5, 3.0, 1.25)[:dim]
    g = dgsem.Grid(dim, cells, lo, hi, N, eq, {"adv_vel": (1.0, 1.0, 1.0), "gamma": 1.4})
    V = float(np.prod([hi[a] - lo[a] for a in range(dim)]))
    c = -1.75
    u = np.full(g.state_shape, c)
    U = np.stack([u] * s)
    assert stdg.lgl_weighted_norm(g, U) == pytest.approx(abs(c) * np.sqrt(2.0 * V * r), rel=1e-13)
    assert stdg.lgl_weighted_norm(g, u) == pytest.approx(abs(c) * np.sqrt(V * r), rel=1e-13)


@pytest.mark.parametrize("N,s", [(3, 3), (4, 4), (2, 5)])
def test_norm_of_polynomial_is_the_exact_integral(N, s):
    """U(x, y, tau) = (p(x), q(y) t(tau)) per component on a 2D grid, p and q of degree N-1,
    t of degree s-2: |U|^2 is within the exactness of both LGL rules (2N-1 and 2s-3)."""
    lo, hi, cells = (0.25, -1.0), (1.75, 1.0), (3, 2)
    g = dgsem.Grid(2, cells, lo, hi, N, "euler", {"gamma": 1.4})
    rng = np.random.default_rng(5)
    pc = rng.uniform(-1, 1, N)          # degree N-1 in x
    qc = rng.uniform(-1, 1, N)          # degree N-1 in y
    tc = rng.uniform(-1, 1, s - 1)      # degree s-2 in tau
    wc = rng.uniform(-1, 1, N)          # second component, degree N-1 in x only
    X, Y = g.coordinates()
    tau = _lgl_nodes(s)
    U = np.zeros((s,) + g.state_shape)
    for m in range(s):
        U[m, ..., 0] = npoly.polyval(X, pc) * npoly.polyval(Y, qc) * npoly.polyval(tau[m], tc)
        U[m, ..., 2] = npoly.polyval(X, wc)
    def integral(c, a, b):
        P = npoly.polyint(npoly.polymul(c, c))
        return npoly.polyval(b, P) - npoly.polyval(a, P)
    Ix, Iy, It = integral(pc, lo[0], hi[0]), integral(qc, lo[1], hi[1]), integral(tc, -1.0, 1.0)
    Iw = integral(wc, lo[0], hi[0]) * (hi[1] - lo[1]) * 2.0
    exact = np.sqrt(Ix * Iy * It + Iw)
    assert stdg.lgl_weighted_norm(g, U) == pytest.approx(exact, rel=1e-12)
    # one time level: the spatial integral alone
    u = U[1]
    exact1 = np.sqrt(Ix * Iy * npoly.polyval(tau[1], tc) ** 2 + Iw / 2.0)
    assert stdg.lgl_weighted_norm(g, u) == pytest.approx(exact1, rel=1e-12)
