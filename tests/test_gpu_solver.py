"""GPU slab solves (Newton + GMRES, stdg_advance_slab) against the oracle's solves.

Both sides iterate far below the configs' tolerances (parity reading of the
Newton stop rule), so the comparison measures the discrete scheme, not the
solver: relative LGL-weighted L2 difference <= 1e-11 in FP64 (the stated
FP64 target).  Failure statuses are produced on the host (NaN input, tiny
memory budget, iteration cap); no GPU fault is involved."""
import numpy as np
import pytest

from helpers import Problem, rel_lgl
from oracle import dgsem, physics, stdg as ost
from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu

TIGHT = dict(newton_rtol=1e-14, newton_atol=1e-13, newton_maxit=12, gmres_m=30, gmres_rtol=1e-11,
             gmres_maxit=600)


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


def _cfl_dt(prob, u0, cfl=0.5):
    lam = max(np.max(physics.wave_speed(prob.eq, u0, a, prob.grid.params)) for a in range(prob.dim))
    return cfl * min(prob.grid.h) / lam


def test_config1_advection_100_slabs(S):
    """1D advection, 16 elements, N = 3, s = 3, dt = 0.01, 100 slabs, u0 = sin(2 pi x)."""
    prob = Problem(dim=1, cells=(16,), N=3, s=3, eq="advection", dt=0.01, adv=(1.0,))
    u0 = inputs.sine(prob.grid.coordinates()[0])
    ref = ost.march("stdg", prob.F, u0, prob.dt, prob.s, 100)
    with S.Context(prob.config(**TIGHT)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        for _ in range(100):
            st = ctx.advance_slab()
        u = ctx.get_state().reshape(u0.shape)
    err = ost.lgl_weighted_norm(prob.grid, u - ref[-1]) / ost.lgl_weighted_norm(prob.grid, ref[-1])
    assert err <= 1e-11, err
    assert st["newton_its"] >= 1 and st["gmres_its"] >= 1


@pytest.mark.parametrize("jv,precond", [("fd", 2), ("exact", 2), ("fd", 1), ("exact", 1), ("fd", 0)])
def test_vortex_slab_matches_oracle(S, jv, precond):
    """2D Euler vortex on [0,10]^2, 8x8 quads, N = 4, s = 4, CFL 0.5: one slab with the
    point-block preconditioner (2), the left temporal-mass scaling (1) and none (0)."""
    prob = Problem(dim=2, cells=(8, 8), N=4, s=4, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(10.0, 10.0))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(5.0, 5.0))
    prob.dt = _cfl_dt(prob, u0)
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)
    mode = S.JV_FD if jv == "fd" else S.JV_EXACT
    with S.Context(prob.config(jv_mode=mode, precond=precond, **TIGHT)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        st = ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
        u1 = ctx.get_state().reshape(u0.shape)
    assert rel_lgl(prob, U, U_or) <= 1e-11, rel_lgl(prob, U, U_or)
    assert np.array_equal(u1, U[prob.s - 1])
    # conservation of the cell sums over the slab (periodic, converged)
    cons = dgsem.integrate(prob.grid, u1) - dgsem.integrate(prob.grid, u0)
    assert np.max(np.abs(cons)) <= 1e-11 * np.max(np.abs(dgsem.integrate(prob.grid, u0)))
    assert st["res_final"] <= max(1e-14 * st["res0"], 1e-13)


def test_density_wave_3d_slab_matches_oracle(S):
    prob = Problem(dim=3, cells=(3, 3, 3), N=3, s=3, eq="euler", dt=0.01)
    u0 = inputs.density_wave(*prob.grid.coordinates())
    prob.dt = _cfl_dt(prob, u0)
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)
    with S.Context(prob.config(**TIGHT)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
    assert rel_lgl(prob, U, U_or) <= 1e-11, rel_lgl(prob, U, U_or)


def test_euler_tiny_matches_dense_newton(S):
    """Brute force: the oracle's dense-Jacobian Newton on a 2x2, N = 2, s = 2 grid."""
    prob = Problem(dim=2, cells=(2, 2), N=2, s=2, eq="euler", dt=0.02)
    u_n = inputs.perturbed(inputs.density_wave(*prob.grid.coordinates()), 4, 0.02)
    U_or, _ = ost.solve_slab_direct("stdg", prob.F, u_n, prob.dt, prob.s)
    with S.Context(prob.config(**TIGHT)) as ctx:
        ctx.set_state(np.ascontiguousarray(u_n).ravel())
        ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
    assert rel_lgl(prob, U, U_or) <= 1e-11


def test_free_stream_needs_no_newton_step(S):
    prob = Problem(dim=2, cells=(5, 4), N=4, s=4, eq="euler", dt=0.05)
    u = np.broadcast_to(np.array([1.0, 0.5, -0.25, 3.0]), prob.grid.state_shape).copy()
    with S.Context(prob.config(newton_atol=1e-12)) as ctx:
        ctx.set_state(np.ascontiguousarray(u).ravel())
        st = ctx.advance_slab()
        assert st["newton_its"] == 0
        assert np.max(np.abs(ctx.get_state() - u.ravel())) <= 1e-14


def test_failure_statuses_from_host_inputs(S):
    prob = Problem(dim=2, cells=(4, 4), N=2, s=2, eq="euler", dt=0.05)
    u = inputs.density_wave(*prob.grid.coordinates())
    bad = np.ascontiguousarray(u).ravel().copy()
    bad[7] = np.nan
    with S.Context(prob.config()) as ctx:
        ctx.set_state(bad)
        st = ctx.advance_slab(check=False)
        assert st["status"] == 6  # STDG_ERR_NAN
        ctx.set_state(np.ascontiguousarray(u).ravel())
        assert ctx.advance_slab(check=False)["status"] == 0
    with S.Context(prob.config(newton_rtol=1e-15, newton_atol=0.0, newton_maxit=1, gmres_rtol=0.5)) as ctx:
        ctx.set_state(np.ascontiguousarray(u).ravel())
        assert ctx.advance_slab(check=False)["status"] == 4  # STDG_ERR_NOT_CONVERGED
    with pytest.raises(S.StdgError) as e:
        S.Context(prob.config(hbm_budget_bytes=1024))
    assert e.value.status == 2  # STDG_ERR_OOM


@pytest.mark.parametrize("jv", ["fd", "exact"])
def test_mixed_precision_refines_to_fp64_solution(S, jv):
    """STDG_MIXED_FP32: FP32 Jacobian-vector products and Krylov basis inside FP64 Newton.
    Iterated to FP64 tolerances the FP64 residual refines the solution to the oracle's
    FP64 solution (1e-11); at the workload tolerances (rtol 1e-10, eta 1e-3) it stays
    within the stated 1e-8 of it."""
    prob = Problem(dim=2, cells=(8, 8), N=4, s=4, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(10.0, 10.0))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(5.0, 5.0))
    prob.dt = _cfl_dt(prob, u0)
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)
    mode = S.JV_FD if jv == "fd" else S.JV_EXACT
    tight = dict(TIGHT, gmres_rtol=1e-4, newton_maxit=30)
    with S.Context(prob.config(jv_mode=mode, precision=S.MIXED_FP32, **tight)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        st = ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
    assert rel_lgl(prob, U, U_or) <= 1e-11, (rel_lgl(prob, U, U_or), st)
    with S.Context(prob.config(jv_mode=mode, precision=S.MIXED_FP32, newton_rtol=1e-10,
                               gmres_rtol=1e-3)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
    assert rel_lgl(prob, U, U_or) <= 1e-8, rel_lgl(prob, U, U_or)


def test_mixed_precision_density_wave_3d(S):
    prob = Problem(dim=3, cells=(3, 3, 3), N=3, s=3, eq="euler", dt=0.01)
    u0 = inputs.density_wave(*prob.grid.coordinates())
    prob.dt = _cfl_dt(prob, u0)
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)
    with S.Context(prob.config(precision=S.MIXED_FP32, jv_mode=S.JV_EXACT,
                               **dict(TIGHT, gmres_rtol=1e-4, newton_maxit=30))) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
    assert rel_lgl(prob, U, U_or) <= 1e-11, rel_lgl(prob, U, U_or)


@pytest.mark.parametrize("eq,dim,cells,N,s,nu", [("advection", 2, (6, 5), 3, 3, 0.01),
                                                ("advection", 1, (8,), 4, 4, 0.05),
                                                ("burgers", 2, (5, 5), 3, 3, 0.02)])
def test_viscous_slab_matches_oracle(S, eq, dim, cells, N, s, nu):
    """Slab solves with the interior-penalty viscous term (FP64 FD Jv; mixed precision with
    exact FP32 Jv) against the oracle's."""
    prob = Problem(dim=dim, cells=cells, N=N, s=s, eq=eq, dt=0.02, nu=nu, adv=(0.7, -0.4))
    X = prob.grid.coordinates()
    u0 = inputs.burgers_fourier(X[0], X[1], 1003) if dim == 2 else inputs.sine(X[0])
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)
    for extra in (dict(), dict(precision=S.MIXED_FP32, jv_mode=S.JV_EXACT, gmres_rtol=1e-4, newton_maxit=30)):
        with S.Context(prob.config(**dict(TIGHT, **extra))) as ctx:
            ctx.set_state(np.ascontiguousarray(u0).ravel())
            ctx.advance_slab()
            U = prob.from_ext(ctx.get_slab())
        assert rel_lgl(prob, U, U_or) <= 1e-11, (extra, rel_lgl(prob, U, U_or))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_extrapolated_guess_reaches_the_same_slabs(S, precision):
    """The extrapolated initial iterate (previous slab's temporal polynomial at tau + 2) changes
    where Newton starts, not what it converges to: five vortex slabs agree with the constant
    guess's to the solve tolerance, the first slab (no previous slab) is unchanged, and the
    later slabs take fewer Newton steps."""
    prob = Problem(dim=2, cells=(8, 8), N=4, s=4, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(10.0, 10.0))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(5.0, 5.0))
    prob.dt = _cfl_dt(prob, u0)
    prec = S.FP64 if precision == "fp64" else S.MIXED_FP32
    tol = dict(newton_rtol=1e-12, newton_atol=1e-14, newton_maxit=20, gmres_rtol=0.05, gmres_maxit=600)
    runs = {}
    for pred in (S.PREDICTOR_CONSTANT, S.PREDICTOR_EXTRAPOLATE):
        with S.Context(prob.config(precision=prec, predictor=pred, **tol)) as ctx:
            ctx.set_state(np.ascontiguousarray(u0).ravel())
            stats = [ctx.advance_slab() for _ in range(5)]
            runs[pred] = (prob.from_ext(ctx.get_slab()), stats)
    (U0, st0), (U1, st1) = runs[S.PREDICTOR_CONSTANT], runs[S.PREDICTOR_EXTRAPOLATE]
    assert rel_lgl(prob, U1, U0) <= 1e-10, rel_lgl(prob, U1, U0)
    assert st1[0] == st0[0]
    for a, b in zip(st0[1:], st1[1:]):
        # same target (relative to the constant guess), reached from a closer start
        assert abs(b["res0"] - a["res0"]) <= 1e-6 * a["res0"]
        assert b["res_final"] <= max(1e-12 * b["res0"], 1e-14)
    assert sum(s["newton_its"] for s in st1[1:]) < sum(s["newton_its"] for s in st0[1:])
