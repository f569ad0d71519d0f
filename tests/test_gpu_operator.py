"""GPU parity of the space-time operator against the oracle, through the C ABI.

R(U; u_prev) and J(U) v of the library (strong form, fused CUDA kernel) vs the
oracle (weak form, complex-step derivative) on the same seeded inputs.
Tolerances are derived in tests/helpers.py (FP64 rounding of differently
associated sums, 1e-12 of the term scale).  Shapes cover every dimension and
equation, the specialised and the runtime-sized kernels, multi-element tiles
with a ragged last tile, one-element periodic grids (an element is its own
neighbour) and the full 64x64, N=4, s=4 vortex grid."""
import numpy as np
import pytest

from helpers import Problem, rel_lgl
from oracle import stdg as ost
from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


CASES = {
    "adv1_fixed": dict(dim=1, cells=(16,), N=3, s=3, eq="advection", dt=0.01, adv=(1.0,)),
    "adv1_generic": dict(dim=1, cells=(7,), N=5, s=2, eq="advection", dt=0.03, adv=(-0.7,)),
    "euler1": dict(dim=1, cells=(9,), N=2, s=4, eq="euler", dt=0.02),
    "euler1_one_elem": dict(dim=1, cells=(1,), N=4, s=3, eq="euler", dt=0.05),
    "euler2_fixed_ragged": dict(dim=2, cells=(21, 17), N=4, s=4, eq="euler", dt=0.01),
    "euler2_generic": dict(dim=2, cells=(5, 3), N=2, s=3, eq="euler", dt=0.02),
    "euler2_one_elem": dict(dim=2, cells=(1, 1), N=3, s=2, eq="euler", dt=0.02),
    "euler2_n8_s5": dict(dim=2, cells=(3, 2), N=7, s=5, eq="euler", dt=0.01),
    "adv2": dict(dim=2, cells=(6, 5), N=3, s=5, eq="advection", dt=0.02),
    "burgers2": dict(dim=2, cells=(4, 6), N=6, s=2, eq="burgers", dt=0.01),
    "euler3_fixed": dict(dim=3, cells=(3, 4, 2), N=3, s=3, eq="euler", dt=0.01),
    "euler3_generic": dict(dim=3, cells=(2, 3, 2), N=2, s=2, eq="euler", dt=0.02),
    "adv3": dict(dim=3, cells=(3, 2, 2), N=1, s=4, eq="advection", dt=0.05),
    # viscous (symmetric interior penalty) terms, scalar equations
    "adv1_visc": dict(dim=1, cells=(7,), N=3, s=3, eq="advection", dt=0.02, adv=(0.8,), nu=0.05),
    "adv1_visc_one_elem": dict(dim=1, cells=(1,), N=4, s=2, eq="advection", dt=0.02, adv=(0.8,), nu=0.1),
    "adv2_visc": dict(dim=2, cells=(5, 3), N=3, s=3, eq="advection", dt=0.01, nu=0.02),
    "burgers2_visc": dict(dim=2, cells=(4, 6), N=5, s=2, eq="burgers", dt=0.01, nu=0.01),
    "burgers2_visc_big": dict(dim=2, cells=(19, 14), N=2, s=4, eq="burgers", dt=0.01, nu=0.003),
}


def _inputs(prob, seed):
    u_n = prob.rough_state(seed)
    U = prob.rough_slab(u_n, seed + 1)
    v = inputs.random_array(U.shape, seed + 2)
    return u_n, U, v


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity(S, name):
    prob = Problem(**CASES[name])
    u_n, U, _ = _inputs(prob, 11)
    R_or = ost.stdg_residual(prob.F, U, u_n, prob.dt)
    with S.Context(prob.config()) as ctx:
        R = prob.from_ext(ctx.residual(prob.ext(U), np.ascontiguousarray(u_n).ravel()))
    tol = 1e-12 * prob.term_scale(U, u_n)
    assert np.max(np.abs(R - R_or)) <= tol, (np.max(np.abs(R - R_or)), tol)


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_jv_parity(S, name):
    prob = Problem(**CASES[name])
    u_n, U, v = _inputs(prob, 23)
    J_or = ost.jv_exact("stdg", prob.F, U, u_n, prob.dt, v)
    with S.Context(prob.config(jv_mode=S.JV_EXACT)) as ctx:
        J = prob.from_ext(ctx.jv(prob.ext(U), np.ascontiguousarray(u_n).ravel(), prob.ext(v)))
    scale = prob.term_scale(U, u_n) * np.max(np.abs(v)) / max(np.max(np.abs(U)), 1e-300)
    assert np.max(np.abs(J - J_or)) <= 1e-11 * max(scale, np.max(np.abs(J_or))), np.max(np.abs(J - J_or))
    assert rel_lgl(prob, J, J_or) <= 1e-12


@pytest.mark.parametrize("name", ["adv1_fixed", "euler1", "euler2_fixed_ragged", "euler3_fixed", "burgers2",
                                  "burgers2_visc"])
def test_fd_jv_close_to_exact(S, name):
    """Finite-difference JFNK product vs the exact derivative: O(eps) truncation, eps ~ 1e-8 relative."""
    prob = Problem(**CASES[name])
    u_n, U, v = _inputs(prob, 31)
    J_or = ost.jv_exact("stdg", prob.F, U, u_n, prob.dt, v)
    with S.Context(prob.config(jv_mode=S.JV_FD)) as ctx:
        J = prob.from_ext(ctx.jv(prob.ext(U), np.ascontiguousarray(u_n).ravel(), prob.ext(v)))
    assert rel_lgl(prob, J, J_or) <= 1e-5, rel_lgl(prob, J, J_or)


def test_device_pointers_match_host(S):
    import torch
    prob = Problem(**CASES["euler2_fixed_ragged"])
    u_n, U, v = _inputs(prob, 41)
    Ue, un, ve = prob.ext(U), np.ascontiguousarray(u_n).ravel(), prob.ext(v)
    with S.Context(prob.config(jv_mode=S.JV_EXACT)) as ctx:
        Rh = ctx.residual(Ue, un)
        Jh = ctx.jv(Ue, un, ve)
        dU, du, dv = (torch.from_numpy(x).cuda() for x in (Ue, un, ve))
        Rd = ctx.residual(dU, du)
        Jd = ctx.jv(dU, du, dv)
        torch.cuda.synchronize()
        assert np.array_equal(Rd.cpu().numpy(), Rh)
        assert np.array_equal(Jd.cpu().numpy(), Jh)
        assert abs(ctx.slab_norm(dU) - np.linalg.norm(Ue)) <= 1e-13 * np.linalg.norm(Ue)


def test_full_size_vortex_grid_parity(S):
    """64 x 64 quads, N = 4, s = 4 on [0, 10]^2 (the 2D Euler vortex workload): residual of a
    perturbed 1 (x) u0 slab and the exact Jv on the full grid against the oracle."""
    prob = Problem(dim=2, cells=(64, 64), N=4, s=4, eq="euler", dt=0.02, lo=(0.0, 0.0), hi=(10.0, 10.0))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(5.0, 5.0))
    U = prob.rough_slab(u0, 5, rel=1e-3)
    v = inputs.random_array(U.shape, 6)
    with S.Context(prob.config(jv_mode=S.JV_EXACT)) as ctx:
        R = prob.from_ext(ctx.residual(prob.ext(U), np.ascontiguousarray(u0).ravel()))
        J = prob.from_ext(ctx.jv(prob.ext(U), np.ascontiguousarray(u0).ravel(), prob.ext(v)))
    R_or = ost.stdg_residual(prob.F, U, u0, prob.dt)
    assert np.max(np.abs(R - R_or)) <= 1e-12 * prob.term_scale(U, u0)
    J_or = ost.jv_exact("stdg", prob.F, U, u0, prob.dt, v)
    assert rel_lgl(prob, J, J_or) <= 1e-12


def test_free_stream_residual_is_zero(S):
    for spec in (CASES["euler2_fixed_ragged"], CASES["euler3_fixed"], CASES["adv1_fixed"]):
        prob = Problem(**spec)
        const = np.array([1.3] + [0.4, -0.2, 0.3][:prob.dim] + [2.9]) if prob.eq == "euler" else np.array([0.6])
        u = np.broadcast_to(const, prob.grid.state_shape).copy()
        U = np.stack([u] * prob.s)
        with S.Context(prob.config()) as ctx:
            R = ctx.residual(prob.ext(U), np.ascontiguousarray(u).ravel())
        assert np.max(np.abs(R)) <= 1e-13 * np.max(np.abs(u))
