"""GPU point-block preconditioner (STDG_PRECOND_POINT_BLOCK) through the C ABI.

* For linear advection the s x s matrix P_I (x) I_r of a spatial node I is
  exactly the block of the slab Jacobian (Eq. Jacobian_ST) that couples the
  temporal nodes and components of I, so z = P^-1 v must equal the inverse of
  that block of the oracle's dense Jacobian applied to v (to rounding).
* For Euler and Burgers the block also holds the wave-speed derivative terms
  the preconditioner drops; there z is checked against P_I assembled here from
  the oracle's wave speeds (Rusanov lambda = max of the two traces per face).
* Slab solves with the preconditioner reach the oracle's solution (1e-11) in
  fewer GMRES iterations than the temporal-mass scaling.
"""
import numpy as np
import pytest

from helpers import Problem, rel_lgl
from oracle import lgl, physics, stdg as ost
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


def _node_blocks(prob, J):
    """Diagonal (s r) x (s r) blocks of a dense slab Jacobian, one per spatial node."""
    shp = (prob.s,) + prob.grid.state_shape
    idx = np.arange(int(np.prod(shp))).reshape(shp)
    d = prob.dim
    perm = tuple(range(1, 2 * d + 1)) + (0, 2 * d + 1)  # (*K_rev, *n_rev, m, c)
    groups = idx.transpose(perm).reshape(-1, prob.s * prob.grid.r)
    return groups, [J[np.ix_(g, g)] for g in groups]


@pytest.mark.parametrize("dim,cells,N,s", [(1, (5,), 3, 3), (2, (3, 2), 2, 4), (3, (2, 2, 2), 1, 2), (1, (1,), 4, 5)])
def test_advection_point_block_is_exact(S, dim, cells, N, s):
    prob = Problem(dim=dim, cells=cells, N=N, s=s, eq="advection", dt=0.07)
    u_n = prob.rough_state(3)
    U = prob.rough_slab(u_n, 4)
    v = inputs.random_array(U.shape, 5)
    J = ost.jacobian_dense("stdg", prob.F, U, u_n, prob.dt)
    groups, blocks = _node_blocks(prob, J)
    z_ref = np.zeros(U.size)
    vf = v.ravel()
    for g, B in zip(groups, blocks):
        z_ref[g] = np.linalg.solve(B, vf[g])
    with S.Context(prob.config()) as ctx:
        z = prob.from_ext(ctx.precond_apply(prob.ext(U), prob.ext(v)))
    z_ref = z_ref.reshape(U.shape)
    assert np.max(np.abs(z - z_ref)) <= 1e-12 * np.max(np.abs(z_ref))


def _p_matrices(prob, U):
    """P_I per spatial node from the oracle's wave speeds (time-major U)."""
    g, s, d, n = prob.grid, prob.s, prob.dim, prob.grid.n
    _, M, D, _ = lgl.temporal_matrices(s)
    om = np.diag(M)
    T = D.T @ M
    T[s - 1, s - 1] -= 1.0
    sig = np.zeros((s,) + g.state_shape[:-1])
    for m in range(s):
        for a in range(d):
            lam = physics.wave_speed(prob.eq, U[m], a, g.params)
            ax_e, ax_n = g.elem_axis(a), g.node_axis(a)
            up = np.take(lam, n - 1, axis=ax_n)
            nb = np.roll(np.take(lam, 0, axis=ax_n), -1, axis=ax_e)
            lf = np.maximum(up, nb) / (g.h[a] * g.w[0])
            hi = [slice(None)] * (2 * d)
            hi[ax_n] = n - 1
            lo = [slice(None)] * (2 * d)
            lo[ax_n] = 0
            sig[m][tuple(hi)] += lf
            sig[m][tuple(lo)] += np.roll(lf, 1, axis=ax_e)
    P = np.broadcast_to(T, sig.shape[1:] + (s, s)).copy()
    for m in range(s):
        P[..., m, m] -= 0.5 * prob.dt * om[m] * sig[m]
    return P


@pytest.mark.parametrize("case", [dict(dim=2, cells=(4, 3), N=4, s=4, eq="euler", dt=0.01),
                                  dict(dim=3, cells=(2, 3, 2), N=3, s=3, eq="euler", dt=0.01),
                                  dict(dim=1, cells=(6,), N=5, s=5, eq="euler", dt=0.02),
                                  dict(dim=2, cells=(3, 3), N=3, s=2, eq="burgers", dt=0.02)])
def test_point_block_apply_matches_definition(S, case):
    prob = Problem(**case)
    u_n = prob.rough_state(8)
    U = prob.rough_slab(u_n, 9)
    v = inputs.random_array(U.shape, 10)
    P = _p_matrices(prob, U)
    # z_m = sum_j (P^-1)[m][j] v_j per node and component
    z_ref = np.einsum("...mj,j...c->m...c", np.linalg.inv(P), v)
    with S.Context(prob.config()) as ctx:
        z = prob.from_ext(ctx.precond_apply(prob.ext(U), prob.ext(v)))
    assert np.max(np.abs(z - z_ref)) <= 1e-12 * np.max(np.abs(z_ref))


def test_point_block_cuts_gmres_iterations(S):
    """2D Euler vortex on [0,10]^2, 8x8 quads, N = 4, s = 4, CFL 0.5: the point-block
    preconditioned solve reaches the oracle's slab (1e-11) with fewer GMRES iterations
    than the temporal-mass scaling, in FP64 (FD Jv) and in mixed precision (exact FP32 Jv)."""
    prob = Problem(dim=2, cells=(8, 8), N=4, s=4, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(10.0, 10.0))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(5.0, 5.0))
    lam = max(np.max(physics.wave_speed("euler", u0, a, prob.grid.params)) for a in range(2))
    prob.dt = 0.5 * min(prob.grid.h) / lam
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)
    its = {}
    jv = {S.FP64: S.JV_FD, S.MIXED_FP32: S.JV_EXACT}  # the precision / Jv pairs the benchmark runs
    for precond in (S.PRECOND_TEMPORAL_MASS, S.PRECOND_POINT_BLOCK):
        for prec in (S.FP64, S.MIXED_FP32):
            with S.Context(prob.config(precond=precond, precision=prec, jv_mode=jv[prec], newton_rtol=1e-10,
                                       gmres_rtol=1e-3)) as ctx:
                ctx.set_state(np.ascontiguousarray(u0).ravel())
                st = ctx.advance_slab()
                its[precond, prec] = st["gmres_its"]
                U = prob.from_ext(ctx.get_slab())
                assert rel_lgl(prob, U, U_or) <= 1e-8
    for prec in (S.FP64, S.MIXED_FP32):
        assert its[S.PRECOND_POINT_BLOCK, prec] < 0.8 * its[S.PRECOND_TEMPORAL_MASS, prec], its
