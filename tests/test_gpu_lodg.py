"""Method-of-lines DG-SEM + Lobatto IIIC (LoDG) residuals on the GPU (stdg_lodg_residual).

* Parity with the oracle: form 0 against oracle.stdg.lodg_residual (Eq. DG_vs_RK:RK with A
  from Eq. SBP_to_RK); form 1 (the A^-1 form) against ((dt A)^-1 (x) I)(U - 1 (x) u^n) - F(U)
  assembled here from the oracle's tableau and spatial operator.
* Equivalence of the formulations on the device: the space-time residual of the library equals
  -(dt/2)(M_tau (x) I) times its A^-1 form residual (to rounding), and at the space-time slab
  solution the Lobatto IIIC stage equations hold (the theorem of Sec. 5).
"""
import numpy as np
import pytest

from helpers import Problem
from oracle import lgl, stdg as ost
from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [dict(dim=1, cells=(9,), N=3, s=3, eq="advection", dt=0.02, adv=(1.0,)),
         dict(dim=2, cells=(5, 4), N=4, s=4, eq="euler", dt=0.01),
         dict(dim=2, cells=(3, 3), N=2, s=5, eq="burgers", dt=0.02, nu=0.01),
         dict(dim=3, cells=(2, 3, 2), N=2, s=2, eq="euler", dt=0.01)]


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


def _scale(prob, U, u_n):
    A, _, _ = lgl.lobatto_iiic_from_dgsem(prob.s)
    fmax = max(np.max(np.abs(prob.F(U[m]))) for m in range(prob.s))
    return np.max(np.abs(U)) + np.max(np.abs(u_n)) + prob.dt * prob.s * np.max(np.abs(A)) * fmax


@pytest.mark.parametrize("case", CASES)
def test_lodg_residual_parity(S, case):
    prob = Problem(**case)
    u_n = prob.rough_state(5)
    U = prob.rough_slab(u_n, 6)
    un = np.ascontiguousarray(u_n).ravel()
    with S.Context(prob.config()) as ctx:
        R0 = prob.from_ext(ctx.lodg_residual(prob.ext(U), un, form=0))
        R1 = prob.from_ext(ctx.lodg_residual(prob.ext(U), un, form=1))
    scale = _scale(prob, U, u_n)
    R0_or = ost.lodg_residual(prob.F, U, u_n, prob.dt)
    assert np.max(np.abs(R0 - R0_or)) <= 1e-12 * scale
    A, _, _ = lgl.lobatto_iiic_from_dgsem(prob.s)
    Ainv = np.linalg.inv(prob.dt * A)
    FU = np.stack([prob.F(U[m]) for m in range(prob.s)])
    R1_or = np.einsum("ij,j...->i...", Ainv, U - u_n[None]) - FU
    scale1 = np.max(np.abs(Ainv)) * prob.s * (np.max(np.abs(U)) + np.max(np.abs(u_n))) + np.max(np.abs(FU))
    assert np.max(np.abs(R1 - R1_or)) <= 1e-12 * scale1


@pytest.mark.parametrize("case", CASES)
def test_space_time_residual_is_scaled_ainv_form(S, case):
    prob = Problem(**case)
    u_n = prob.rough_state(7)
    U = prob.rough_slab(u_n, 8)
    un = np.ascontiguousarray(u_n).ravel()
    with S.Context(prob.config()) as ctx:
        R_st = prob.from_ext(ctx.residual(prob.ext(U), un))
        R1 = prob.from_ext(ctx.lodg_residual(prob.ext(U), un, form=1))
    _, M, _, _ = lgl.temporal_matrices(prob.s)
    rhs = -0.5 * prob.dt * np.einsum("i,i...->i...", np.diag(M), R1)
    assert np.max(np.abs(R_st - rhs)) <= 1e-12 * prob.term_scale(U, u_n)


def test_stage_equations_hold_at_the_space_time_solution(S):
    prob = Problem(dim=2, cells=(6, 6), N=4, s=4, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(10.0, 10.0))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(5.0, 5.0))
    prob.dt = 0.15
    tight = dict(newton_rtol=1e-14, newton_atol=1e-13, newton_maxit=12, gmres_rtol=1e-11, gmres_maxit=600)
    with S.Context(prob.config(**tight)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        ctx.advance_slab()
        Ue = ctx.get_slab()
        R0 = prob.from_ext(ctx.lodg_residual(Ue, np.ascontiguousarray(u0).ravel(), form=0))
    U = prob.from_ext(Ue)
    # the LoDG stage residual of the STDG solution is at the level of the solve tolerance
    assert np.max(np.abs(R0)) <= 1e-11 * _scale(prob, U, u0)
    # and u^{n+1} = U^s equals the Runge-Kutta update u^n + dt b^T F(U) (stiffly accurate: A's last row = b)
    _, b, _ = lgl.lobatto_iiic_from_dgsem(prob.s)
    u_rk = u0 + prob.dt * sum(b[j] * prob.F(U[j]) for j in range(prob.s))
    assert np.max(np.abs(u_rk - U[prob.s - 1])) <= 1e-11 * np.max(np.abs(u0))
