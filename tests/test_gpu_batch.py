"""Batched device-driven slab solves (stdg_batch_*) through the C ABI.

* Every slot of a mixed batch (different grids, N, s, dt) reaches the oracle's
  FP64 slab solution: 1e-11 (relative LGL-weighted L2) when iterated to FP64
  tolerances (the FP64 residual refines the FP32 Krylov solves), 1e-8 at the
  workload tolerances (Newton rtol 1e-10, GMRES rtol 1e-3).
* A slot's result is bitwise the same alone and in a mix of other slots.
* Admission by memory: a full arena refuses a slot with STDG_ERR_OOM; removing
  a finished slot makes room.
"""
import numpy as np
import pytest

from helpers import Problem, rel_lgl
from oracle import physics, stdg as ost
from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu

TIGHT = dict(newton_rtol=1e-14, newton_atol=1e-13, newton_maxit=30, gmres_m=30, gmres_rtol=1e-4)
WORK = dict(newton_rtol=1e-10, newton_atol=0.0, newton_maxit=30, gmres_m=30, gmres_rtol=1e-3)


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


def _vortex(cells, N, s, box=10.0):
    prob = Problem(dim=2, cells=cells, N=N, s=s, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(box, box))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(box / 2, box / 2))
    lam = max(np.max(physics.wave_speed("euler", u0, a, prob.grid.params)) for a in range(2))
    prob.dt = 0.5 * min(prob.grid.h) / lam
    return prob, u0


def _advection(cells, N, s, dt):
    prob = Problem(dim=1, cells=cells, N=N, s=s, eq="advection", dt=dt, adv=(1.0,))
    return prob, inputs.sine(prob.grid.coordinates()[0])


def _oracle(prob, u0):
    return ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-14, atol=1e-13,
                                       gmres_tol=1e-11, gmres_m=40)


# (cells, N, s) of the 2D vortex on [0,10]^2 at CFL 0.5.  The N = 6 grid is stiff (nodal CFL
# number ~ 12): its residual stalls near 1e-13 (FP64 rounding), so it is iterated to the
# workload tolerances only.
EULER_MIX = [((4, 4), 3, 3), ((6, 5), 4, 4), ((3, 4), 2, 2), ((5, 3), 5, 5), ((4, 4), 6, 3)]


@pytest.mark.parametrize("tol,bound,cases", [(TIGHT, 1e-11, EULER_MIX[:4]), (WORK, 1e-8, EULER_MIX)])
def test_euler_mix_matches_oracle(S, tol, bound, cases):
    probs = [_vortex(*c) for c in cases]
    with S.Batch(2, S.EULER, 16, 256 << 20) as B:
        slots = [B.add(p.config(**tol), np.ascontiguousarray(u0).ravel()) for p, u0 in probs]
        assert B.run(20000) == 0
        for (p, u0), slot in zip(probs, slots):
            done, status, st = B.query(slot)
            assert done and status == 0, (status, st)
            U = p.from_ext(B.get_slab(slot))
            err = rel_lgl(p, U, _oracle(p, u0))
            assert err <= bound, (p.cells, p.N, p.s, err, st)
            u1 = B.get_state(slot).reshape(u0.shape)
            assert np.array_equal(u1, U[p.s - 1])


def test_advection_mix_matches_oracle(S):
    cases = [((16,), 3, 3, 0.01), ((7,), 5, 2, 0.03), ((9,), 2, 5, 0.05), ((1,), 4, 4, 0.02)]
    probs = [_advection(*c) for c in cases]
    with S.Batch(1, S.ADVECTION, 8, 64 << 20) as B:
        slots = [B.add(p.config(**TIGHT), np.ascontiguousarray(u0).ravel()) for p, u0 in probs]
        B.run(20000)
        for (p, u0), slot in zip(probs, slots):
            done, status, st = B.query(slot)
            assert done and status == 0
            U = p.from_ext(B.get_slab(slot))
            assert rel_lgl(p, U, _oracle(p, u0)) <= 1e-11


def test_alone_equals_in_mix_bitwise(S):
    probs = [_vortex(*c) for c in EULER_MIX]
    target = 1
    p, u0 = probs[target]
    with S.Batch(2, S.EULER, 4, 64 << 20) as B:
        s_alone = B.add(p.config(**WORK), np.ascontiguousarray(u0).ravel())
        B.run(20000)
        alone = B.get_slab(s_alone)
        st_alone = B.query(s_alone)[2]
    with S.Batch(2, S.EULER, 16, 256 << 20) as B:
        # others admitted before and after, and one admitted while the target is running
        first = [B.add(q.config(**WORK), np.ascontiguousarray(v).ravel()) for q, v in probs[:1]]
        s_mix = B.add(p.config(**WORK), np.ascontiguousarray(u0).ravel())
        B.step(5)
        late = [B.add(q.config(**WORK), np.ascontiguousarray(v).ravel()) for q, v in probs[2:]]
        B.run(20000)
        mixed = B.get_slab(s_mix)
        st_mix = B.query(s_mix)[2]
        assert all(B.query(sl)[0] for sl in first + late)
    assert np.array_equal(alone, mixed)
    assert st_alone == st_mix


def test_admission_by_memory(S):
    p, u0 = _vortex((8, 8), 4, 4)
    with S.Batch(2, S.EULER, 4, 1 << 20) as probe:
        need = probe.slot_bytes(p.config(**WORK))
    with S.Batch(2, S.EULER, 4, need + need // 2) as B:
        a = B.add(p.config(**WORK), np.ascontiguousarray(u0).ravel())
        assert B.try_add(p.config(**WORK), np.ascontiguousarray(u0).ravel()) is None
        B.run(20000)
        assert B.query(a)[0]
        B.remove(a)
        b = B.try_add(p.config(**WORK), np.ascontiguousarray(u0).ravel())
        assert b is not None
        B.run(20000)
        assert B.query(b)[:2] == (True, 0)


def test_failure_statuses(S):
    p, u0 = _vortex((4, 4), 3, 3)
    bad = np.ascontiguousarray(u0).ravel().copy()
    bad[5] = np.nan
    with S.Batch(2, S.EULER, 4, 64 << 20) as B:
        s_nan = B.add(p.config(**WORK), bad)
        s_cap = B.add(p.config(**dict(WORK, newton_rtol=1e-15, newton_maxit=1, gmres_rtol=0.5)),
                      np.ascontiguousarray(u0).ravel())
        s_ok = B.add(p.config(**WORK), np.ascontiguousarray(u0).ravel())
        B.run(20000)
        assert B.query(s_nan)[:2] == (True, 6)   # STDG_ERR_NAN
        assert B.query(s_cap)[:2] == (True, 4)   # STDG_ERR_NOT_CONVERGED
        assert B.query(s_ok)[:2] == (True, 0)


def _burgers(i, max_side=16):
    """Instance i of the batched viscous Burgers workload (grid side capped for the oracle),
    dt = 0.5 h / max |u0| (CFL 0.5 on the initial data)."""
    spec = inputs.burgers_instance(i, sides=tuple(x for x in (8, 16, 32, 64) if x <= max_side))
    side = spec["side"]
    prob = Problem(dim=2, cells=(side, side), N=spec["N"], s=spec["s"], eq="burgers", dt=1.0, nu=spec["nu"])
    X = prob.grid.coordinates()
    u0 = inputs.burgers_fourier(X[0], X[1], spec["seed"])
    prob.dt = 0.5 * (1.0 / side) / np.max(np.abs(u0))
    return prob, u0


def test_viscous_burgers_mix_matches_oracle(S):
    """Six instances of the batched viscous Burgers workload (8^2 and 16^2 grids) in one batch:
    each slot within 1e-8 of the oracle at the workload tolerances."""
    probs = [_burgers(i) for i in range(6)]
    with S.Batch(2, S.BURGERS, 8, 256 << 20) as B:
        slots = [B.add(p.config(**WORK), np.ascontiguousarray(u0).ravel()) for p, u0 in probs]
        assert B.run(20000) == 0
        for (p, u0), slot in zip(probs, slots):
            done, status, st = B.query(slot)
            assert done and status == 0, (status, st)
            U = p.from_ext(B.get_slab(slot))
            err = rel_lgl(p, U, _oracle(p, u0))
            assert err <= 1e-8, (p.cells, p.N, p.s, p.nu, err, st)


def test_scheduling_knobs_keep_results(S):
    """Size-aware sharing (a large slot advances every k-th tick) and graph replay change only
    when slots advance: results are bitwise those of plain ticking.  Tile autotuning changes
    the CTA tiling of the operator only: results agree to rounding."""
    probs = [_vortex(*c) for c in EULER_MIX[:4]] + [_vortex((12, 10), 4, 4)]
    results = {}
    for name, kw in [("plain", dict(use_graphs=False, autotune=False)),
                     ("graphs", dict(use_graphs=True, autotune=False)),
                     ("shared", dict(share_quantum=2000.0, share_max_stride=8, use_graphs=True, autotune=False)),
                     ("tuned", dict(use_graphs=True, autotune=True))]:
        with S.Batch(2, S.EULER, 8, 256 << 20) as B:
            B.configure(**kw)
            slots = [B.add(p.config(**WORK), np.ascontiguousarray(u0).ravel()) for p, u0 in probs]
            assert B.run(50000) == 0
            results[name] = [(B.query(sl)[1], B.get_slab(sl)) for sl in slots]
    for name in ("graphs", "shared"):
        for (st0, U0), (st1, U1) in zip(results["plain"], results[name]):
            assert st1 == st0 == 0 and np.array_equal(U0, U1), name
    for (p, _), (_, U0), (st1, U1) in zip(probs, results["plain"], results["tuned"]):
        assert st1 == 0 and rel_lgl(p, p.from_ext(U1), p.from_ext(U0)) <= 1e-9


def test_element_preconditioner_cuts_iterations_on_stiff_viscous_slots(S):
    """Viscous Burgers instances with N = 6 and nu ~ 0.07-0.1 on 8^2 grids: the element tensor-
    product preconditioner (default for scalar equations) needs far fewer GMRES iterations than
    the point-block one and both reach the oracle's slab."""
    probs = [_burgers(i) for i in (60, 79)]
    its = {}
    for pc in (S.PRECOND_POINT_BLOCK, S.PRECOND_TEMPORAL_MASS):
        with S.Batch(2, S.BURGERS, 4, 256 << 20) as B:
            slots = [B.add(p.config(**dict(WORK, precond=pc, newton_maxit=60)), np.ascontiguousarray(u0).ravel())
                     for p, u0 in probs]
            assert B.run(100000) == 0
            its[pc] = []
            for (p, u0), sl in zip(probs, slots):
                done, status, st = B.query(sl)
                assert status == 0, (pc, st)
                its[pc].append(st["gmres_its"])
                if pc == S.PRECOND_TEMPORAL_MASS:
                    assert rel_lgl(p, p.from_ext(B.get_slab(sl)), _oracle(p, u0)) <= 1e-8
    for a, b in zip(its[S.PRECOND_TEMPORAL_MASS], its[S.PRECOND_POINT_BLOCK]):
        assert a < 0.6 * b, its


def test_global_preconditioner_is_exact_for_pure_diffusion(S):
    """u_t = nu (u_xx + u_yy) (advection with zero velocity, viscous): the global fast-
    diagonalisation preconditioner of scalar slots inverts the slab Jacobian exactly (the linear
    operator has no convective part), so every Newton step needs one or two FGMRES iterations
    (FP32 rounding of the transforms); the slab reaches the oracle's."""
    prob = Problem(dim=2, cells=(8, 16), N=4, s=4, eq="advection", dt=0.02, adv=(0.0, 0.0), nu=0.05)
    X = prob.grid.coordinates()
    u0 = (np.sin(2 * np.pi * X[0]) * np.cos(4 * np.pi * X[1]) + 0.3 * np.sin(6 * np.pi * X[1]))[..., None]
    with S.Batch(2, S.ADVECTION, 2, 256 << 20) as B:
        sl = B.add(prob.config(**WORK), np.ascontiguousarray(u0).ravel())
        assert B.run(20000) == 0
        done, status, st = B.query(sl)
        assert status == 0 and st["newton_its"] >= 1, st
        assert st["gmres_its"] <= 2 * st["newton_its"], st
        assert rel_lgl(prob, prob.from_ext(B.get_slab(sl)), _oracle(prob, u0)) <= 1e-8


def test_global_preconditioner_on_a_1d_viscous_advection_slot(S):
    """1D advection-diffusion (16 elements, N = 5, s = 5): the global preconditioner handles the
    dissipation of the upwind flux as well; few iterations, the oracle's slab."""
    prob = Problem(dim=1, cells=(16,), N=5, s=5, eq="advection", dt=0.05, adv=(1.0,), nu=0.02)
    u0 = inputs.sine(prob.grid.coordinates()[0])
    with S.Batch(1, S.ADVECTION, 2, 64 << 20) as B:
        sl = B.add(prob.config(**WORK), np.ascontiguousarray(u0).ravel())
        assert B.run(20000) == 0
        done, status, st = B.query(sl)
        assert status == 0, st
        assert st["gmres_its"] <= 12 * st["newton_its"], st
        assert rel_lgl(prob, prob.from_ext(B.get_slab(sl)), _oracle(prob, u0)) <= 1e-8


def test_stiffest_workload_instances_converge(S):
    """The stiffest instances of the batched viscous Burgers workload (N = 6, s = 4 or 5,
    nu ~ 0.03-0.09 on 32^2 and 64^2 grids, dt/2 times the largest element eigenvalue above 1e4),
    which the element-local preconditioner left at the Newton cap: with the global preconditioner
    each converges, alone and together, with the same result."""
    import bench
    items = bench._burgers_instances(S, 301)
    ids = (113, 186, 264, 280, 300)
    with S.Batch(2, S.BURGERS, 8, 8 << 30) as B:
        slots = [B.add(items[i][0], items[i][1]) for i in ids]
        assert B.run(200000) == 0
        mixed = []
        for i, sl in zip(ids, slots):
            done, status, st = B.query(sl)
            assert done and status == 0, (i, st)
            mixed.append(B.get_state(sl))
    with S.Batch(2, S.BURGERS, 2, 4 << 30) as B:
        sl = B.add(items[ids[0]][0], items[ids[0]][1])
        assert B.run(200000) == 0
        assert np.array_equal(B.get_state(sl), mixed[0])


def test_long_slot_takes_the_wide_dot_pass(S):
    """A slot of at least 2^21 values takes the 16-row dot pass (64 x 64 vortex, N = 5, s = 4:
    2,359,296 values), a small one the 8-row pass.  The long slot's slab agrees with the
    single-slab FP64 path's (pinned against the oracle at full size elsewhere) to the workload
    tolerance, and it is bitwise the same alone and next to the small slot."""
    prob, u0 = _vortex((64, 64), 5, 4)
    assert 64 * 64 * 36 * 4 * 4 >= 1 << 21
    small, us = _vortex((4, 4), 3, 3)
    with S.Context(prob.config(**WORK)) as c:
        c.set_state(np.ascontiguousarray(u0).ravel())
        st = c.advance_slab()
        assert st["status"] == 0, st
        U_ref = prob.from_ext(c.get_slab())
    out = []
    for with_small in (False, True):
        with S.Batch(2, S.EULER, 4, 4 << 30) as B:
            if with_small:
                s_small = B.add(small.config(**WORK), np.ascontiguousarray(us).ravel())
            sl = B.add(prob.config(**WORK), np.ascontiguousarray(u0).ravel())
            assert B.run(20000) == 0
            done, status, stb = B.query(sl)
            assert done and status == 0, (status, stb)
            if with_small:
                assert B.query(s_small)[1] == 0
            out.append(B.get_slab(sl).copy())
    assert np.array_equal(out[0], out[1])
    assert rel_lgl(prob, prob.from_ext(out[0]), U_ref) <= 1e-8
