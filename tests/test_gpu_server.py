"""Continuous-batching server (stdg_server_*) through the C ABI.

Requests of 2D Euler vortex slab solves with different grids, N and s arrive
on a seeded Poisson clock while earlier ones run; the server admits them by
device memory and runs them in shared launches.  Each result must be bitwise
the same as the batch gives for the request alone, and within 1e-8 of the
oracle's FP64 slab (workload tolerances).  A small arena bounds how many run
at once; a request larger than the arena is refused with STDG_ERR_OOM."""
import time

import numpy as np
import pytest

from helpers import Problem, rel_lgl
from oracle import physics, stdg as ost
from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu

WORK = dict(newton_rtol=1e-10, newton_atol=0.0, newton_maxit=30, gmres_m=30, gmres_rtol=1e-3)


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


def _vortex(side, N, s, box=10.0):
    prob = Problem(dim=2, cells=(side, side), N=N, s=s, eq="euler", dt=1.0, lo=(0.0, 0.0), hi=(box, box))
    X = prob.grid.coordinates()
    u0 = inputs.isentropic_vortex(X[0], X[1], center=(box / 2, box / 2))
    lam = max(np.max(physics.wave_speed("euler", u0, a, prob.grid.params)) for a in range(2))
    prob.dt = 0.5 * min(prob.grid.h) / lam
    return prob, u0


def _requests(n, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        side = int(rng.choice([4, 6, 8, 12]))
        N = int(rng.integers(2, 5))
        s = int(rng.integers(2, 5))
        out.append(_vortex(side, N, s))
    return out


def _alone(S, prob, u0):
    with S.Batch(2, S.EULER, 2, 256 << 20) as B:
        slot = B.add(prob.config(**WORK), np.ascontiguousarray(u0).ravel())
        B.run(50000)
        return B.get_state(slot), B.query(slot)


def test_poisson_stream_same_alone_and_in_mix(S):
    reqs = _requests(10)
    rng = np.random.default_rng(11)
    gaps = rng.exponential(1.0 / 400.0, size=len(reqs))  # ~400 requests/s: they overlap
    with S.Server(2, S.EULER, 16, 512 << 20) as srv:
        tickets = []
        for (p, u0), gap in zip(reqs, gaps):
            time.sleep(gap)
            tickets.append(srv.submit(p.config(**WORK), u0))
        results = [srv.poll(t, wait_s=120.0) for t in tickets]
        counters = srv.counters()
    assert counters["fatal"] == 0 and counters["completed"] == len(reqs)
    assert counters["max_running"] >= 2  # requests did share the device
    for (p, u0), r in zip(reqs, results):
        assert r is not None and r["status"] == 0, r
        u_alone, (done, status, st) = _alone(S, p, u0)
        assert done and status == 0
        assert np.array_equal(r["u"], u_alone)
        assert r["stats"] == st
        assert r["latency_s"] >= r["service_s"] >= 0.0
    # accuracy of a few results against the oracle's slab (final temporal node)
    for (p, u0), r in list(zip(reqs, results))[:3]:
        U_or = ost.solve_slab_newton_gmres("stdg", p.F, u0, p.dt, p.s, rtol=1e-14, atol=1e-13, gmres_tol=1e-11,
                                           gmres_m=40)
        u_or = U_or[p.s - 1]
        W = p.grid.jacobian() * p.grid.node_weights()[..., None]
        norm = lambda x: np.sqrt(np.sum(W * x * x))  # LGL-weighted L2 norm of one time level
        err = norm(r["u"].reshape(u0.shape) - u_or) / norm(u_or)
        assert err <= 1e-8, err


def test_admission_by_memory_bounds_concurrency(S):
    p, u0 = _vortex(8, 3, 3)
    with S.Batch(2, S.EULER, 2, 1 << 20) as probe:
        need = probe.slot_bytes(p.config(**WORK))
    u_alone, _ = _alone(S, p, u0)
    with S.Server(2, S.EULER, 16, 2 * need + need // 2) as srv:
        tickets = [srv.submit(p.config(**WORK), u0) for _ in range(6)]
        results = [srv.poll(t, wait_s=120.0) for t in tickets]
        c = srv.counters()
    assert c["completed"] == 6 and c["max_running"] <= 2
    for r in results:
        assert r["status"] == 0 and np.array_equal(r["u"], u_alone)
    # later requests waited in the queue for memory
    assert max(r["queue_s"] for r in results) > 0.0


def test_request_larger_than_arena_is_refused(S):
    p, u0 = _vortex(8, 4, 4)
    with S.Server(2, S.EULER, 4, 1 << 16) as srv:
        t = srv.submit(p.config(**WORK), u0)
        r = srv.poll(t, wait_s=60.0)
    assert r is not None and r["status"] == 2  # STDG_ERR_OOM


def test_cancel_queued_and_running_requests(S):
    """A cancelled request reports STDG_ERR_CANCELLED whether it was queued or running; the
    other requests finish with their alone results.  A bounded queue refuses submissions."""
    p, u0 = _vortex(8, 3, 3)
    u_alone, _ = _alone(S, p, u0)
    with S.Batch(2, S.EULER, 2, 1 << 20) as probe:
        need = probe.slot_bytes(p.config(**WORK))
    with S.Server(2, S.EULER, 8, need + need // 2) as srv:  # one request runs at a time
        tickets = [srv.submit(p.config(**WORK), u0) for _ in range(4)]
        srv.cancel(tickets[2])                 # still queued
        time.sleep(0.05)
        srv.cancel(tickets[0])                 # running (or, if very fast, finished)
        results = [srv.poll(t, wait_s=120.0) for t in tickets]
        srv.set_queue_limit(1)
        more = [srv.submit(p.config(**WORK), u0)]
        with pytest.raises(S.StdgError) as e:
            for _ in range(3):
                more.append(srv.submit(p.config(**WORK), u0))
        assert e.value.status == 2  # STDG_ERR_OOM: the queue is full
        for t in more:
            r = srv.poll(t, wait_s=120.0)
            assert r["status"] == 0 and np.array_equal(r["u"], u_alone)
        assert srv.counters()["fatal"] == 0
    assert results[2]["status"] == 8  # STDG_ERR_CANCELLED
    assert results[0]["status"] in (8, 0)
    if results[0]["status"] == 0:
        assert np.array_equal(results[0]["u"], u_alone)
    for r in (results[1], results[3]):
        assert r["status"] == 0 and np.array_equal(r["u"], u_alone)


@pytest.mark.parametrize("order,cap", [(1, 0.0), (1, 3000.0), (0, 3000.0)])
def test_admission_policy_keeps_results(S, order, cap):
    """Smallest-first admission and a cap on the admitted space-time DOF change only when a
    request runs: every result stays bitwise the one it has alone.  With the cap, the DOF held
    by the admitted requests never exceeds it (a larger request runs alone)."""
    reqs = _requests(8, seed=5)
    with S.Server(2, S.EULER, 16, 512 << 20) as srv:
        srv.set_policy(order, cap)
        tickets = [srv.submit(p.config(**WORK), u0) for p, u0 in reqs]
        results = [srv.poll(t, wait_s=120.0) for t in tickets]
        counters = srv.counters()
    assert counters["fatal"] == 0 and counters["completed"] == len(reqs)
    if cap:
        dof = np.cumsum(sorted(u0.size * p.s for p, u0 in reqs))
        assert counters["max_running"] <= max(1, int(np.sum(dof <= cap)))
    for (p, u0), r in zip(reqs, results):
        assert r is not None and r["status"] == 0, r
        u_alone, (done, status, st) = _alone(S, p, u0)
        assert np.array_equal(r["u"], u_alone) and r["stats"] == st


def test_admission_policy_rejects_bad_arguments(S):
    with S.Server(2, S.EULER, 4, 64 << 20) as srv:
        for order, cap in ((2, 0.0), (-1, 0.0), (0, -1.0), (0, float("nan"))):
            with pytest.raises(S.StdgError):
                srv.set_policy(order, cap)
