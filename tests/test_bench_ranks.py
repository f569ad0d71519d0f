"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

On N GPUs the benchmark runs N independent replicas of the workload (the slab solve has no
exchange step on one GPU): each rank times its own steps, the reported time is the maximum over
ranks and the throughput the sum of all ranks' work divided by that time.  These helpers are
exercised here with two gloo ranks; no GPU is involved."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo")
    w, r, loc = bench._dist()
    bench._barrier(w)
    t = bench._max_over_ranks(10.0 + r, w)       # rank times 10 and 11 -> 11
    s = bench._sum_over_ranks(100.0 * (r + 1), w)  # work 100 and 200 -> 300
    out[r] = (w, r, loc, t, s)
    dist.destroy_process_group()


def test_max_time_and_summed_work_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = 29500 + os.getpid() % 1000
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    for r in range(2):
        assert res[r][3] == 11.0 and res[r][4] == 300.0


def _build_rank(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import time

    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo")
    log = []

    def fake_build():
        log.append(("build_start", time.time()))
        time.sleep(1.0)  # a slow compile: the other rank must wait for it
        log.append(("build_end", time.time()))

    def fake_load():
        log.append(("load", time.time()))
        return "lib"

    assert bench._build_then_load(ws, rank, fake_build, fake_load) == "lib"
    out[rank] = log
    dist.destroy_process_group()


def test_rank_zero_builds_and_every_rank_loads_after_it():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = 29500 + (os.getpid() + 500) % 1000
        procs = [ctx.Process(target=_build_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert [k for k, _ in res[0]] == ["build_start", "build_end", "load"]
    assert [k for k, _ in res[1]] == ["load"]  # rank 1 never builds
    assert res[1][0][1] >= res[0][1][1]       # and loads only after rank 0's build ended


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench._max_over_ranks(3.5, 1) == 3.5 and bench._sum_over_ranks(2.0, 1) == 2.0
