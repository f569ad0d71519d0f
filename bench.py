#!/usr/bin/env python
"""Benchmark: JFNK slab solves of the 2D Euler isentropic vortex on one GB300.

Workload (the paper's 2D Euler vortex, Sec. 7.3, on the periodic box [0,10]^2):
64 x 64 quadrilaterals, N = 4 (5 x 5 LGL nodes), N_tau = s = 4, Rusanov flux,
CFL 0.5 (dt = 0.5 h / max(|v| + c) over the initial LGL nodes, held fixed),
Newton rtol 1e-10 with GMRES(30), FP64 plain path.  Synthetic analytic data.

One step = one slab solve (stdg_advance_slab): the whole hot path (residual,
Jacobian-vector products, Gram-Schmidt, Newton updates) over one slab of
1,638,400 space-time DOF; steps march consecutive slabs.

Reported value: space-time GDOF of residual evaluations per second over the
timed slab solves (every FP64 residual and every Jacobian-vector product -- a
residual evaluation at U + eps v -- counts DOF_st), i.e. the effective residual
throughput of the whole solver; slab solves/s and the kernel-level numbers are
extra keys.  --impl reference runs the FP64 CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "space-time GDOF residual evals/s + slab solves/s, p50/p99 latency vs plain GPU"
UNIT = "GDOF/s"
# gmres_rtol is the constant inexact-Newton forcing term eta (the paper gives none): 0.05 was the
# fastest of {1e-5, 1e-4, 1e-3, 1e-2, 2e-2, 5e-2, 1e-1} for this workload on GB300 (21.8 ms vs 33.6 ms
# per FP64 slab at 1e-3; 7 Newton steps of ~11 GMRES iterations instead of 4 of ~27).  The stopping
# test, and so the accuracy, is the Newton one (rtol 1e-10) either way.  Each slab starts from the
# previous slab's temporal polynomial extrapolated to the new nodes (predictor 1); the Newton target
# stays relative to the residual of the constant guess 1 (x) u^n, as with predictor 0.
WORKLOAD = dict(dim=2, cells=(64, 64), lo=(0.0, 0.0), hi=(10.0, 10.0), N=4, s=4, gamma=1.4, cfl=0.5,
                newton_rtol=1e-10, gmres_m=30, gmres_rtol=0.05, predictor=1)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # SMs x FP64 FMA/clk/SM x flop/FMA x max SM clock


def _workload_name():
    w = WORKLOAD
    return "2D Euler isentropic vortex, %dx%d quads on [0,10]^2, N=%d, s=%d, CFL %.1f, JFNK GMRES(%d) " \
           "forcing %g, Newton rtol %g, %s initial guess, FP64" % (
               w["cells"][0], w["cells"][1], w["N"], w["s"], w["cfl"], w["gmres_m"], w["gmres_rtol"],
               w["newton_rtol"], "extrapolated" if w["predictor"] else "constant")


def _vortex_state(coords):
    from paper_2201_05800_gb300 import inputs
    return inputs.isentropic_vortex(coords[:, 0], coords[:, 1], gamma=WORKLOAD["gamma"], center=(5.0, 5.0))


def _cfl_dt(u, h):
    """dt = CFL h / max over nodes and directions of |v_a| + c (initial state)."""
    import numpy as np
    g = WORKLOAD["gamma"]
    rho, m1, m2, E = u[:, 0], u[:, 1], u[:, 2], u[:, 3]
    p = (g - 1.0) * (E - 0.5 * (m1 * m1 + m2 * m2) / rho)
    c = np.sqrt(g * p / rho)
    lam = max(np.max(np.abs(m1 / rho) + c), np.max(np.abs(m2 / rho) + c))
    return WORKLOAD["cfl"] * h / lam


def algorithmic_flops_per_node(eq, d, n, s, mode):
    """Minimal FP64 flops per space-time node of one operator launch (FMA = 2, div = sqrt = 1);
    face terms counted once per face (d/n face points per node).  Euler (r = d + 2): flux and wave
    speeds 1 div + (2d+3) pressure + 1 + d(d+3); volume d r 2(n+1); temporal coupling 2 r s + r/s;
    per face point 12 r + (2d+8) + 9 (+ 2r for the perturbed neighbour of the FD Jv); combination
    2r + r/s (residual) or 4r plus 2r for U + eps v (FD Jv)."""
    r = d + 2 if eq == "euler" else 1
    if eq == "euler":
        flux = 1 + (2 * d + 3) + 1 + d * (d + 3)
        face = 12 * r + (2 * d + 8) + 9
    else:
        flux = d
        face = 12 * r + 3
    vol = d * r * 2 * (n + 1)
    time_c = r * 2 * s + r / s
    if mode == "residual":
        comb = 2 * r + r / s
        state = 0
    else:
        comb = 4 * r
        state = 2 * r
        face += 2 * r
    return state + flux + vol + time_c + comb + (d / n) * face


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _build_then_load(ws, rank, build_fn, load_fn):
    """Rank 0 alone compiles the in-tree library (all ranks share one build folder and one .so, so
    concurrent builds would race on the object files and the link); every rank loads it after a
    barrier."""
    if rank == 0:
        build_fn()
    _barrier(ws)
    return load_fn()


# ----------------------------------------------------------------------------- oracle legs

ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import dgsem, stdg
from paper_2201_05800_gb300 import inputs
w = json.loads(%(w)r)
g = dgsem.Grid(2, w["cells"], w["lo"], w["hi"], w["N"], "euler", {"gamma": w["gamma"]})
X = g.coordinates()
u0 = inputs.isentropic_vortex(X[0], X[1], gamma=w["gamma"], center=(5.0, 5.0))
U = np.stack([inputs.perturbed(u0, 100 + m, 1e-3) for m in range(w["s"])])
v = inputs.random_array(U.shape, 7)
F = lambda x: dgsem.spatial_operator(g, x)
dt = w["dt"]
dof = U.size
times = []
for step in range(%(steps)d):
    t0 = time.perf_counter()
    stdg.stdg_residual(F, U, u0, dt)
    stdg.jv_exact("stdg", F, U, u0, dt, v)
    times.append(time.perf_counter() - t0)
print(json.dumps({"times": times, "dof": dof, "evals_per_step": 2}))
"""


def run_oracle(steps, dt):
    """Time the FP64 oracle (as it stands) on one host core: per step one residual and one exact
    (complex-step) Jv evaluation of the full slab.  Returns (per-step seconds, dof, evals/step)."""
    w = dict(WORKLOAD)
    w["dt"] = dt
    code = ORACLE_SNIPPET % {"root": ROOT, "w": json.dumps(w), "steps": steps}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle run failed: " + out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    return res["times"], res["dof"], res["evals_per_step"]


# ----------------------------------------------------------------------------- oracle checks
#
# The oracle (plain FP64 NumPy, one thread per process) is run after every GPU timing has ended,
# in worker processes started with "spawn".  It supplies the CPU baseline (timings) and, from the
# same runs, the error of each benchmarked GPU result against the oracle's own slab solution.

def _cpu_info():
    """Host CPU model and core counts (for the CPU baseline)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "nproc": os.cpu_count(), "usable": usable}


def _oracle_env():
    """One BLAS/OpenMP thread per oracle process (the processes themselves use the cores)."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _rel_lgl(grid, a, b):
    from oracle import stdg as ost
    return float(ost.lgl_weighted_norm(grid, a - b) / ost.lgl_weighted_norm(grid, b))


def _oracle_job(job):
    """One oracle task in a worker process; returns a small dict (errors, times, iterations)."""
    import numpy as np
    from oracle import dgsem, physics, stdg as ost
    from paper_2201_05800_gb300 import inputs
    kind = job["kind"]
    t_start = time.perf_counter()
    if kind == "eval_loop":
        # per repetition: one FP64 residual and one exact (complex-step) Jv of the full vortex slab
        w = job["w"]
        g = dgsem.Grid(2, w["cells"], w["lo"], w["hi"], w["N"], "euler", {"gamma": w["gamma"]})
        X = g.coordinates()
        u0 = inputs.isentropic_vortex(X[0], X[1], gamma=w["gamma"], center=(5.0, 5.0))
        U = np.stack([inputs.perturbed(u0, 100 + m, 1e-3) for m in range(w["s"])])
        v = inputs.random_array(U.shape, 7)
        F = lambda x: dgsem.spatial_operator(g, x)
        times = []
        for _ in range(job["reps"]):
            t0 = time.perf_counter()
            ost.stdg_residual(F, U, u0, job["dt"])
            ost.jv_exact("stdg", F, U, u0, job["dt"], v)
            times.append(time.perf_counter() - t0)
        return {"times": times, "dof": int(U.size), "evals_per_rep": 2}
    if kind == "vortex_march":
        # the headline workload's first slabs, each solved by the oracle from the oracle's previous slab
        w = job["w"]
        g = dgsem.Grid(2, w["cells"], w["lo"], w["hi"], w["N"], "euler", {"gamma": w["gamma"]})
        X = g.coordinates()
        u = inputs.isentropic_vortex(X[0], X[1], gamma=w["gamma"], center=(5.0, 5.0))
        F = lambda x: dgsem.spatial_operator(g, x)
        slabs = []
        for k, ug in enumerate(job["gpu"]):
            t0 = time.perf_counter()
            st = {}
            U = ost.solve_slab_newton_gmres("stdg", F, u, job["dt"], w["s"], rtol=w["newton_rtol"],
                                            maxit=30, gmres_m=w["gmres_m"], gmres_tol=w["gmres_rtol"],
                                            gmres_maxit=600, stats=st, scaling="temporal_mass")
            u = U[w["s"] - 1]
            slabs.append({"slab": k + 1, "oracle_s": time.perf_counter() - t0, "newton_its": st["newton_its"],
                          "gmres_its": st["gmres_its"],
                          "rel_l2_vs_oracle": _rel_lgl(g, ug.reshape(g.state_shape), u)})
        return {"slabs": slabs}
    if kind in ("burgers", "vortex_request", "wave3d", "advection1d"):
        if kind == "burgers":
            sp = inputs.burgers_instance(job["i"])
            g = dgsem.Grid(2, (sp["side"],) * 2, (0.0, 0.0), (1.0, 1.0), sp["N"], "burgers",
                           {"viscosity": sp["nu"]})
            X = g.coordinates()
            u = inputs.burgers_fourier(X[0], X[1], sp["seed"])
            s, dt = sp["s"], 0.5 * (1.0 / sp["side"]) / float(np.max(np.abs(u)))
            exact = None
        elif kind == "vortex_request":
            side, N, s = job["side"], job["N"], job["s"]
            g = dgsem.Grid(2, (side, side), (0.0, 0.0), (10.0, 10.0), N, "euler", {"gamma": 1.4})
            X = g.coordinates()
            u = inputs.isentropic_vortex(X[0], X[1], gamma=1.4, center=(5.0, 5.0))
            lam = max(float(np.max(physics.wave_speed("euler", u, a, g.params))) for a in range(2))
            dt = 0.5 * (10.0 / side) / lam
            exact = None
        elif kind == "wave3d":
            K, N, s = job["K"], job["N"], job["s"]
            g = dgsem.Grid(3, (K, K, K), (0.0,) * 3, (1.0,) * 3, N, "euler", {"gamma": 1.4})
            X = g.coordinates()
            u = inputs.density_wave(*X, gamma=1.4)
            lam = max(float(np.max(physics.wave_speed("euler", u, a, g.params))) for a in range(3))
            dt = 0.5 * (1.0 / K) / lam
            exact = lambda t: inputs.density_wave(*X, t=t, gamma=1.4)
        else:
            K, N, s, dt = 16, 3, 3, 0.01
            g = dgsem.Grid(1, (K,), (0.0,), (1.0,), N, "advection", {"adv_vel": (1.0,)})
            X = g.coordinates()
            u = inputs.sine(X[0])
            exact = lambda t: inputs.sine(X[0], t=t)
        F = lambda x: dgsem.spatial_operator(g, x)
        nslabs = job.get("nslabs", 1)
        its = [0, 0]
        for _ in range(nslabs):
            if kind == "advection1d":
                U, _ = ost.solve_slab_direct("stdg", F, u, dt, s)
            else:
                st = {}
                U = ost.solve_slab_newton_gmres("stdg", F, u, dt, s, rtol=job["rtol"], maxit=30, gmres_m=30,
                                                gmres_tol=job["eta"], gmres_maxit=2000, stats=st,
                                                scaling="temporal_mass")
                its[0] += st["newton_its"]
                its[1] += st["gmres_its"]
            u = U[s - 1]
        out = {"oracle_s": time.perf_counter() - t_start, "dof_st": int(U.size), "oracle_newton_its": its[0],
               "oracle_gmres_its": its[1], "rel_l2_vs_oracle": {}}
        for name, ug in job["gpu"].items():
            out["rel_l2_vs_oracle"][name] = _rel_lgl(g, ug.reshape(g.state_shape), u)
        if exact is not None:
            ue = exact(dt * nslabs)
            out["oracle_rel_l2_nodal_vs_exact"] = float(np.linalg.norm(u - ue) / np.linalg.norm(ue))
        return out
    raise ValueError(kind)


def _oracle_pool_map(jobs, workers):
    """Run oracle jobs in `workers` spawned processes; results in job order."""
    import concurrent.futures
    import multiprocessing
    _oracle_env()
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=max(1, workers), mp_context=ctx) as ex:
        return list(ex.map(_oracle_job, jobs))


def _default_dt():
    """dt of the workload, computed with the same CFL rule on the host (no GPU needed)."""
    import numpy as np
    from oracle import dgsem
    g = dgsem.Grid(2, WORKLOAD["cells"], WORKLOAD["lo"], WORKLOAD["hi"], WORKLOAD["N"], "euler",
                   {"gamma": WORKLOAD["gamma"]})
    X = g.coordinates()
    from paper_2201_05800_gb300 import inputs
    u0 = inputs.isentropic_vortex(X[0], X[1], gamma=WORKLOAD["gamma"], center=(5.0, 5.0)).reshape(-1, 4)
    return _cfl_dt(u0, min(g.h))


def reference_arm(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    dt = _default_dt()
    times, dof, evals = run_oracle(args.warmup + args.steps, dt)
    timed = times[args.warmup:]
    T = sum(timed)
    value = evals * dof * len(timed) / T / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload_name(), "dof_st": dof, "dt": dt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: 1 FP64 residual + 1 complex-step Jv of the full "
                                       "64x64 N=4 s=4 slab (NumPy oracle, weak form)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm

def gpu_arm(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2201_05800_gb300 import build, stdg
    _build_then_load(ws, rank, build.build, stdg.load)
    stream = torch.cuda.Stream()
    w = WORKLOAD
    desc = stdg.make_config(dim=2, cells=[w["cells"][0], w["cells"][1], 1], lo=[w["lo"][0], w["lo"][1], 0.0],
                            hi=[w["hi"][0], w["hi"][1], 1.0], N=w["N"], s=w["s"], equation=stdg.EULER,
                            gamma=w["gamma"], dt=1.0, newton_rtol=w["newton_rtol"], gmres_m=w["gmres_m"],
                            gmres_rtol=w["gmres_rtol"], newton_maxit=30, gmres_maxit=600,
                            predictor=w["predictor"])
    with torch.cuda.stream(stream):
        probe = stdg.Context(desc, stream.cuda_stream)
        coords = probe.node_coordinates()
        probe.close()
        u0 = np.ascontiguousarray(_vortex_state(coords)).ravel()
        h = (w["hi"][0] - w["lo"][0]) / w["cells"][0]
        dt = _cfl_dt(u0.reshape(-1, 4), h)
        desc.dt = dt
        ctx = stdg.Context(desc, stream.cuda_stream)
        dof = ctx.slab_len
        ctx.set_state(u0)
        for _ in range(args.warmup):
            ctx.advance_slab()
        # ---- timed region: K consecutive slab solves (the library counts its launches; its
        #      per-kernel event timing stays off here and runs on the K slabs that follow)
        ctx.profile_read(reset=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        lat = []
        with ClockSampler(local) as clk:
            _barrier(ws)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                t0 = time.perf_counter()
                stats.append(ctx.advance_slab())
                lat.append(time.perf_counter() - t0)
            ev1.record(stream)
            torch.cuda.synchronize()
            _barrier(ws)
        launches = sum(p["launches"] for p in ctx.profile_read(reset=True).values())
        u_fp64 = ctx.get_state()  # state after warm-up + timed slabs (FP64 path)
        # ---- attribution: the next K slabs with in-library kernel timing (not part of the timing)
        ctx.profile_enable(True)
        prof_stats = [ctx.advance_slab() for _ in range(args.steps)]
        prof = ctx.profile_read(reset=True)
        ctx.profile_enable(False)
        ms_total = ev0.elapsed_time(ev1)
        ms_total = _max_over_ranks(ms_total, ws)
        evals = sum(st["residual_evals"] + st["jv_evals"] for st in stats)
        evals_all = _sum_over_ranks(float(evals * dof), ws)
        value = evals_all / (ms_total * 1e-3) / 1e9
        solves_per_s = _sum_over_ranks(float(args.steps), ws) / (ms_total * 1e-3)

        # ---- dominant kernel roofline (class with the largest in-solve device time)
        cls = max(prof, key=lambda k: prof[k]["ms"])
        n, s = w["N"] + 1, w["s"]
        nodes = w["cells"][0] * w["cells"][1] * s * n ** 2
        # average over the Jacobian-vector products actually computed (launches enqueued after a
        # device-driven GMRES cycle ended return at once and are not counted as products)
        jv_count = sum(st["jv_evals"] for st in prof_stats)
        jv_launch_ms = prof["jv"]["ms"] / max(jv_count, 1)
        jv_flops = algorithmic_flops_per_node("euler", 2, n, s, "jv") * nodes
        achieved = jv_flops / (jv_launch_ms * 1e-3) / 1e12
        traffic = _ncu_traffic()
        roofline = {"bound": "alu", "kernel": "st_operator_kernel<2,EULER,f64,JvFD,5,4> (FD Jacobian-vector)",
                    "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz "
                                   "(FMA microbenchmark 1.203 TFLOP/s at 1995 MHz)",
                    "algorithmic_flops_per_launch": jv_flops, "avg_launch_ms": jv_launch_ms,
                    "dominant_class": cls}
        # ---- residual kernel alone (isolated, L2 flushed between launches)
        dU = torch.from_numpy(np.tile(u0.reshape(-1, 1, n * n * 4), (1, s, 1)).ravel()).cuda()
        du = torch.from_numpy(u0).cuda()
        dR = torch.empty_like(dU)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        rt = []
        for i in range(8):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.residual(dU, du, dR)
            e1.record(stream)
            torch.cuda.synchronize()
            rt.append(e0.elapsed_time(e1))
        r_ms = statistics.median(rt[2:])
        r_flops = algorithmic_flops_per_node("euler", 2, n, s, "residual") * nodes
        residual_kernel = {"ms": r_ms, "gdof_per_s": dof / (r_ms * 1e-3) / 1e9,
                           "tflops_algorithmic": r_flops / (r_ms * 1e-3) / 1e12,
                           "frac_fp64_peak": r_flops / (r_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                           "hbm_gbs_algorithmic": (2 * dof + dof / s) * 8 / (r_ms * 1e-3) / 1e9}
        clocks = clk.summary()

        # ---- end to end through the public API with host (pinned) buffers
        hin = torch.from_numpy(ctx.get_state()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        hin_np, hout_np = hin.numpy(), hout.numpy()
        _barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_evals = 0
        for _ in range(args.steps):
            ctx.set_state(hin_np)
            st = ctx.advance_slab()
            ctx.get_state(hout_np)
            e2e_evals += st["residual_evals"] + st["jv_evals"]
            hin_np[:] = hout_np
        torch.cuda.synchronize()
        e2e_s = _max_over_ranks(time.perf_counter() - t0, ws)
        e2e_value = _sum_over_ranks(float(e2e_evals * dof), ws) / e2e_s / 1e9
        ctx.close()
        # the first slabs of the same configuration from u0, for the oracle check (not timed)
        with stdg.Context(desc, stream.cuda_stream) as cc:
            cc.set_state(u0)
            check_states = []
            for _ in range(ORACLE_CHECK_SLABS):
                cc.advance_slab()
                check_states.append(cc.get_state())

        # ---- the same slabs on the mixed-precision path (FP32 exact Jv and Krylov basis,
        #      FP64 Newton residual and update): throughput and distance to the FP64 path
        mixed = _mixed_path(stdg, desc, u0, args, stream, u_fp64, ws) if "mixed" in args.legs else None
        batched = _batched_leg(stdg, stream, args.batch_instances, args.batch_sequential, args.batch_graphs) \
            if "batched" in args.legs and ws == 1 else None
        served = _serving_leg(stdg, [int(r) for r in args.serve_rates.split(",")], args.serve_requests) \
            if "serving" in args.legs and ws == 1 else None
        wave3d = _density_wave_leg(stdg, stream) if "wave3d" in args.legs and ws == 1 else None
        adv1d = _advection_leg(stdg, stream) if "adv1d" in args.legs and ws == 1 else None

    lat_ms = sorted(1e3 * x for x in lat)
    cpu, oracle_check = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the CPU-baseline leg: the oracle timed on the host cores, and the error of every
        # benchmarked GPU result against the oracle's solution from the same oracle runs
        try:
            cpu, oracle_check = _cpu_baseline_leg(dt, check_states, batched, served, wave3d, adv1d)
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: %r" % e}
    for leg in (batched, served, wave3d, adv1d):
        if leg is not None:
            leg.pop("_check", None)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": _workload_name(), "dof_st": dof, "dt": dt, "parallelism":
                           "replicas" if ws > 1 else "single GPU",
                           "l2": "working set per step > L2 (Krylov basis 31 x 13.1 MB FP64); the isolated "
                                 "residual timing flushes L2 (256 MB write) before each launch"},
                "slab_solves_per_s": solves_per_s,
                "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1,
                                                                                   int(0.99 * len(lat_ms)))]},
                "solver": {"newton_its": [st["newton_its"] for st in stats],
                           "gmres_its": [st["gmres_its"] for st in stats],
                           "residual_evals": sum(st["residual_evals"] for st in stats),
                           "jv_evals": sum(st["jv_evals"] for st in stats)},
                "kernel_time_ms": {k: v["ms"] for k, v in prof.items()},
                "kernel_launches": {k: v["launches"] for k, v in prof.items()},
                "kernel_accounting": "kernel_time_ms / kernel_launches: the %d slabs after the timed "
                                     "ones, with per-launch CUDA events; gpu_launches: counted in the "
                                     "timed region" % args.steps,
                "residual_kernel": residual_kernel,
                "roofline": roofline, "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(hin.numel() * 8),
                        "d2h_bytes_per_step": int(hout.numel() * 8)},
                "gpu_launches": launches, "cpu_baseline": cpu, "oracle_check": oracle_check,
                "mixed_fp32": mixed, "batched": batched, "served": served, "density_wave_3d": wave3d,
                "advection_1d": adv1d}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


ORACLE_CHECK_SLABS = 2      # headline slabs re-solved by the oracle
ORACLE_SAMPLE = 16          # batched instances and served requests re-solved by the oracle
ORACLE_MAX_DOF = 20000      # ... among those with at most this many space-time DOF (oracle time)
SERVE_ORACLE_MAX_DOF = 120000
CPU_REPS_1 = 60             # single-thread oracle sample: 60 x (residual + Jv) of the vortex slab
CPU_REPS_ALL = 8            # all-core sample: every core runs 8 x (residual + Jv) concurrently


def _cpu_baseline_leg(dt, check_states, batched, served, wave3d, adv1d):
    """Oracle timings (one thread; all host cores as concurrent processes) and the oracle checks."""
    import numpy as np
    info = _cpu_info()
    cores = max(1, info["usable"] or 1)
    w = dict(WORKLOAD)
    # (1) one thread
    t0 = time.perf_counter()
    one = _oracle_pool_map([{"kind": "eval_loop", "w": w, "dt": dt, "reps": 1 + CPU_REPS_1}], 1)[0]
    t1 = time.perf_counter()
    T1 = sum(one["times"][1:])
    v1 = one["evals_per_rep"] * one["dof"] * CPU_REPS_1 / T1 / 1e9
    # (2) every usable core: one process per core, each its own copy of the sample
    allr = _oracle_pool_map([{"kind": "eval_loop", "w": w, "dt": dt, "reps": 1 + CPU_REPS_ALL}] * cores, cores)
    v_all = sum(r["evals_per_rep"] * r["dof"] * CPU_REPS_ALL / sum(r["times"][1:]) for r in allr) / 1e9
    # (3) oracle slab solves and the error of each benchmarked GPU result against them
    jobs = [{"kind": "vortex_march", "w": w, "dt": dt, "gpu": check_states}]
    names = ["headline"]
    for leg, tag in ((batched, "batched"), (served, "served"), (wave3d, "density_wave_3d"),
                     (adv1d, "advection_1d")):
        for j in (leg or {}).get("_check", []):
            jobs.append(j)
            names.append(tag)
    t2 = time.perf_counter()
    res = _oracle_pool_map(jobs, min(cores, len(jobs)))
    t3 = time.perf_counter()
    check = {"tolerance_note": "relative LGL-weighted L2 distance of the GPU result to the oracle's FP64 slab "
                               "solution of the same problem at the same Newton tolerance (each side stops at "
                               "its own ||R|| <= rtol ||R(U0)||, so agreement is to the solve tolerance)",
             "oracle_wall_s": t3 - t2}
    head = res[0]["slabs"]
    check["headline"] = {"slabs": head, "max_rel_l2_vs_oracle": max(x["rel_l2_vs_oracle"] for x in head)}
    for tag in ("batched", "served", "density_wave_3d", "advection_1d"):
        rs = [(j, r) for j, r, nm in zip(jobs, res, names) if nm == tag]
        if not rs:
            continue
        errs = {}
        for j, r in rs:
            for k, e in r["rel_l2_vs_oracle"].items():
                errs[k] = max(errs.get(k, 0.0), e)
        entry = {"cases": [dict({kk: vv for kk, vv in j.items() if kk not in ("gpu", "kind")}, **r) for j, r in rs],
                 "max_rel_l2_vs_oracle": errs}
        check[tag] = entry
    slab_times = [x["oracle_s"] for x in head]
    cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d x (1 FP64 residual + 1 complex-step Jv) of the full 64x64 N=4 s=4 vortex slab (NumPy "
                     "oracle, weak form, one thread) after one warm-up; %.1f s" % (CPU_REPS_1, T1),
           "cpu": info,
           "all_cores": {"value": v_all, "unit": UNIT, "cores": cores,
                         "sample": "%d processes (one per usable core), each %d x (residual + Jv) of its own copy "
                                   "of the slab after one warm-up; summed throughput" % (cores, CPU_REPS_ALL)},
           "oracle_slab_solve_s": {"per_slab": slab_times, "slabs_per_s": len(slab_times) / sum(slab_times),
                                   "what": "the oracle's Newton-GMRES solve (left temporal-mass scaling, exact "
                                           "complex-step Jv, one thread) of the first %d slabs of the headline "
                                           "workload, run while other cores solved the other checks"
                                           % len(slab_times)},
           "single_thread_wall_s": t1 - t0}
    return cpu, check


def _mixed_path(stdg, desc, u0, args, stream, u_ref, ws):
    """March the same warm-up + timed slabs with STDG_MIXED_FP32 (exact FP32 Jv); time the
    timed ones with CUDA events and compare the final state with the FP64 path's."""
    import ctypes

    import numpy as np
    import torch
    dm = stdg.stdg_config_desc()
    ctypes.memmove(ctypes.byref(dm), ctypes.byref(desc), ctypes.sizeof(desc))
    dm.precision = stdg.MIXED_FP32
    dm.jv_mode = stdg.JV_EXACT
    ctx = stdg.Context(dm, stream.cuda_stream)
    dof = ctx.slab_len
    ctx.set_state(u0)
    for _ in range(args.warmup):
        ctx.advance_slab()
    ctx.profile_read(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = [ctx.advance_slab() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = _max_over_ranks(e0.elapsed_time(e1), ws)
    u = ctx.get_state()
    ctx.profile_read(reset=True)
    ctx.profile_enable(True)
    for _ in range(args.steps):
        ctx.advance_slab()
    prof = ctx.profile_read(reset=True)
    ctx.close()
    evals = sum(st["residual_evals"] + st["jv_evals"] for st in stats)
    return {"precision": "FP32 Jv (exact, forward mode) + FP32 Krylov basis, FP64 Newton residual/update",
            "value": _sum_over_ranks(float(evals * dof), ws) / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": ms / args.steps,
            "slab_solves_per_s": _sum_over_ranks(float(args.steps), ws) / (ms * 1e-3),
            "rel_l2_vs_fp64_path": float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)),
            "newton_its": [st["newton_its"] for st in stats], "gmres_its": [st["gmres_its"] for st in stats],
            "kernel_time_ms": {k: v["ms"] for k, v in prof.items()},
            "kernel_launches": {k: v["launches"] for k, v in prof.items()}}


# ----------------------------------------------------------------------------- batched / served legs

WORK_TOL = dict(newton_rtol=1e-10, newton_atol=0.0, newton_maxit=30, gmres_m=30, gmres_rtol=1e-3)


class _Coords:
    """Node coordinates per (equation, box, side, N), taken from the library (a small context)."""

    def __init__(self, stdg):
        self.stdg, self.cache = stdg, {}

    def __call__(self, eq, box, side, N):
        key = (eq, box, side, N)
        if key not in self.cache:
            S = self.stdg
            d = S.make_config(dim=2, cells=[side, side, 1], lo=[0, 0, 0], hi=[box, box, 1], N=N, s=2, equation=eq,
                              dt=1.0, gmres_m=1)
            with S.Context(d) as c:
                self.cache[key] = c.node_coordinates()
        return self.cache[key]


def _burgers_instances(stdg, n):
    """The batched viscous Burgers workload: instance i from seed 1000 + i (grid side in
    {8,16,32,64}, N in 2..6, s in 2..5, viscosity log-uniform in [1e-3, 1e-1]), 8 Fourier modes
    of amplitude 0.5 on the periodic unit square, dt = 0.5 h / max|u0| (CFL 0.5)."""
    import numpy as np
    from paper_2201_05800_gb300 import inputs
    xy = _Coords(stdg)
    out = []
    for i in range(n):
        sp = inputs.burgers_instance(i)
        X = xy(stdg.BURGERS, 1.0, sp["side"], sp["N"])
        u0 = np.ascontiguousarray(inputs.burgers_fourier(X[:, 0], X[:, 1], sp["seed"]).ravel())
        dt = 0.5 * (1.0 / sp["side"]) / float(np.max(np.abs(u0)))
        d = stdg.make_config(dim=2, cells=[sp["side"], sp["side"], 1], lo=[0, 0, 0], hi=[1, 1, 1], N=sp["N"],
                             s=sp["s"], equation=stdg.BURGERS, dt=dt, viscosity=sp["nu"], **WORK_TOL)
        out.append((d, u0, u0.size * sp["s"]))
    return out


def _vortex_requests(stdg, n, seed=7):
    """Served requests: single-slab solves of the 2D Euler vortex on [0,10]^2, grid side uniform
    in {16,32,64,128}, N uniform in 2..7, s uniform in 2..5, CFL 0.5 (seeded)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    xy = _Coords(stdg)
    out = []
    for _ in range(n):
        side = int(rng.choice([16, 32, 64, 128]))
        N = int(rng.integers(2, 8))
        s = int(rng.integers(2, 6))
        X = xy(stdg.EULER, 10.0, side, N)
        u0 = np.ascontiguousarray(_vortex_state(X).ravel())
        dt = _cfl_dt(u0.reshape(-1, 4), 10.0 / side)
        d = stdg.make_config(dim=2, cells=[side, side, 1], lo=[0, 0, 0], hi=[10, 10, 1], N=N, s=s,
                             equation=stdg.EULER, gamma=WORKLOAD["gamma"], dt=dt, **WORK_TOL)
        out.append((d, u0, u0.size * s))
    return out


def _sequential_config(stdg, d):
    """The plain one-solve-at-a-time GPU path at the same accuracy: a context with FP32 exact
    Jacobian-vector products, FP64 Newton and restarted GMRES, preconditioned by the point blocks
    for the scalar (viscous) equations and by the temporal-mass scaling for Euler (the point
    block stalls on high-degree Euler slabs with s = 2)."""
    import ctypes
    dm = stdg.stdg_config_desc()
    ctypes.memmove(ctypes.byref(dm), ctypes.byref(d), ctypes.sizeof(d))
    pc = stdg.PRECOND_TEMPORAL_MASS if d.equation == stdg.EULER else stdg.PRECOND_POINT_BLOCK
    dm.precision, dm.jv_mode, dm.precond, dm.gmres_maxit = stdg.MIXED_FP32, stdg.JV_EXACT, pc, 600
    return dm


def _run_batch(stdg, B, items):
    """Admit items in arrival order while the arena has room, tick, retire: returns per-item
    (status, stats, state)."""
    pending = list(range(len(items)))
    slots, res = {}, {}
    while pending or slots:
        while pending:
            sl = B.try_add(items[pending[0]][0], items[pending[0]][1])
            if sl is None:
                break
            slots[sl] = pending.pop(0)
        if not slots:
            raise RuntimeError("an item does not fit the arena")
        B.step(8)
        for sl in B.done_slots():
            _, st, stats = B.query(sl)
            res[slots.pop(sl)] = (st, stats, B.get_state(sl))
            B.remove(sl)
    return [res[i] for i in range(len(items))]


def _batched_leg(stdg, stream, n_inst, n_seq, graphs=1):
    import numpy as np
    import torch
    items = _burgers_instances(stdg, n_inst)
    free, _ = torch.cuda.mem_get_info()
    arena = int(free * 0.7)
    # the same instances with the heuristic tile sizes (autotuning off), for comparison
    with stdg.Batch(2, stdg.BURGERS, n_inst, arena, stream.cuda_stream) as B:
        B.configure(use_graphs=bool(graphs), autotune=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out_h = _run_batch(stdg, B, items)
        torch.cuda.synchronize()
        T_heur = time.perf_counter() - t0
    # the leg itself: tile sizes measured per (dim, N, s) class on a loaded virtual grid (the
    # measurement, on first use of a class, is inside the timed region)
    with stdg.Batch(2, stdg.BURGERS, n_inst, arena, stream.cuda_stream) as B:
        B.configure(use_graphs=bool(graphs), autotune=True)  # graphs 0: plain launches (per-kernel profiling)
        need = sum(B.slot_bytes(d) for d, _, _ in items)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = _run_batch(stdg, B, items)
        torch.cuda.synchronize()
        T = time.perf_counter() - t0
        # the same instances again: the tile table is kept for the process, so this run measures no tiles
        t0 = time.perf_counter()
        out_w = _run_batch(stdg, B, items)
        torch.cuda.synchronize()
        T_warm = time.perf_counter() - t0
        # the same first n_seq instances alone in the batch engine, for the like-for-like comparison
        t1 = time.perf_counter()
        out_small = _run_batch(stdg, B, items[:n_seq])
        torch.cuda.synchronize()
        T_small = time.perf_counter() - t1
    statuses = [st for st, _, _ in out]
    evals_ok = sum((st["residual_evals"] + st["jv_evals"]) * dof
                   for (code, st, _), (_, _, dof) in zip(out, items) if code == 0)
    # sequential plain path on the first n_seq instances: solve time per instance (the context is
    # created and the state copied in outside the timing)
    seq, seq_t = [], []
    for d, u0, _ in items[:n_seq]:
        with stdg.Context(_sequential_config(stdg, d), stream.cuda_stream) as c:
            c.set_state(u0)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            st = c.advance_slab(check=False)
            torch.cuda.synchronize()
            seq_t.append(time.perf_counter() - t2)
            seq.append((st["status"], c.get_state()))
    T_seq = sum(seq_t)
    # the instances the sequential path solves, alone in a batch (warm: tile classes measured)
    conv = [i for i in range(min(n_seq, len(seq))) if seq[i][0] == 0]
    T_conv = None
    if conv:
        with stdg.Batch(2, stdg.BURGERS, max(1, len(conv)), arena, stream.cuda_stream) as B:
            B.configure(use_graphs=bool(graphs), autotune=True)
            _run_batch(stdg, B, [items[i] for i in conv])
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            _run_batch(stdg, B, [items[i] for i in conv])
            torch.cuda.synchronize()
            T_conv = time.perf_counter() - t3
    diffs = [float(np.linalg.norm(a[2] - b[1]) / np.linalg.norm(b[1])) for a, b in zip(out[:n_seq], seq)
             if a[0] == 0 and b[0] == 0]
    its = [st["gmres_its"] for _, st, _ in out]
    # a seeded sample of instances small enough for the oracle, with their GPU results
    import numpy as np
    small = [i for i, it in enumerate(items) if it[2] <= ORACLE_MAX_DOF]
    pick = sorted(np.random.default_rng(2201).choice(small, size=min(ORACLE_SAMPLE, len(small)), replace=False))
    check = [{"kind": "burgers", "i": int(i), "rtol": WORK_TOL["newton_rtol"], "eta": WORK_TOL["gmres_rtol"],
              "gpu_status": int(out[i][0]), "gpu": {"batched": out[i][2]}} for i in pick]
    vs_seq = None
    if n_seq > 0:
        T_seq_conv = sum(seq_t[i] for i in conv)
        vs_seq = {"instances": n_seq, "sequential_converged": len(conv), "sequential_failed": n_seq - len(conv),
                  "speedup": T_seq_conv / T_conv if T_conv else None,
                  "speedup_counting": "the instances the sequential path solves (status 0): their summed "
                                      "sequential solve times over the batch's wall time for the same set",
                  "converged_set": {"batched_s": T_conv, "sequential_s": T_seq_conv,
                                    "batched_instances_per_s": len(conv) / T_conv if T_conv else None,
                                    "sequential_instances_per_s": len(conv) / T_seq_conv if T_seq_conv else None},
                  "all_instances": {"batched_s": T_small, "sequential_s": T_seq,
                                    "batched_converged": [x[0] for x in out_small].count(0)},
                  "max_rel_diff_to_sequential": max(diffs) if diffs else None,
                  "pairs_compared": len(diffs),
                  "sequential_path": "stdg_advance_slab per instance (FP32 exact Jv, point-block "
                                     "preconditioner, restarted GMRES(30); solve time only)"}
    return {"workload": "%d independent 2D viscous Burgers instances (seed 1000+i; side in {8,16,32,64}, N 2-6, "
                        "s 2-5, nu log-uniform [1e-3,1e-1]), one slab each, FP32 Krylov + FP64 Newton "
                        "refinement, Newton rtol 1e-10, FGMRES(30) rtol 1e-3" % n_inst,
            "instances": n_inst, "dof_total": int(sum(x[2] for x in items)), "arena_gb": arena / 1e9,
            "slot_memory_gb": need / 1e9, "seconds": T, "instances_per_s": statuses.count(0) / T,
            "gdof_evals_per_s": evals_ok / T / 1e9, "failed": n_inst - statuses.count(0),
            "counting": "instances_per_s and gdof_evals_per_s count the instances that converged (status 0)",
            "status_counts": {str(k): statuses.count(k) for k in sorted(set(statuses))},
            "gmres_its_mean": float(np.mean(its)), "gmres_its_max": int(max(its)),
            "graphs": bool(graphs), "autotune": True,
            "autotune_note": "seconds includes measuring the tile sizes of every (N, s) class on first use; "
                             "tiles_cached is a second run of the same instances with the measured table",
            "tiles_cached": {"seconds": T_warm, "instances_per_s": [x[0] for x in out_w].count(0) / T_warm,
                             "failed": n_inst - [x[0] for x in out_w].count(0)},
            "heuristic_tiles": {"seconds": T_heur, "instances_per_s": [x[0] for x in out_h].count(0) / T_heur,
                                "failed": n_inst - [x[0] for x in out_h].count(0)},
            "vs_sequential": vs_seq, "_check": check}


SERVE_DOF_CAP = 16e6  # smallest-first run: space-time DOF the admitted requests may hold at once
SERVE_FIFO_CAP = 32e6  # capped arrival-order runs: the same limit for admission in arrival order


def _serving_leg(stdg, rates, n_req):
    """Served stream: n_req single-slab vortex requests per arrival rate, submitted on their Poisson
    clock to a server; latency from submission to result.  The sequential baseline runs every
    request alone through stdg_advance_slab (its service time measured on the GPU); its latencies
    under the same arrivals are modelled from those service times with one FIFO queue."""
    import numpy as np
    import torch
    reqs = _vortex_requests(stdg, n_req)
    free, _ = torch.cuda.mem_get_info()
    arena = int(free * 0.5)
    rng = np.random.default_rng(7)
    out = {"workload": "single-slab 2D Euler vortex solves on [0,10]^2, side in {16,32,64,128}, N 2-7, s 2-5, "
                       "CFL 0.5, Newton rtol 1e-10, FGMRES(30) rtol 1e-3; Poisson arrivals (seed 7)",
           "requests_per_rate": n_req, "arena_gb": arena / 1e9, "rates": {}}
    # service times of the plain sequential GPU path (solve only, contexts created outside the timing)
    svc, seq_status, seq_u = [], [], []
    stream = torch.cuda.Stream()
    for d, u0, _ in reqs:
        with stdg.Context(_sequential_config(stdg, d), stream.cuda_stream) as c:
            c.set_state(u0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = c.advance_slab(check=False)
            svc.append(time.perf_counter() - t0)
            seq_status.append(st["status"])
            seq_u.append(c.get_state())
    # every rate with arrival-order admission; one rate with smallest-first admission under a cap on
    # the admitted space-time DOF, and two with arrival-order admission under a cap
    # (stdg_server_set_policy)
    pol_rate = rates[min(2, len(rates) - 1)]
    runs = [(str(r), r, 0, 0.0) for r in rates] + [("%d_smallest_first" % pol_rate, pol_rate, 1, SERVE_DOF_CAP)]
    runs += [("%d_arrival_order_capped" % r, r, 0, SERVE_FIFO_CAP) for r in rates if r in (pol_rate, 1000)]
    first_res = None
    pct = lambda v, q: 1e3 * v[min(len(v) - 1, int(q * len(v)))] if v else None
    for key, rate, order, cap in runs:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
        with stdg.Server(2, stdg.EULER, max(64, n_req), arena) as srv:
            srv.set_policy(order, cap)
            t0 = time.perf_counter()
            tickets = []
            for (d, u0, _), ta in zip(reqs, arrivals):
                while time.perf_counter() - t0 < ta:
                    pass
                tickets.append(srv.submit(d, u0))
            res = [srv.poll(t, wait_s=600.0) for t in tickets]
            T = time.perf_counter() - t0
            cnt = srv.counters()
        if first_res is None:
            first_res = res
        ok = [r for r in res if r["status"] == 0]
        lat = sorted(r["latency_s"] for r in ok)
        # the sequential path under the same arrivals (one FIFO queue, measured service times)
        fin, seq_lat = 0.0, []
        for ta, sv, stt in zip(arrivals, svc, seq_status):
            fin = max(fin, ta) + sv
            if stt == 0:
                seq_lat.append(fin - ta)
        seq_lat.sort()
        out["rates"][key] = {
            "served": {"p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "solves_per_s": len(ok) / T,
                       "failed": n_req - len(ok), "max_running": cnt["max_running"],
                       "arrivals_span_s": float(arrivals[-1]),
                       "statuses": {str(k): [r["status"] for r in res].count(k)
                                    for k in sorted({r["status"] for r in res})}},
            "sequential_modelled": {"p50_ms": pct(seq_lat, 0.5), "p99_ms": pct(seq_lat, 0.99),
                                    "solves_per_s": len(seq_lat) / fin}}
    out["scheduling"] = {"graphs": True, "autotune": False,
                         "admission": "arrival order by device memory, except the '<rate>_smallest_first' run: "
                                      "the queued request with the fewest space-time DOF first, while the admitted "
                                      "ones hold at most %g DOF; and the '<rate>_arrival_order_capped' runs: arrival "
                                      "order while the admitted ones hold at most %g DOF" % (SERVE_DOF_CAP,
                                                                                            SERVE_FIFO_CAP)}
    out["sequential_path"] = ("stdg_advance_slab per request (FP32 exact Jv, temporal-mass scaling, restarted "
                              "GMRES); service times measured on the GPU, latencies modelled from them under the "
                              "same arrivals with one FIFO queue")
    out["sequential_statuses"] = {str(k): seq_status.count(k) for k in sorted(set(seq_status))}
    out["counting"] = "solves_per_s and the latency percentiles count the requests that converged (status 0)"
    # a seeded sample of requests small enough for the oracle, with the served and sequential results
    small = [k for k, rq in enumerate(reqs) if rq[2] <= SERVE_ORACLE_MAX_DOF]
    pick = sorted(np.random.default_rng(2202).choice(small, size=min(ORACLE_SAMPLE, len(small)), replace=False))
    out["_check"] = [{"kind": "vortex_request", "side": int(reqs[k][0].cells[0]), "N": int(reqs[k][0].N),
                      "s": int(reqs[k][0].s), "rtol": WORK_TOL["newton_rtol"], "eta": WORK_TOL["gmres_rtol"],
                      "gpu_status": [int(first_res[k]["status"]), int(seq_status[k])],
                      "gpu": {"served": first_res[k]["u"], "sequential": seq_u[k]}} for k in pick]
    return out


def _density_wave_leg(stdg, stream, slabs=2):
    """3D Euler density wave (rho = 1 + 0.2 sin(2 pi (x+y+z)), v = (1,1,1), p = 1) on the periodic
    unit cube, 32^3 hexes, N = 3, s = 3 (31.5 M space-time DOF), CFL 0.5: one warm-up slab and
    `slabs` timed slabs on the FP64 path (FD Jv) and on the mixed path (FP32 exact Jv and Krylov
    basis, FP64 Newton refinement); differences between the paths and to the exact solution."""
    import ctypes
    import numpy as np
    import torch
    from paper_2201_05800_gb300 import inputs
    K, N, s = 32, 3, 3
    base = dict(dim=3, cells=[K, K, K], lo=[0, 0, 0], hi=[1, 1, 1], N=N, s=s, equation=stdg.EULER, gamma=1.4,
                dt=1.0, newton_rtol=1e-10, gmres_m=30, gmres_rtol=WORKLOAD["gmres_rtol"], newton_maxit=30,
                gmres_maxit=600, predictor=WORKLOAD["predictor"])
    d = stdg.make_config(**base)
    with stdg.Context(d, stream.cuda_stream) as c:
        X = c.node_coordinates()
    u0 = np.ascontiguousarray(inputs.density_wave(X[:, 0], X[:, 1], X[:, 2]).ravel())
    ur = u0.reshape(-1, 5)
    rho = ur[:, 0]
    p = 0.4 * (ur[:, 4] - 0.5 * (ur[:, 1] ** 2 + ur[:, 2] ** 2 + ur[:, 3] ** 2) / rho)
    lam = float(np.max(np.abs(ur[:, 1] / rho) + np.sqrt(1.4 * p / rho)))
    dt = 0.5 * (1.0 / K) / lam
    out = {"workload": "3D Euler density wave on the periodic unit cube, 32^3 hexes, N=3, s=3, CFL 0.5 "
                       "(dt = %.6g), Newton rtol 1e-10, GMRES(30) forcing %g, %s initial guess" % (
                           dt, WORKLOAD["gmres_rtol"], "extrapolated" if WORKLOAD["predictor"] else "constant")}
    finals = {}
    for name, prec, jv in (("fp64", stdg.FP64, stdg.JV_FD), ("mixed_fp32", stdg.MIXED_FP32, stdg.JV_EXACT),
                           ("mixed_bf16", stdg.MIXED_BF16, stdg.JV_EXACT)):
        dd = stdg.make_config(**dict(base, dt=dt, precision=prec, jv_mode=jv))
        with stdg.Context(dd, stream.cuda_stream) as c:
            dof = c.slab_len
            c.set_state(u0)
            c.advance_slab()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            st = [c.advance_slab() for _ in range(slabs)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            finals[name] = c.get_state()
            if name != "fp64":
                out["roofline_" + name + "_jv"] = _jv32_roofline(stdg, c, dof, inputs, name)
            evals = sum(x["residual_evals"] + x["jv_evals"] for x in st)
            out[name] = {"ms_per_slab": ms / slabs, "gdof_evals_per_s": evals * dof / (ms * 1e-3) / 1e9,
                         "newton_its": [x["newton_its"] for x in st], "gmres_its": [x["gmres_its"] for x in st],
                         "device_gb": c.device_bytes / 1e9}
    t = (slabs + 1) * dt
    exact = inputs.density_wave(X[:, 0], X[:, 1], X[:, 2], t=t).ravel()
    for name in finals:
        out[name]["rel_l2_nodal_vs_exact"] = float(np.linalg.norm(finals[name] - exact) / np.linalg.norm(exact))
    out["dof_st"] = int(dof)
    out["rel_l2_mixed_vs_fp64"] = float(np.linalg.norm(finals["mixed_fp32"] - finals["fp64"]) /
                                        np.linalg.norm(finals["fp64"]))
    out["speedup_mixed"] = out["fp64"]["ms_per_slab"] / out["mixed_fp32"]["ms_per_slab"]
    out["rel_l2_mixed_bf16_vs_fp64"] = float(np.linalg.norm(finals["mixed_bf16"] - finals["fp64"]) /
                                             np.linalg.norm(finals["fp64"]))
    out["mixed_bf16"]["what"] = ("as mixed_fp32, with the volume contractions of the exact Jacobian-vector "
                                 "product on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation)")
    # the same configuration on a reduced grid (K^3, same N, s, CFL, tolerances, guess), both
    # precisions, for the oracle check: the 32^3 grid is beyond the oracle's time budget
    Kr = WAVE3D_CHECK_K
    gpu = {}
    for name, prec, jv in (("fp64", stdg.FP64, stdg.JV_FD), ("mixed_fp32", stdg.MIXED_FP32, stdg.JV_EXACT),
                           ("mixed_bf16", stdg.MIXED_BF16, stdg.JV_EXACT)):
        dd = stdg.make_config(**dict(base, cells=[Kr, Kr, Kr], dt=1.0, precision=prec, jv_mode=jv))
        with stdg.Context(dd, stream.cuda_stream) as c:
            Xr = c.node_coordinates()
        ur = np.ascontiguousarray(inputs.density_wave(Xr[:, 0], Xr[:, 1], Xr[:, 2]).ravel())
        q = ur.reshape(-1, 5)
        pr = 0.4 * (q[:, 4] - 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2 + q[:, 3] ** 2) / q[:, 0])
        dtr = 0.5 * (1.0 / Kr) / float(np.max(np.abs(q[:, 1] / q[:, 0]) + np.sqrt(1.4 * pr / q[:, 0])))
        with stdg.Context(stdg.make_config(**dict(base, cells=[Kr, Kr, Kr], dt=dtr, precision=prec, jv_mode=jv)),
                          stream.cuda_stream) as c:
            c.set_state(ur)
            for _ in range(WAVE3D_CHECK_SLABS):
                c.advance_slab()
            gpu[name] = c.get_state()
    out["_check"] = [{"kind": "wave3d", "K": Kr, "N": N, "s": s, "nslabs": WAVE3D_CHECK_SLABS,
                      "rtol": base["newton_rtol"], "eta": base["gmres_rtol"], "gpu": gpu}]
    return out


def _hbm_peak():
    """(GB/s, source): the measured copy bandwidth in MEASURED_PEAKS.json, else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def _jv32_roofline(stdg, c, dof, inputs, name, reps=12):
    """The FP32 exact Jacobian-vector kernel of the 3D leg alone (stdg_jv_fp32 on the final slab and
    a random direction, L2 flushed by a 256 MB write before each launch, the library's per-launch
    CUDA events): algorithmic bytes 12 per DOF (read U and v, write J v) / median launch time."""
    import torch
    U32 = torch.from_numpy(c.get_slab()).cuda().float()
    v32 = torch.from_numpy(inputs.random_array(dof, 5)).cuda().float()
    out = torch.empty_like(U32)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    c.profile_read(reset=True)
    c.profile_enable(True)
    ms = []
    for i in range(reps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        c.jv_fp32(U32, v32, out)
        pr = c.profile_read(reset=True)
        ms.append(pr["jv"]["ms"] / max(1, pr["jv"]["launches"]))
    c.profile_enable(False)
    t = sorted(ms[2:])[len(ms[2:]) // 2]
    peak, src = _hbm_peak()
    gbs = 12.0 * dof / (t * 1e-3) / 1e9
    prof = "jv_tangent32_euler3d_dw32.txt" if name == "mixed_fp32" else "jv_tangent_bf16_euler3d_dw32.txt"
    return {"bound": "hbm", "kernel": "jv_tangent_kernel<3,4,3,%s> (%s exact J v)" % (
                "1,false" if name == "mixed_fp32" else "2,true", "FP32" if name == "mixed_fp32" else "BF16 tensor-core"),
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_source": src,
            "avg_launch_ms": t, "algorithmic_bytes_per_launch": 12.0 * dof,
            "traffic": _ncu_value(prof, "dram_bytes_per_launch")}


WAVE3D_CHECK_K = 4
WAVE3D_CHECK_SLABS = 2


def _advection_leg(stdg, stream, slabs=100, reps=5):
    """1D linear advection u_t + u_x = 0 on the periodic unit interval: 16 elements, N = 3, s = 3,
    dt = 0.01, 100 slabs from u0 = sin(2 pi x) (192 space-time DOF per slab).  Launch-latency bound:
    reported as microseconds per slab (CUDA events around each 100-slab march; best and median of
    `reps` marches) and compared with the oracle's march."""
    import numpy as np
    import torch
    from paper_2201_05800_gb300 import inputs
    d = stdg.make_config(dim=1, cells=[16, 1, 1], lo=[0, 0, 0], hi=[1, 1, 1], N=3, s=3, equation=stdg.ADVECTION,
                         adv_vel=[1.0, 0.0, 0.0], dt=0.01, newton_rtol=1e-10, gmres_m=30, gmres_rtol=1e-3)
    with stdg.Context(d, stream.cuda_stream) as c:
        X = c.node_coordinates()
        u0 = np.ascontiguousarray(inputs.sine(X[:, 0]).ravel())
        ms = []
        for _ in range(reps + 1):
            c.set_state(u0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            st = [c.advance_slab() for _ in range(slabs)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        u = c.get_state()
        launches = sum(p["launches"] for p in c.profile_read(reset=True).values())
    ms = ms[1:]
    exact = inputs.sine(X[:, 0], t=slabs * 0.01).ravel()
    return {"workload": "1D linear advection, 16 elements on [0,1], N=3, s=3, dt=0.01, u0=sin(2 pi x), "
                        "%d slabs, Newton rtol 1e-10, GMRES(30) rtol 1e-3, FP64" % slabs,
            "dof_st": 192, "us_per_slab_best": 1e3 * min(ms) / slabs,
            "us_per_slab_median": 1e3 * sorted(ms)[len(ms) // 2] / slabs,
            "newton_its_last": st[-1]["newton_its"], "gmres_its_last": st[-1]["gmres_its"],
            "launches_per_slab": launches / ((reps + 1) * slabs),
            "rel_l2_nodal_vs_exact": float(np.linalg.norm(u - exact) / np.linalg.norm(exact)),
            "_check": [{"kind": "advection1d", "nslabs": slabs, "gpu": {"fp64": u}}]}


def _ncu_value(fname, key):
    """A 'key: value' figure from a committed ncu summary under profiles/, or None."""
    p = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith(key + ":"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


def _ncu_traffic():
    """DRAM bytes per launch of the FD Jv kernel from the committed ncu summary, or None."""
    return _ncu_value("jv_fd_euler2d_vortex64.txt", "dram_bytes_per_launch")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="mixed,batched,serving,wave3d,adv1d",
                    help="extra legs after the main FP64 line: mixed,batched,serving,wave3d,adv1d (or none)")
    ap.add_argument("--batch-instances", type=int, default=4096)
    ap.add_argument("--batch-sequential", type=int, default=48,
                    help="instances solved one at a time for the batched-vs-sequential comparison")
    ap.add_argument("--batch-graphs", type=int, choices=[0, 1], default=1,
                    help="0: the batched leg launches its kernels per tick instead of replaying a CUDA graph")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rates", default="5,10,100,1000,5000")
    ap.add_argument("--kernel", choices=["jv32", "jv_bf16"], default=None,
                    help="only the 3D density-wave Jacobian-vector kernel (FP32 or BF16 tensor cores) on a "
                         "K^3 grid with a one-row Krylov basis (a small device footprint for ncu captures)")
    ap.add_argument("--kernel-grid", type=int, default=32)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.kernel:
        return kernel_only(args)
    return gpu_arm(args)


def kernel_only(args):
    """The 3D density-wave Jacobian-vector kernel alone: --warmup + --steps launches, L2 flushed before
    each, CUDA-event time per launch from the library's profiler; one JSON line (not the bench line)."""
    import numpy as np
    import torch
    from paper_2201_05800_gb300 import build, inputs, stdg
    _build_then_load(1, 0, build.build, stdg.load)
    K = args.kernel_grid
    prec = stdg.MIXED_BF16 if args.kernel == "jv_bf16" else stdg.MIXED_FP32
    d = stdg.make_config(dim=3, cells=[K, K, K], lo=[0, 0, 0], hi=[1, 1, 1], N=3, s=3, equation=stdg.EULER,
                         gamma=1.4, dt=0.5 / K / 2.6, gmres_m=1, jv_mode=stdg.JV_EXACT, precision=prec)
    with stdg.Context(d) as c:
        X = c.node_coordinates()
        u0 = inputs.density_wave(X[:, 0], X[:, 1], X[:, 2]).ravel()
        L = c.slab_len
        U = torch.from_numpy(np.tile(u0.reshape(-1, 1, 64 * 5), (1, 3, 1)).ravel()).cuda()
        U = (U * (1.0 + 1e-3 * torch.from_numpy(inputs.random_array(L, 21)).cuda())).float()
        v = torch.from_numpy(inputs.random_array(L, 22)).cuda().float()
        out = torch.empty_like(U)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        c.profile_enable(True)
        ms = []
        for i in range(args.warmup + args.steps):
            flush.fill_(i & 255)
            torch.cuda.synchronize()
            c.profile_read(reset=True)
            c.jv_fp32(U, v, out)
            pr = c.profile_read(reset=True)
            ms.append(pr["jv"]["ms"] / max(1, pr["jv"]["launches"]))
        t = sorted(ms[args.warmup:])[len(ms[args.warmup:]) // 2]
        peak, src = _hbm_peak()
        print(json.dumps({"kernel": args.kernel, "grid": K, "dof": int(L), "launch_ms_median": t,
                          "algorithmic_bytes": 12.0 * L, "gbs": 12.0 * L / (t * 1e-3) / 1e9,
                          "frac_hbm": 12.0 * L / (t * 1e-3) / 1e9 / peak, "peak_gbs": peak, "peak_source": src}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
