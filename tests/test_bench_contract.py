"""bench.py's reference arm (the oracle timed on the host cores) keeps the JSON contract: one
line with the GPU arm's metric, unit and direction, `impl: reference`, a cpu_baseline that
describes the run and an e2e object with no host-device traffic.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench._workload_name()
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_oracle_check_reports_the_error_it_is_given():
    """The bench's oracle check measures what it says: handed the oracle's own 1D advection march
    as the GPU result it reports 0, handed that result scaled by (1 + 1e-6) it reports 1e-6
    (relative LGL-weighted L2 of a scaled vector), and the march's nodal error against the exact
    solution sin(2 pi (x - t)) is small (fourth-order scheme, 10 slabs of dt = 0.01)."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import dgsem, stdg as ost
    from paper_2201_05800_gb300 import inputs
    g = dgsem.Grid(1, (16,), (0.0,), (1.0,), 3, "advection", {"adv_vel": (1.0,)})
    F = lambda x: dgsem.spatial_operator(g, x)
    u = inputs.sine(g.coordinates()[0])
    for _ in range(10):
        U, _ = ost.solve_slab_direct("stdg", F, u, 0.01, 3)
        u = U[2]
    res = bench._oracle_job({"kind": "advection1d", "nslabs": 10, "gpu": {"same": u.copy(), "scaled": u * (1 + 1e-6)}})
    assert res["rel_l2_vs_oracle"]["same"] == 0.0
    assert abs(res["rel_l2_vs_oracle"]["scaled"] - 1e-6) <= 1e-12
    assert res["oracle_rel_l2_nodal_vs_exact"] < 1e-4
    assert res["dof_st"] == 16 * 4 * 3
