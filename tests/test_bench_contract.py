"""The benchmark's contract pieces that need no GPU: the compulsory bytes
behind the roofline, derived here from the pairs the method must move, the
roofline arithmetic, and the reference arm's JSON line (the FP64 oracle on
the host cores), with and without its time-to-residual run."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_algorithmic_bytes_of_the_64x64_cavity():
    """The compulsory bytes of one iteration, from the pairs of f the method
    must move: f~ read before the predictor, f~ read after it and Delta*
    written, Delta* and f~ read and f~ written; float64 side data per cell."""
    import bench
    prob = bench.workload("cavity64")
    N, V = prob.ncells, prob.nvel
    assert (N, V) == (4096, 1024)
    pair = 2 * 4  # one {G, H} pair of float32
    expect = {
        "cell_prep": N * V * pair,
        "face_moments": 64 * N,
        "face_flux": 64 * N,
        "macro": 64 * N,
        "k_sweep_fwd": 2 * N * V * pair,
        "k_sweep_bwd": 3 * N * V * pair,
    }
    assert bench.algorithmic_bytes(prob, 4) == expect
    assert sum(expect.values()) - 3 * 64 * N == 6 * N * V * pair  # 12 scalars: the planned design
    assert bench.ITER_SCALARS * 4 == 40  # the lower bound, 40 B per cell-velocity


def test_roofline_picks_the_slowest_group_and_recomputes_by_hand():
    import bench
    prob = bench.workload("cavity64")
    N, V = prob.ncells, prob.nvel
    kms = [0.066, 0.100, 0.048, 0.206, 0.102, 0.078]  # the macroscopic group is the slowest
    r = bench.roofline(prob, 4, kms, 0.587, 6805.1)
    assert r["kernel"] == "macro" and r["kernel_ms"] == 0.206
    assert abs(r["achieved"] - 64 * N / 0.206e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6805.1) < 1e-12
    it = r["iteration"]
    assert it["algorithmic_bytes"] == 40 * N * V
    assert abs(it["frac"] - 40 * N * V / 0.587e-3 / 1e9 / 6805.1) < 1e-12
    assert abs(r["groups"]["k_sweep_fwd"]["frac"] - 16 * N * V / 0.102e-3 / 1e9 / 6805.1) < 1e-12
    kms[4] = 0.3
    assert bench.roofline(prob, 4, kms, 0.7, 6805.1)["kernel"] == "k_sweep_fwd"


def _run(*args):
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                       text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_prints_one_contract_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "3", "--no-ttr")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "cell-velocity updates/s"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "cavity_64x64_kn0.075_v32"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_times_the_oracle_to_the_residual():
    """The reference arm with its time-to-residual part (the oracle from the
    uniform start to 1e-6) on the 64-cell Couette flow: the line is valid
    JSON with plain booleans and numbers."""
    d = _run("--impl", "reference", "--workload", "couette64", "--steps", "1", "--warmup", "3")
    t = d["time_to_residual_1e-6"]["fp64_oracle"]
    assert t["converged"] is True and isinstance(t["iterations"], int)
    assert 0 < t["residual"] <= 1e-6 and t["seconds"] > 0
    assert d["cpu_baseline"]["cpu_model"] and d["cpu_baseline"]["nproc"] >= 1


def test_reference_arm_of_the_batch_is_unavailable():
    d = _run("--impl", "reference", "--workload", "batch64", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and "unavailable" in d
