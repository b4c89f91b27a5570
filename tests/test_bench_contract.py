"""The benchmark's contract pieces that need no GPU: the compulsory bytes
behind the roofline, derived here from the pairs each launch group must move,
and the reference arm's JSON line (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_algorithmic_bytes_of_the_64x64_cavity():
    import bench
    from oracle import oracle as O
    prob = bench.workload("cavity64")
    nf = O.Oracle(prob).nf
    N, V = prob.ncells, prob.nvel
    assert (N, V, nf) == (4096, 1024, 2 * 64 * 65)
    pair = 2 * 4  # one {G, H} pair of float32
    expect = {
        # f~ read by the moments and by fb+, fb+ written
        "cell_prep": 3 * N * V * pair,
        # fb+ read once (neighbour reuse from cache), fb written per face
        "face_moments": N * V * pair + nf * V * pair,
        # fb read, flux written, per face
        "face_flux": 2 * nf * V * pair,
        # residual: fluxes (each face once), f~, R written; forward sweep: R read, Delta* written
        "k_sweep_fwd": nf * V * pair + 4 * N * V * pair,
        # backward sweep: Delta* and f~ read, f~ written
        "k_sweep_bwd": 3 * N * V * pair,
    }
    assert bench.algorithmic_bytes(prob, 4, nf) == expect
    lim = bench.algorithmic_bytes(bench.workload("cylinder61x41"), 4, 1)
    cyl = bench.workload("cylinder61x41")
    # with the limiter the gradients are written (2 pairs) and read back, fb+ read again
    assert lim["face_moments"] == 12 * 4 * cyl.ncells * cyl.nvel + 2 * 4 * 1 * cyl.nvel


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


def test_reference_arm_of_the_batch_is_unavailable():
    d = _run("--impl", "reference", "--workload", "batch64", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and "unavailable" in d
