"""Parity at the full sizes of the benchmark workloads, in the launch shapes
the benchmark times (the autotuner's choice), and at the library's size
limits.

Workloads: plane Couette flow on 64 cells with 32^2 velocities (FP64,
converged to 1e-8), the 64^2 lid-driven cavity with 32^2 velocities, the
128^2 tanh-stretched cavity with 28^2 Gauss-Hermite velocities, the 121 x 81
O-grid cylinder at Ma 5 with 89^2 Simpson velocities and the limiter, and
the batch of 64 seeded cavities; limits: a hyperplane of 256 cells
(min(ni, nj) = 256) and 16384 velocities.

FP64: the whole state against the oracle's after a few iterations, 1e-12
relative to the field's largest entry (the oracle runs these in seconds on
the host cores).  Mixed: u and T within rel. L2 1e-5 of the FP64 oracle on
the converged 64^2 cavity (the headline claim); on the other workloads,
after a few iterations, f~ and W within 1e-5 of the FP64 oracle relative to
each field's largest entry (max norm: cells in the evacuated wake of the
impulsively started cylinder have a u and T that float32 storage does not
resolve, and contribute nothing at that scale).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_01819_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_01819_gb300 import build
    build.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _tuned(prob, precision):
    """A solver in the launch shape the benchmark would time (autotuned)."""
    from paper_1709_01819_gb300.solver import Autotuner, Solver
    s = Solver(prob, precision)
    s.init_uniform()
    Autotuner().tune(s)
    s.init_uniform()
    return s


def _fp64_parity(s, o, tag):
    G, H, W = s.get_state()
    Go, Ho, Wo = o.get_state()
    assert _rel(G, Go) < 1e-12, (tag, _rel(G, Go))
    assert _rel(H, Ho) < 1e-12, (tag, _rel(H, Ho))
    for q in range(4):
        assert _rel(W[:, q], Wo[:, q]) < 1e-12, (tag, q, _rel(W[:, q], Wo[:, q]))


def _mixed_close(s, o, tag):
    G, H, W = s.get_state()
    Go, Ho, Wo = o.get_state()
    assert _rel(G, Go) < 1e-5, (tag, _rel(G, Go))
    assert _rel(H, Ho) < 1e-5, (tag, _rel(H, Ho))
    for q in range(4):
        assert _rel(W[:, q], Wo[:, q]) < 1e-5, (tag, q, _rel(W[:, q], Wo[:, q]))


def test_couette_64_v32_fp64_converged_to_1e8_matches_oracle():
    prob = I.couette_c1()
    o = O.Oracle(prob)
    o.init_uniform()
    s = _tuned(prob, "fp64")
    ok, n, r = s.iterate(5000, 1e-8)
    assert ok and r <= 1e-8
    ro = o.iterate(n)
    assert ro[-1] <= 1e-8 * ro[0]
    # converged fields: 1e-10 on each quantity's natural scale (the
    # y-momentum of Couette flow is ~1e-7: relative to itself it carries the
    # rounding of hundreds of iterations)
    G, H, W = s.get_state()
    Go, Ho, Wo = o.get_state()
    assert _rel(G, Go) < 1e-10 and _rel(H, Ho) < 1e-10
    scale = [1.0, 0.1, 0.1, 1.0]  # density, velocity components (U = 0.1), energy / temperature
    m, mo = s.moments(), o.moments()
    for q in range(4):
        assert np.abs(W[:, q] - Wo[:, q]).max() <= 1e-10 * scale[q], q
        assert np.abs(m[:, q] - mo[:, q]).max() <= 1e-10 * scale[q], q


@pytest.mark.parametrize("workload", ["cavity_64_v32", "cavity_128_tanh_gh28", "cylinder_121x81_v89"])
def test_full_size_fp64_and_mixed_per_iteration(workload):
    prob = {"cavity_64_v32": I.cavity_c2, "cavity_128_tanh_gh28": I.cavity_c3,
            "cylinder_121x81_v89": I.cylinder_c5}[workload]()
    n = 2 if workload.startswith("cylinder") else 3
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(n)
    for prec in ("fp64", "mixed"):
        s = _tuned(prob, prec)
        s.iterate(n)
        (_fp64_parity if prec == "fp64" else _mixed_close)(s, o, (workload, prec, s.tuning()))
        del s


def test_cavity_64_v32_mixed_converged_within_1e5_of_fp64_oracle():
    prob = I.cavity_c2()
    s = _tuned(prob, "mixed")
    ok, n, r = s.iterate(20000, 1e-6)
    assert ok
    o = O.Oracle(prob)
    o.init_uniform()
    ro = o.iterate(n)
    assert ro[-1] <= 1.5e-6 * ro[0]
    m, mo = s.moments(), o.moments()
    speed = np.hypot(mo[:, 1], mo[:, 2])
    du = np.sqrt(np.sum((m[:, 1] - mo[:, 1]) ** 2 + (m[:, 2] - mo[:, 2]) ** 2) / np.sum(speed ** 2))
    dT = np.linalg.norm(m[:, 3] - mo[:, 3]) / np.linalg.norm(mo[:, 3])
    print("64^2 cavity, mixed, converged in", n, "iterations: du", du, "dT", dT)
    assert du < 1e-5, du
    assert dT < 1e-5, dT


def test_batch_of_64_cavities_full_size_sampled_instances():
    """The benchmark's batch (one launch per kernel over 64 instances,
    autotuned): sampled instances equal their single-instance runs bitwise,
    and are within the mixed-precision bar of the FP64 oracle."""
    from paper_1709_01819_gb300.solver import BatchSolver, Solver
    probs = I.batch_c4()
    bs = BatchSolver(probs, "mixed", autotune=True)
    ok, n, r, conv = bs.iterate(3)
    assert n == 3
    sizes = [p.ni for p in probs]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17})
    for b in picks:
        sb = bs.solvers[b]
        s = Solver(probs[b], "mixed")
        s.set_tuning(**sb.tuning())
        s.init_uniform()
        s.iterate(3)
        for x, y in zip(s.get_state(), sb.get_state()):
            assert np.array_equal(x, y), b
        o = O.Oracle(probs[b])
        o.init_uniform()
        o.iterate(3)
        _mixed_close(sb, o, ("batch instance", b, probs[b].name))


def test_largest_hyperplane_256_cells():
    """min(ni, nj) = 256, the library's limit: the micro sweeps hold 256 cells
    per hyperplane step, the macroscopic wavefront 256 cells."""
    prob = I.cavity(256, Kn=0.075, U=0.15, nv=6, vmax=4.0)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(3)
    s = _tuned(prob, "fp64")
    s.iterate(3)
    _fp64_parity(s, o, "256 x 256 cells")
    s = _tuned(prob, "mixed")
    s.iterate(3)
    _mixed_close(s, o, "256 x 256 cells, mixed")


def test_largest_velocity_grid_16384():
    """128 x 128 = 16384 velocities, the library's limit (one block of cells
    with a ragged hyperplane)."""
    prob = I.cavity(5, Kn=0.075, U=0.15, nv=128, vmax=6.0)
    prob.nodes_x, prob.nodes_y = I.uniform_nodes(5, 3, 0, 1, 0, 0.6)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(3)
    for prec in ("fp64", "mixed"):
        s = _tuned(prob, prec)
        assert s.Nv == 16384
        s.iterate(3)
        (_fp64_parity if prec == "fp64" else _mixed_close)(s, o, ("16384 velocities", prec))
