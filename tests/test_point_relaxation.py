"""The point-relaxation predictor (idg_set_predictor, n Jacobi sweeps of the
predictor equations) on the GPU against the oracle's, through the C ABI.

FP64: 1e-12 relative per iteration on f~ and W, as for the LU-SGS predictor.
Mixed: u and T of the steady cavity within rel. L2 1e-5 of the FP64 oracle's.
"""
import dataclasses

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


def _solver(prob, precision="fp64"):
    from paper_1709_01819_gb300.solver import Solver
    return Solver(prob, precision)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cases():
    c = {}
    p = I.cavity(12, Kn=0.075, U=0.15, nv=15, vmax=4.0)
    X, Y = I.uniform_nodes(12, 9, 0, 1, 0, 0.8)
    p.nodes_x, p.nodes_y, p.nvy = X, Y, 13
    c["cavity_shakhov_12x9_v15x13"] = p
    # periodic direction one cell wide: every cell wrapped onto itself in x
    c["couette_16_v16"] = I.couette(16, U=0.1, Kn=0.1, nv=16, vmax=4.0)
    # periodic seam, far field, limiter
    c["cylinder_20x8_simpson11_limiter"] = I.cylinder(ntheta=20, nr=8, nv=11, vmax=8.0, Ma=2.0, Kn=0.5)
    return c


CASES = _cases()


@pytest.mark.parametrize("sweeps", [1, 2, 5])
@pytest.mark.parametrize("name", sorted(CASES))
def test_point_relaxation_fp64_matches_oracle_per_iteration(name, sweeps):
    prob = dataclasses.replace(CASES[name], relax_sweeps=sweeps)
    o = O.Oracle(prob)
    o.init_uniform()
    s = _solver(prob)
    s.init_uniform()
    for n in (1, 2, 5):
        ro = o.iterate(n)
        s.iterate(n)
        G, H, W = s.get_state()
        Go, Ho, Wo = o.get_state()
        assert _rel(G, Go) < 1e-12, (name, sweeps, n, _rel(G, Go))
        assert _rel(H, Ho) < 1e-12, (name, sweeps, n, _rel(H, Ho))
        for q in range(4):
            assert _rel(W[:, q], Wo[:, q]) < 1e-12 or np.abs(W[:, q] - Wo[:, q]).max() < 1e-14, (name, q)
    rg = s.residual_history()
    assert abs(rg[-1] - ro[-1]) <= 1e-10 * ro[-1]


def test_point_relaxation_mixed_converged_cavity_within_1e5_of_fp64_oracle():
    prob = dataclasses.replace(I.cavity(16, Kn=0.075, U=0.15, nv=16, vmax=4.0, cfl_imp=1000.0), relax_sweeps=5)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(300)
    mo = o.moments()
    s = _solver(prob, "mixed")
    s.init_uniform()
    s.iterate(300)
    m = s.moments()
    speed = np.hypot(mo[:, 1], mo[:, 2])
    du = np.sqrt(np.sum((m[:, 1] - mo[:, 1]) ** 2 + (m[:, 2] - mo[:, 2]) ** 2) / np.sum(speed ** 2))
    dT = np.linalg.norm(m[:, 3] - mo[:, 3]) / np.linalg.norm(mo[:, 3])
    print("point relaxation, mixed: du", du, "dT", dT)
    assert du < 1e-5, du
    assert dT < 1e-5, dT


def test_point_relaxation_graph_replay_is_bitwise_equal_to_plain_launches():
    prob = dataclasses.replace(CASES["cylinder_20x8_simpson11_limiter"], relax_sweeps=3)
    a = _solver(prob, "mixed")
    b = _solver(prob, "mixed")
    b.set_tuning(graph=0)
    for s in (a, b):
        s.init_uniform()
        s.iterate(35)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.residual_history(), b.residual_history())


def test_point_relaxation_rejections():
    from paper_1709_01819_gb300 import binding as B

    prob = CASES["couette_16_v16"]
    lu = _solver(prob)
    pr = _solver(dataclasses.replace(prob, relax_sweeps=3))
    for s in (lu, pr):
        s.init_uniform()
    with pytest.raises(B.IdgError):  # one predictor per batch
        B.idg_batch_create([lu.ctx, pr.ctx])
    with pytest.raises(B.IdgError):  # the adjoint transposes LU-SGS only
        pr.adjoint(B.IDG_OBJ_FORCE_X, 1 << I.JMAX, [], 1, 0.0)
    ctx = B.idg_create(B.IDG_FP64, 0)
    try:
        with pytest.raises(B.IdgError):
            B.idg_set_predictor(ctx, -1)
        with pytest.raises(B.IdgError):
            B.idg_set_predictor(ctx, 65)
    finally:
        B.idg_destroy(ctx)
