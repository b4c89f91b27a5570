"""The linearised diffuse wall of the micro sweeps (Section 2.3, Eq. 33-35;
idg_set_implicit_wall) on the GPU against the oracle's, through the C ABI.

FP64: 1e-12 relative per iteration on f~ and W (as for the default zero
ghost increments), across a restart by set_state.  Mixed: u and T of the
steady cavity within rel. L2 1e-5 of the FP64 oracle's.
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


def _solver(prob, precision="fp64", explicit=False):
    from paper_1709_01819_gb300.solver import Solver
    return Solver(prob, precision, explicit=explicit)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cases():
    c = {}
    # moving lid, corner cells with two wall faces, ragged velocity count
    p = I.cavity(12, Kn=0.075, U=0.15, nv=15, vmax=4.0)
    X, Y = I.uniform_nodes(12, 9, 0, 1, 0, 0.8)
    p.nodes_x, p.nodes_y, p.nvy = X, Y, 13
    c["cavity_shakhov_12x9_v15x13"] = p
    # walls moving in opposite directions, periodic direction one cell wide
    c["couette_16_v16"] = I.couette(16, U=0.1, Kn=0.1, nv=16, vmax=4.0)
    # curved wall next to a periodic seam, far field, limiter
    c["cylinder_20x8_simpson11_limiter"] = I.cylinder(ntheta=20, nr=8, nv=11, vmax=8.0, Ma=2.0, Kn=0.5)
    # triangles: wall faces of oblique and axis-aligned cells, level-scheduled sweeps
    q = I.cavity(9, Kn=0.075, U=0.15, nv=15, vmax=4.0)
    X, Y = I.uniform_nodes(9, 7, 0, 1, 0, 0.8)
    q.nodes_x, q.nodes_y, q.nvy = X, Y, 13
    c["tri_cavity_9x7_v15"] = I.as_unstructured(q, tri=lambda i, j: True)
    return {k: dataclasses.replace(v, implicit_wall=1) for k, v in c.items()}


CASES = _cases()


def _compare(s, o, tag):
    G, H, W = s.get_state()
    Go, Ho, Wo = o.get_state()
    assert _rel(G, Go) < 1e-12, (tag, _rel(G, Go))
    assert _rel(H, Ho) < 1e-12, (tag, _rel(H, Ho))
    for q in range(4):
        assert _rel(W[:, q], Wo[:, q]) < 1e-12 or np.abs(W[:, q] - Wo[:, q]).max() < 1e-14, (tag, q)


@pytest.mark.parametrize("name", sorted(CASES))
def test_implicit_wall_fp64_matches_oracle_per_iteration(name):
    prob = CASES[name]
    o = O.Oracle(prob)
    o.init_uniform()
    s = _solver(prob)
    s.init_uniform()
    for n in (1, 2, 5):
        ro = o.iterate(n)
        s.iterate(n)
        _compare(s, o, (name, n))
    rg = s.residual_history()
    assert abs(rg[-1] - ro[-1]) <= 1e-10 * ro[-1]
    # the term is live: without it the oracle's state after 8 iterations differs
    off = O.Oracle(dataclasses.replace(prob, implicit_wall=0))
    off.init_uniform()
    off.iterate(8)
    assert _rel(off.get_state()[0], o.get_state()[0]) > 1e-9, name
    # a restart clears the last increment on both sides
    G, H, W = I.random_state(prob, seed=11)
    o.set_state(G, H, W)
    s.set_state(G, H, W)
    for n in (1, 2):
        o.iterate(n)
        s.iterate(n)
        _compare(s, o, (name, "restart", n))


def test_implicit_wall_mixed_converged_cavity_within_1e5_of_fp64_oracle():
    prob = dataclasses.replace(I.cavity(16, Kn=0.075, U=0.15, nv=16, vmax=4.0, cfl_imp=1000.0),
                               implicit_wall=1)
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
    print("implicit wall, mixed: du", du, "dT", dT)
    assert du < 1e-5, du
    assert dT < 1e-5, dT


def test_implicit_wall_graph_replay_is_bitwise_equal_to_plain_launches():
    prob = CASES["cylinder_20x8_simpson11_limiter"]
    a = _solver(prob, "mixed")
    b = _solver(prob, "mixed")
    b.set_tuning(graph=0)
    for s in (a, b):
        s.init_uniform()
        s.iterate(35)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.residual_history(), b.residual_history())


def test_implicit_wall_rejections():
    from paper_1709_01819_gb300 import binding as B

    prob = CASES["couette_16_v16"]
    s = _solver(prob)
    s.init_uniform()
    with pytest.raises(B.IdgError):  # batches keep zero ghost increments
        B.idg_batch_create([s.ctx])
    with pytest.raises(B.IdgError):  # the adjoint transposes the default sweeps
        s.adjoint(B.IDG_OBJ_FORCE_X, 1 << I.JMAX, [], 1, 0.0)
    with pytest.raises(B.IdgError):  # the term belongs to the implicit sweeps
        _solver(prob, explicit=True)
    with pytest.raises(B.IdgError):  # setters close at bind
        B.idg_set_implicit_wall(s.ctx, 0)
    ctx = B.idg_create(B.IDG_FP64, 0)
    try:
        with pytest.raises(B.IdgError):
            B.idg_set_implicit_wall(ctx, 2)
    finally:
        B.idg_destroy(ctx)
