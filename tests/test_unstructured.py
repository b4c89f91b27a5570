"""Unstructured triangle / quadrilateral meshes on the GPU
(idg_set_mesh_unstructured) against the oracle, through the C ABI.

FP64: 1e-12 relative per iteration on f~ and W, as on structured blocks.
Mixed: steady u and T within rel. L2 1e-5 of the FP64 oracle.
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


def _solver(prob, precision="fp64", **kw):
    from paper_1709_01819_gb300.solver import Solver
    return Solver(prob, precision, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cases():
    c = {}
    # 2 x 9 x 7 triangles: ragged, a mesh corner triangle without a gradient
    p = I.cavity(9, Kn=0.075, U=0.15, nv=15, vmax=4.0)
    p.nodes_x, p.nodes_y = I.uniform_nodes(9, 7, 0, 1, 0, 0.8)
    c["tri_cavity_9x7_v15"] = I.as_unstructured(p, tri=lambda i, j: True)
    # hybrid: quads at the wall, triangles outside, ring closed by
    # connectivity; far field, Ma 2, limiter
    c["hybrid_cylinder_16x8_limiter"] = I.hybrid_cylinder(ntheta=16, nr=8, nr_quad=3, nv=11, vmax=8.0,
                                                          Ma=2.0, Kn=0.5)
    # mixed checkerboard of quads and triangle pairs
    q = I.cavity(8, Kn=0.3, U=0.2, nv=12, vmax=4.0, shakhov=0, Pr=1.0)
    c["checker_cavity_8_bgk"] = I.as_unstructured(q, tri=lambda i, j: (i + j) % 2 == 0)
    return c


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_unstructured_fp64_matches_oracle_per_iteration(name):
    prob = CASES[name]
    o = O.Oracle(prob)
    o.init_uniform()
    s = _solver(prob)
    assert (s.N, s.nf) == (o.N, o.nf)
    s.init_uniform()
    for n in (1, 2, 5):
        ro = o.iterate(n)
        s.iterate(n)
        G, H, W = s.get_state()
        Go, Ho, Wo = o.get_state()
        assert _rel(G, Go) < 1e-12, (name, n, _rel(G, Go))
        assert _rel(H, Ho) < 1e-12, (name, n, _rel(H, Ho))
        for q in range(4):
            assert _rel(W[:, q], Wo[:, q]) < 1e-12 or np.abs(W[:, q] - Wo[:, q]).max() < 1e-14, (name, q)
    assert abs(s.residual_history()[-1] - ro[-1]) <= 1e-10 * ro[-1]
    phio = o.face_phi()
    assert np.abs(s.face_flux_moments() - phio).max() < 1e-12 * np.abs(phio).max()


def test_unstructured_quads_equal_the_structured_block_on_the_gpu():
    """The structured kernels (hyperplanes, shared-memory ring) and the
    scheduled ones (levels, neighbours from global memory) on the same block."""
    p = I.cavity(10, Kn=0.075, U=0.15, nv=16, vmax=4.0)
    p.nodes_x, p.nodes_y = I.uniform_nodes(10, 7, 0, 1, 0, 0.7)
    out = []
    for q in (p, I.as_unstructured(p)):
        s = _solver(q)
        s.init_uniform()
        s.iterate(12)
        out.append(s.get_state())
    for a, b in zip(out[0], out[1]):
        assert _rel(b, a) < 1e-13


def test_unstructured_point_relaxation_and_explicit_match_oracle():
    prob = dataclasses.replace(CASES["tri_cavity_9x7_v15"], relax_sweeps=5)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(4)
    s = _solver(prob)
    s.init_uniform()
    s.iterate(4)
    for a, b in zip(s.get_state(), o.get_state()):
        assert _rel(a, b) < 1e-12
    prob = CASES["hybrid_cylinder_16x8_limiter"]
    o = O.Oracle(prob)
    o.init_uniform()
    o.explicit(6)
    s = _solver(prob, explicit=True)
    s.init_uniform()
    s.iterate(6)
    for a, b in zip(s.get_state(), o.get_state()):
        assert _rel(a, b) < 1e-12


def test_unstructured_mixed_converged_within_1e5_of_fp64_oracle():
    prob = I.tri_cavity(12, Kn=0.075, U=0.15, nv=16, vmax=4.0, cfl_imp=1000.0)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(400)
    mo = o.moments()
    s = _solver(prob, "mixed")
    s.init_uniform()
    s.iterate(400)
    m = s.moments()
    speed = np.hypot(mo[:, 1], mo[:, 2])
    du = np.sqrt(np.sum((m[:, 1] - mo[:, 1]) ** 2 + (m[:, 2] - mo[:, 2]) ** 2) / np.sum(speed ** 2))
    dT = np.linalg.norm(m[:, 3] - mo[:, 3]) / np.linalg.norm(mo[:, 3])
    print("triangles, mixed: du", du, "dT", dT)
    assert du < 1e-5 and dT < 1e-5, (du, dT)


def test_unstructured_graph_replay_and_tuning_do_not_change_results():
    prob = CASES["hybrid_cylinder_16x8_limiter"]
    out = []
    for graph, tv, vpt in ((1, 4, 1), (0, 2, 2), (1, 1, 4)):
        s = _solver(prob, "mixed")
        s.set_tuning(graph=graph, sweep_tv=tv, sweep_vpt=vpt)
        s.init_uniform()
        s.iterate(21)
        out.append(s.get_state())
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            assert np.array_equal(a, b)


def test_unstructured_rejections():
    from paper_1709_01819_gb300 import binding as B

    prob = CASES["tri_cavity_9x7_v15"]
    s = _solver(prob)
    s.init_uniform()
    with pytest.raises(B.IdgError):
        s.adjoint(B.IDG_OBJ_FORCE_X, 1 << I.JMAX, [], 1, 0.0)
    with pytest.raises(B.IdgError):
        B.idg_batch_create([s.ctx])


def test_state_round_trip_leaves_a_mixed_triangle_run_unchanged():
    """Reading and writing the state stages float64 G and H of every cell in
    the workspace; on triangles (about 1.5 faces per cell) that staging is
    larger than the face-flux buffer of float32 storage, and must not touch
    anything the iteration keeps: 5 + (get, set) + 5 iterations equal 10."""
    prob = I.tri_cavity(10, Kn=0.075, U=0.15, nv=16, vmax=4.0)
    a = _solver(prob, "mixed")
    a.init_uniform()
    a.iterate(5)
    G, H, W = a.get_state()
    a.set_state(G, H, W)
    a.iterate(5)
    b = _solver(prob, "mixed")
    b.init_uniform()
    b.iterate(5)
    b.iterate(5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
