"""idg_set_state from page-locked host memory (read in place by the
conversion kernel) and from pageable memory (staged through the device):
the same device state, bitwise, in both precisions, and the same iterations
after it."""
import numpy as np
import pytest

from paper_1709_01819_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_01819_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_set_state_from_pinned_and_pageable_memory_agree(precision):
    import torch
    from paper_1709_01819_gb300.solver import Solver
    prob = I.cavity(24, Kn=0.075, U=0.15, nv=12, vmax=4.0)
    src = Solver(prob, precision)
    src.init_uniform()
    src.iterate(5)
    G, H, W = src.get_state()
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (G, H, W)]
    assert all(t.is_pinned() for t in pinned)
    a, b = Solver(prob, precision), Solver(prob, precision)
    for s in (a, b):
        s.init_uniform()
    a.set_state(*[t.numpy() for t in pinned])   # in place over the host link
    b.set_state(G.copy(), H.copy(), W.copy())   # pageable: staged copies
    for x, y, z in zip(a.get_state(), b.get_state(), (G, H, W)):
        assert np.array_equal(x, y)
        if precision == "fp64":
            assert np.array_equal(x, z)
    a.iterate(3)
    b.iterate(3)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
