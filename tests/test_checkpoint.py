"""Checkpoint files (idg_save / idg_load) through the C ABI: a context
restarted from a file in the precision that saved it continues bitwise as if
never stopped (the reference Maxwellian and the stored deviations travel with
the float64 view); headers that do not match are refused."""
import struct

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


def _prob():
    p = I.cylinder(ntheta=20, nr=8, nv=11, vmax=8.0, Ma=2.0, Kn=0.5)
    return p


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_restart_from_a_checkpoint_continues_the_run(prec, tmp_path):
    from paper_1709_01819_gb300.solver import Solver
    a = Solver(_prob(), prec)
    a.init_uniform()
    a.iterate(7)
    path = tmp_path / "state.ckpt"
    a.save(path)
    G0, H0, W0 = a.get_state()
    raw = path.read_bytes()
    magic, ver, precision, ncell, nvel, iters, hsh = struct.unpack("<8siiqqqq", raw[:48])
    assert magic == b"IDGCKPT1" and ver == 2 and (ncell, nvel) == (a.N, a.Nv) and iters == 7 and hsh > 0
    assert len(raw) == 48 + 8 * (4 * a.N * a.Nv + 4 * a.N + 4)
    assert np.array_equal(np.frombuffer(raw, "<f8", a.N * a.Nv, 48).reshape(a.N, a.Nv), G0)
    b = Solver(_prob(), prec)
    b.init_uniform(rho=1.2, T=0.9)  # another reference Maxwellian: the file's replaces it
    b.load(path)
    G1, H1, W1 = b.get_state()
    assert np.array_equal(W1, W0)
    a.iterate(5)
    b.iterate(5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.residual_history()[-5:], b.residual_history())


def test_mismatched_or_foreign_files_are_refused(tmp_path):
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300.solver import Solver
    a = Solver(_prob(), "fp64")
    a.init_uniform()
    path = tmp_path / "a.ckpt"
    a.save(path)
    other = Solver(I.cavity(6, nv=8), "fp64")
    other.init_uniform()
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a checkpoint" * 8)
    short = tmp_path / "short.ckpt"
    short.write_bytes(path.read_bytes()[:1000])
    # same cell and velocity counts, another mesh (a stretched O-grid) or
    # another velocity range: refused by the discretisation hash
    import dataclasses
    q = _prob()
    q.nodes_x, q.nodes_y = I.ogrid_nodes(20, 8, q=1.1)
    moved = Solver(q, "fp64")
    moved.init_uniform()
    wider = Solver(dataclasses.replace(_prob(), vrange=(-9.0, 9.0, -9.0, 9.0)), "fp64")
    wider.init_uniform()
    # a different Kn is a continuation: accepted
    kn = Solver(dataclasses.replace(_prob(), Kn=0.7), "fp64")
    kn.init_uniform()
    B.idg_load(kn.ctx, path)
    for ctx, f in ((other.ctx, path), (moved.ctx, path), (wider.ctx, path), (a.ctx, junk), (a.ctx, short),
                   (a.ctx, tmp_path / "missing")):
        with pytest.raises(B.IdgError) as e:
            B.idg_load(ctx, f)
        assert e.value.status == B.IDG_ERR_ARG
