"""The macroscopic LU-SGS sweeps with one thread per line of cells
(IDG_TUNE_MACRO_KIND 1) against the FP64 oracle per iteration,
and against the hyperplane-slot kernel (kind 0), on the shapes that exercise
each of its neighbour paths: lines along j (columns) and along i (rows), a
periodic seam between the last and the first line (O-grids with fewer
circumferential than radial cells), a periodic seam along the lines, and
line counts that cross one to four warp boundaries at ragged positions, the
float64 line kernel's records filling shared memory at 140 and 150 lines
(Eq. 30).  The cavities run the kernel's seam-free instantiation, the O-grids
the one with seam terms; in mixed precision both are held to the slot kernel
(whose reciprocals are correctly rounded)."""
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


CASES = {
    # columns (ni <= nj), periodic i: the seam between line ni-1 and line 0
    "ogrid_8x20_cols_seam": I.cylinder(ntheta=8, nr=20, nv=11, vmax=8.0, Ma=2.0, Kn=0.5, cfl_imp=10.0),
    # columns over two warps (34 lines), periodic i across the warp boundary
    "ogrid_34x40_cols_seam_2warps": I.cylinder(ntheta=34, nr=40, nv=11, vmax=8.0, Ma=2.0, Kn=0.5, cfl_imp=10.0),
    # rows (ni > nj) over two warps (33 lines), periodic along the lines
    "ogrid_40x33_rows_2warps": I.cylinder(ntheta=40, nr=33, nv=11, vmax=8.0, Ma=2.0, Kn=0.5, cfl_imp=10.0),
    # 70 columns over three warps, the last one ragged
    "ogrid_70x74_cols_seam_3warps": I.cylinder(ntheta=70, nr=74, nv=11, vmax=8.0, Ma=2.0, Kn=0.5, cfl_imp=10.0),
    # 150 columns over five warps: the seam between line 149 (warp 4) and
    # line 0 (warp 0)
    "ogrid_150x156_cols_seam_5warps": I.cylinder(ntheta=150, nr=156, nv=11, vmax=8.0, Ma=2.0, Kn=0.5,
                                                  cfl_imp=10.0),
    # a closed box whose lines cross a warp boundary at 36
    "cavity_40x36_rows": I.cavity(40, Kn=0.075, U=0.15, nv=8, vmax=4.0),
    # 140 rows over five warps, the last one ragged
    "cavity_150x140_rows_5warps": I.cavity(150, Kn=0.075, U=0.15, nv=6, vmax=4.0),
}
_p = CASES["cavity_40x36_rows"]
_p.nodes_x, _p.nodes_y = I.uniform_nodes(40, 36, 0, 1, 0, 0.9)
_p = CASES["cavity_150x140_rows_5warps"]
_p.nodes_x, _p.nodes_y = I.uniform_nodes(150, 140, 0, 1, 0, 140 / 150)


@pytest.mark.parametrize("name", sorted(CASES))
def test_line_sweeps_match_oracle_and_hyperplane_kernel(name):
    kind = 1
    from paper_1709_01819_gb300.solver import Solver
    prob = CASES[name]
    o = O.Oracle(prob)
    o.init_uniform()
    s1 = Solver(prob, "fp64")
    s0 = Solver(prob, "fp64")
    assert s0.tuning()["macro_kind"] == 0  # the float64 default
    s1.set_tuning(macro_kind=kind)
    for s in (s0, s1):
        s.init_uniform()
    for n in (1, 3):
        o.iterate(n)
        s0.iterate(n)
        s1.iterate(n)
        Go, Ho, Wo = o.get_state()
        G1, H1, W1 = s1.get_state()
        G0, H0, W0 = s0.get_state()
        assert _rel(G1, Go) < 1e-12 and _rel(H1, Ho) < 1e-12, (name, n, _rel(G1, Go))
        for q in range(4):
            assert _rel(W1[:, q], Wo[:, q]) < 1e-12 or np.abs(W1[:, q] - Wo[:, q]).max() < 1e-14
            assert _rel(W1[:, q], W0[:, q]) < 1e-13 or np.abs(W1[:, q] - W0[:, q]).max() < 1e-15
        assert _rel(G1, G0) < 1e-13


@pytest.mark.parametrize("name", ["ogrid_150x156_cols_seam_5warps", "cavity_150x140_rows_5warps"])
def test_line_sweeps_mixed_precision_agree_with_hyperplane_kernel(name):
    kind = 1
    from paper_1709_01819_gb300.solver import Solver
    prob = CASES[name]
    s1 = Solver(prob, "mixed")
    s0 = Solver(prob, "mixed")
    s1.set_tuning(macro_kind=kind)
    s0.set_tuning(macro_kind=0)
    for s in (s0, s1):
        s.init_uniform()
        s.iterate(20)
    _, _, W1 = s1.get_state()
    _, _, W0 = s0.get_state()
    for q in range(4):
        assert _rel(W1[:, q], W0[:, q]) < 1e-5, (q, _rel(W1[:, q], W0[:, q]))
