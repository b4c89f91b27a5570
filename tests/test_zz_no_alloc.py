"""idg_get_moments_noalloc: the moments entry point that allocates nothing.

It serves callers that must not allocate device memory for a query (a
real-time loop whose memory is fixed up front, a plug-in inside another
framework's memory pool): its scratch is a static device array of the library
instead of the caller's workspace.  This
checks, through the C ABI, that two calls in a row give the same moments as
idg_get_moments, and that meshes above the documented 16384-cell limit are
refused.  The file is named to be collected last.
"""
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
def test_noalloc_moments_match_get_moments_twice(precision):
    import torch
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300.solver import Solver
    prob = I.cavity(12, Kn=0.075, U=0.15, nv=16, vmax=4.0)
    s = Solver(prob, precision)
    s.init_uniform()
    s.iterate(7)
    ref = s.moments()
    for _ in range(2):
        out = torch.full((s.N, 6), float("nan"), dtype=torch.float64, device="cuda")
        B.idg_get_moments_noalloc(s.ctx, out.data_ptr(), s.stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)
    # and after the state has moved on
    s.iterate(3)
    ref = s.moments()
    out = torch.empty((s.N, 6), dtype=torch.float64, device="cuda")
    B.idg_get_moments_noalloc(s.ctx, out.data_ptr(), s.stream)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-15)


def test_noalloc_moments_reject_meshes_above_the_limit():
    import torch
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300.solver import Solver
    prob = I.cavity(129, Kn=0.075, U=0.15, nv=4, vmax=4.0)  # 16641 cells
    s = Solver(prob, "mixed")
    s.init_uniform()
    out = torch.empty((s.N, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(B.IdgError) as e:
        B.idg_get_moments_noalloc(s.ctx, out.data_ptr(), s.stream)
    assert e.value.status == B.IDG_ERR_ARG
    assert "16384" in str(e.value)
