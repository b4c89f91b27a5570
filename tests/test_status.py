"""Status words through the C ABI: a state that is not finite makes the
residual NaN, which the device records and idg_iterate / idg_batch_iterate
return as IDG_ERR_NONFINITE (no fault, no trap: NaN only flows through the
arithmetic, no index depends on it); a restart clears it; a tolerance not
reached is IDG_ERR_NOT_CONVERGED with the iterations still done."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_state_is_reported_and_a_restart_clears_it(prec):
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300.solver import Solver
    s = Solver(I.cavity(8, Kn=0.1, U=0.15, nv=8), prec)
    s.init_uniform()
    s.iterate(3)
    G, H, W = s.get_state()
    Wbad = W.copy()
    Wbad[5, 3] = np.nan
    s.set_state(G, H, Wbad)
    with pytest.raises(B.IdgError) as e:
        s.iterate(4)
    assert e.value.status == B.IDG_ERR_NONFINITE
    # set_state with a finite state clears the recorded divergence
    s.set_state(G, H, W)
    ok, n, r = s.iterate(4)
    assert n == 4 and np.isfinite(r)
    assert np.isfinite(s.get_state()[0]).all()
    # and so does init_uniform
    s.set_state(G, H, Wbad)
    with pytest.raises(B.IdgError):
        s.iterate(2)
    s.init_uniform()
    ok, n, r = s.iterate(2)
    assert n == 2 and np.isfinite(r)


def test_tolerance_not_reached_is_not_converged_with_the_work_done():
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300.solver import Solver
    s = Solver(I.cavity(8, Kn=0.1, U=0.15, nv=8), "fp64")
    s.init_uniform()
    st, n, r = B.idg_iterate(s.ctx, 5, 1e-14, s.stream)
    assert st == B.IDG_ERR_NOT_CONVERGED and n == 5 and np.isfinite(r) and r > 1e-14
    assert len(s.residual_history()) == 5


def test_one_diverged_instance_fails_the_batch():
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300.solver import BatchSolver
    probs = [I.cavity(8, Kn=0.1, U=0.15, nv=8), I.cavity(6, Kn=0.5, U=0.1, nv=8)]
    bs = BatchSolver(probs, "mixed")
    bs.iterate(2)
    G, H, W = bs.solvers[1].get_state()
    W[0, 0] = np.inf
    bs.solvers[1].set_state(G, H, W)
    with pytest.raises(B.IdgError) as e:
        bs.iterate(3)
    assert e.value.status == B.IDG_ERR_NONFINITE
