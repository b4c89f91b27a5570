"""Mixed precision (f in float32; moments, predictor and residual in float64)
against the float64 path at steady state, on reduced versions of the two
HBM-sized workloads: the near-continuum stretched cavity (Kn 1e-3,
Gauss-Hermite velocities, CFL 1e4) and the Ma 5 cylinder with the
Venkatakrishnan limiter.  The bar is the stated tolerance of the method's
mixed-precision form: rel. L2 <= 1e-5 on the velocity and the temperature.
The float64 path itself equals the oracle to 1e-12 per iteration
(test_gpu_parity, test_full_size)."""
import dataclasses

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


CASES = {
    # 32^2 tanh-stretched cavity, 16^2 Gauss-Hermite velocities, Kn 1e-3; the
    # point-relaxation predictor only shortens the way to the same fixed point
    "cavity32_gh16_kn1e-3": dataclasses.replace(
        I.cavity(32, Kn=1e-3, U=0.15, nv=16, vrule=I.GAUSS_HERMITE, stretch_beta=1.83297, cfl_imp=1e4),
        relax_sweeps=25),
    # 30 x 20 O-grid, Ma 5, 41^2 Simpson velocities on [-12, 12], limiter on
    "cylinder30x20_ma5_v41": I.cylinder(ntheta=30, nr=20, nv=41, vmax=12.0, cfl_imp=30.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_steady_field_within_1e5_of_fp64(name):
    """Mixed precision converged to its float32 floor (the relative residual
    stops near 3e-7); float64 continued from that state until its own
    residual has fallen by at least 1e5 more; the two fields compared.  At
    full size (the 128^2 cavity, the 121 x 81 cylinder) the same measurement
    gives rel. L2 8.5e-8 / 1.7e-6 on u and 5.9e-9 / 5.6e-6 on T.  The
    float32 path's vacuum limit of Eq. 18 (faces below 1e-6 of the reference
    density) acts only in the impulsive start's transient: at the converged
    field every cell's density is far above it, and the float64 path, which
    has no such limit, keeps the field."""
    from paper_1709_01819_gb300.solver import Solver
    prob = CASES[name]
    m = Solver(prob, "mixed")
    m.init_uniform()
    ok, n, r = m.iterate(30000, 1e-6)
    assert ok, ("mixed", n, r)
    m.iterate(n)  # as far again: onto the float32 floor
    G, H, W = m.get_state()
    mm = m.moments()
    f = Solver(prob, "fp64")
    f.init_uniform()
    f.set_state(G, H, W)
    f.iterate(max(4 * n, 2000))
    h = f.residual_history()
    assert h[-1] <= 1e-5 * h[0], (h[0], h[-1])
    mf = f.moments()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    eu = rel(mm[:, 1:3], mf[:, 1:3])
    eT = rel(mm[:, 3], mf[:, 3])
    print(f"{name}: rel. L2 u {eu:.3g}, T {eT:.3g}, min density {mm[:, 0].min():.3g}")
    assert eu <= 1e-5 and eT <= 1e-5, (eu, eT)
    assert mm[:, 0].min() > 1e-3 * prob.init[0], mm[:, 0].min()
