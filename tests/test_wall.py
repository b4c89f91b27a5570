"""idg_get_wall: per-face wall pressure, shear stress and heat flux (the wall
quantities Section 3 plots along the cylinder), through the C ABI.

Checked three ways: against the same definitions applied to the oracle's
face flux moments (Eq. 27) on a cavity, lid moving; against the discrete
free-molecular closed form of the Couette shear stress (each half-range the
Maxwellian of the wall it left); and against Fourier conduction between two
resting walls at different temperatures (the heat flux into the cold wall
equals the one out of the hot wall and the conducted flux of the interior)."""
import math

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


def _converge(s, tol, max_iter=60000):
    ok, n, r = s.iterate(max_iter, tol)
    assert ok, (n, r)


def test_wall_quantities_match_the_oracles_face_fluxes():
    from paper_1709_01819_gb300.solver import Solver
    n, U = 12, 0.15
    prob = I.cavity(n, Kn=0.075, U=U, nv=16, vmax=4.0)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(6)
    s = Solver(prob, "fp64")
    s.init_uniform()
    s.iterate(6)
    fc, phi = o.faces(), o.face_phi()
    for side in range(4):
        got = s.wall(side)
        sel = [f for f in range(o.nf) if fc["bc"][f] == I.BC_WALL and fc["side"][f] == side]
        assert got.shape == (len(sel), 5) and len(sel) == n
        Uw = prob.bc[side][2]
        for row, f in zip(got, sel):
            on = 1.0 if fc["L"][f] >= 0 else -1.0
            nx, ny, S = on * fc["nx"][f], on * fc["ny"][f], fc["S"][f]
            px, py, en = (on * phi[f, q] / S for q in (1, 2, 3))
            want = [px * nx + py * ny, -px * ny + py * nx, en - Uw * px]
            scale = max(abs(px), abs(py), abs(en))
            assert np.abs(row[2:] - want).max() <= 1e-12 * scale, (side, f, row, want)
        # midpoints on the side's edge of the unit square, in face order
        x, y = got[:, 0], got[:, 1]
        edge = {0: (x, 0.0), 1: (x, 1.0), 2: (y, 0.0), 3: (y, 1.0)}[side]
        assert np.allclose(edge[0], edge[1], atol=1e-14)
        along = y if side < 2 else x
        assert np.allclose(np.sort(along), (np.arange(n) + 0.5) / n, atol=1e-14)
    # the lid (n = +y, t = (-1, 0)) drags the slower gas along and the gas
    # holds it back: the x-momentum flux into the lid is negative, tau_w > 0
    lid = s.wall(I.JMAX)
    assert lid[:, 3].sum() > 0 and np.mean(lid[:, 3] > 0) > 0.5


def test_free_molecular_couette_shear_is_the_half_range_closed_form():
    from paper_1709_01819_gb300.solver import Solver
    U = 0.1
    prob = I.couette(8, U=U, Kn=1e6, nv=32, vmax=4.0, cfl_imp=1000.0)
    s = Solver(prob, "fp64")
    s.init_uniform()
    s.iterate(200)
    ux, uy, w = s.velocity_grid()
    M = lambda Uw: (1.0 / math.pi) * np.exp(-((ux - Uw) ** 2 + uy ** 2))
    up, dn = uy > 0, uy < 0
    closed = (np.sum((w * ux * uy * M(-U))[up]) + np.sum((w * ux * uy * M(U))[dn])) / \
             (np.sum((w * M(-U))[up]) + np.sum((w * M(U))[dn]))
    G, _, _ = s.get_state()
    rho = (G @ w).mean()
    for side in (I.JMIN, I.JMAX):
        wq = s.wall(side)
        assert wq.shape == (1, 5)
        # both walls: tau_w = -Pi_xy (t = (-n_y, n_x)), Pi_xy = rho * closed
        assert abs(wq[0, 3] + rho * closed) < 1e-6 * abs(rho * closed), (side, wq[0, 3], -rho * closed)
    assert abs(s.wall(I.JMIN)[0, 2] - s.wall(I.JMAX)[0, 2]) < 1e-8 * abs(s.wall(I.JMAX)[0, 2])


@pytest.mark.parametrize("shakhov", [0, 1])
def test_heat_flux_between_walls_at_different_temperatures(shakhov):
    from paper_1709_01819_gb300.solver import Solver
    n, kn = 32, 2e-3
    kw = dict(shakhov=1, Pr=2.0 / 3.0) if shakhov else {}
    pr = 2.0 / 3.0 if shakhov else 1.0
    prob = I.couette(n, U=0.0, Kn=kn, nv=16, vmax=4.0, cfl_imp=1000.0, **kw)
    prob.bc[2] = (I.BC_WALL, 1.0, 0.0, 0.0, 0.95)
    prob.bc[3] = (I.BC_WALL, 1.0, 0.0, 0.0, 1.05)
    s = Solver(prob, "fp64")
    s.init_uniform()
    _converge(s, 1e-10)
    cold, hot = s.wall(I.JMIN)[0], s.wall(I.JMAX)[0]
    # energy goes from the hot wall through the gas into the cold wall
    assert cold[4] > 0 and hot[4] < 0
    # (to the convergence level: the residual stops at 1e-10 of its start)
    assert abs(cold[4] + hot[4]) < 1e-6 * abs(cold[4])
    # and equals the conducted flux of Fourier's law in the interior,
    # q = -((D+2)/2) (mu(T)/Pr) d(RT)/dy with D = 2 + K = 3, mu = mu_ref T^0.5
    m = s.moments()
    T = m[:, 3]
    y = (np.arange(n) + 0.5) / n
    mu_ref = 15 * math.sqrt(2 * math.pi * 0.5) * kn / (2 * 4 * 6)
    g = np.gradient(T, y)
    mid = n // 2
    qf = -2.5 * (mu_ref * T[mid] ** 0.5 / pr) * 0.5 * g[mid]
    assert abs(cold[4] / -qf - 1) < 5e-3, (cold[4], -qf)
