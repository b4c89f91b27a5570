"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle alone): the oracle still reproduces them, and the stored profile
itself obeys what plane Couette flow with walls moving at -U and +U fixes
independently of any implementation -- u antisymmetric and rho, T symmetric
about the mid-plane, a monotone shear profile with a slip velocity below the
wall speed, and no wall-normal flow beyond the discretisation level.  (The
total mass is not fixed: the LU-SGS predictor's approximate factorisation
does not conserve it per iteration, so a closed box settles on the steady
state of the mass it drifted to, 1.0004 here.)"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "couette_64_kn0.1_v32_oracle.txt")


def _stored():
    return np.loadtxt(GOLD, comments="#")


def test_stored_couette_profile_obeys_the_symmetries_and_conservation():
    d = _stored()
    y, rho, u, v, T = d[:, 0], d[:, 1], d[:, 2], d[:, 3], d[:, 4]
    n = len(y)
    assert n == 64 and np.allclose(y, (np.arange(n) + 0.5) / n, rtol=0, atol=1e-15)
    assert np.abs(u + u[::-1]).max() <= 1e-10
    assert np.abs(rho - rho[::-1]).max() <= 1e-10
    assert np.abs(T - T[::-1]).max() <= 1e-10
    assert 0 < -u[0] < 0.1 and 0 < u[-1] < 0.1  # slip at Kn 0.1
    assert np.all(np.diff(u) > 0)  # monotone shear profile
    assert np.abs(v).max() <= 1e-4 * 0.1  # 1.7e-6 in the wall cells


def test_oracle_reproduces_the_stored_couette_profile():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    o, n, rel = make_golden.converged_couette()
    assert rel <= make_golden.TOL
    m = o.moments()
    d = _stored()
    scale = np.array([1.0, 0.1, 0.1, 1.0, 0.01, 0.01])  # rho, u, v, T, qx, qy
    assert np.all(np.abs(m - d[:, 1:]).max(axis=0) <= 1e-13 * scale / 0.01)
