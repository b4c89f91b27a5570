"""Central finite differences of the oracle's steady wall force.

TEST INFRASTRUCTURE ONLY: used by tests/ to check the GPU adjoint.  The
objective is the force of the gas on the walls of the sides in a mask: the sum
over their faces of the momentum flux Phi (Eq. 27) of the converged state,
oriented from the gas into the wall.  Parameters are set through
inputs.with_params (Knudsen number, wall temperature and velocity).

A domain closed by walls and periodic sides has a one-parameter family of
steady states, indexed by the total mass sum_c Omega_c rho_c (the macroscopic
LU-SGS does not conserve mass per iteration, so the member reached from a
uniform start depends on the path).  There the perturbed solutions are
converged at the total mass of the unperturbed one, by adjusting the density
of the uniform start (secant steps), so that the differences are those of the
steady state at fixed mass.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_1709_01819_gb300 import inputs as I

from .oracle import Oracle


def wall_force(orc: Oracle, side_mask: int) -> np.ndarray:
    """(Fx, Fy) from the face fluxes of the oracle's last iteration."""
    phi = orc.face_phi()
    fc = orc.faces()
    F = np.zeros(2)
    for f in range(orc.nf):
        if fc["bc"][f] != I.BC_WALL or not (side_mask >> int(fc["side"][f])) & 1:
            continue
        on = 1.0 if fc["L"][f] >= 0 else -1.0
        F += on * phi[f, 1:3]
    return F


def total_mass(orc: Oracle) -> float:
    _, _, area = orc.geometry()
    _, _, W = orc.get_state()
    return float(np.sum(area * W[:, 0]))


def closed(prob) -> bool:
    return all(b[0] != I.BC_FARFIELD for b in prob.bc)


def steady(prob, tol: float = 1e-13, max_iter: int = 20000, chunk: int = 50):
    """Iterate the oracle from the problem's uniform start until the residual,
    relative to the first iteration, is <= tol.  Returns (oracle, iterations,
    relative residual)."""
    orc = Oracle(prob)
    orc.init_uniform()
    r0, n, rel = None, 0, np.inf
    while n < max_iter:
        res = orc.iterate(chunk)
        if r0 is None:
            r0 = res[0]
        n += chunk
        rel = res[-1] / r0
        if rel <= tol:
            break
    return orc, n, rel


def steady_at_mass(prob, mass, tol: float = 1e-13, max_iter: int = 20000):
    """Steady state of a closed problem with total mass `mass` (to 1e-14)."""
    rho0 = prob.init[0]
    orc, _, _ = steady(prob, tol, max_iter)
    m = total_mass(orc)
    for _ in range(6):
        if abs(m - mass) <= 1e-14 * abs(mass):
            break
        rho0 *= mass / m  # the converged mass is nearly proportional to the start density
        p = dataclasses.replace(prob, init=(rho0,) + tuple(prob.init[1:]))
        orc, _, _ = steady(p, tol, max_iter)
        m = total_mass(orc)
    return orc


def objective(prob, side_mask: int, axis: int, mass=None, **kw) -> float:
    orc = steady(prob, **kw)[0] if mass is None else steady_at_mass(prob, mass, **kw)
    orc.iterate(1)  # fluxes of the converged state
    return float(wall_force(orc, side_mask)[axis])


def fd_gradient(prob, params, side_mask: int, axis: int, rel_step: float = 1e-4, **kw) -> np.ndarray:
    """dJ/dp by central differences, step rel_step * |p| per parameter (at the
    base solution's total mass for a closed domain)."""
    mass = total_mass(steady(prob, **kw)[0]) if closed(prob) else None
    base = []
    for pid in params:
        kind, mask = pid & 0xFF, pid >> 8
        if kind == I.PAR_KN:
            base.append(prob.Kn)
        else:
            side = (mask & -mask).bit_length() - 1
            base.append(prob.bc[side][{I.PAR_WALL_T: 4, I.PAR_WALL_U: 2, I.PAR_WALL_V: 3}[kind]])
    g = np.zeros(len(params))
    for i, pid in enumerate(params):
        h = rel_step * max(abs(base[i]), 1e-3)
        vp, vm = list(base), list(base)
        vp[i] += h
        vm[i] -= h
        jp = objective(I.with_params(prob, params, vp), side_mask, axis, mass, **kw)
        jm = objective(I.with_params(prob, params, vm), side_mask, axis, mass, **kw)
        g[i] = (jp - jm) / (2 * h)
    return g
