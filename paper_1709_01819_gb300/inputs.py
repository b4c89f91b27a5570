"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module only describes problems: mesh node coordinates, boundary and gas
settings, velocity-grid choices and seeded random draws.  It holds none of the
scheme's arithmetic (no equilibria, moments, fluxes or sweeps), so the oracle
and the CUDA library each compute everything from the same description.

Units: reference density 1, reference length 1, velocity unit sqrt(2 R T_ref);
temperatures are in units of T_ref and R T_ref = 1/2.

The five workloads (uniform-Maxwellian starts, no dataset is involved):
  couette_c1     1 x 64 periodic-x Couette, walls at +-U, 32^2 trapezoid velocities
  cavity_c2      64^2 lid-driven cavity, Shakhov Pr=2/3, Kn=0.075, 32^2 trapezoid
  cavity_c3      128^2 tanh-stretched cavity, Kn=1e-3, 28^2 Gauss-Hermite
  batch_c4       64 cavities with seeded Kn, lid speed and grid size
  cylinder_c5    121 x 81 O-grid around a cylinder, Ma=5, 89^2 Simpson velocities
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

BC_PERIODIC, BC_WALL, BC_FARFIELD = 0, 1, 2
NC_TRAP, NC_SIMPSON, GAUSS_HERMITE = 0, 1, 2
IMIN, IMAX, JMIN, JMAX = 0, 1, 2, 3
# parameters of the steady solve that gradients are taken with respect to:
# kind | (mask of sides << 8), the ids of idg_adjoint
PAR_KN, PAR_WALL_T, PAR_WALL_U, PAR_WALL_V = 0, 1, 2, 3


def param(kind: int, side_mask: int = 0) -> int:
    return kind | (side_mask << 8)


@dataclasses.dataclass
class Problem:
    """One steady-flow problem on a structured 2-D block."""

    nodes_x: np.ndarray            # (nj+1, ni+1) node x coordinates
    nodes_y: np.ndarray            # (nj+1, ni+1)
    bc: List[Tuple[int, float, float, float, float]]  # per side: kind, rho, u, v, T
    vrule: int = NC_TRAP
    nvx: int = 32
    nvy: int = 32
    vrange: Tuple[float, float, float, float] = (-4.0, 4.0, -4.0, 4.0)
    K: int = 1
    Pr: float = 1.0
    omega: float = 0.5
    Kn: float = 0.1
    RT_ref: float = 0.5
    shakhov: int = 0
    cfl_imp: float = 100.0
    cfl_phys: float = 0.5
    limiter: int = 0
    flags: int = 0
    lusgs_omega: float = 2.0
    relax_sweeps: int = 0          # macroscopic predictor: 0 LU-SGS, n >= 1 n point-relaxation sweeps
    implicit_wall: int = 0         # 1: linearised diffuse-wall ghost increments in the micro sweeps (Eq. 34-35)
    venkat_k: float = 0.0          # limiter smoothing constant K (eps^2 = (K sqrt(area))^3); 0: Eq. 16-17 as printed
    # unstructured mesh (triangles and quadrilaterals): nodes_x, nodes_y are
    # then flat node arrays, cell_nodes [ncells][4] int (counter-clockwise, -1
    # as the 4th node of a triangle), edge_side [ncells][4] int: boundary group
    # (0..3, the bc entry) of edge m (node m -> m+1) where it has no neighbour
    cell_nodes: Optional[np.ndarray] = None
    edge_side: Optional[np.ndarray] = None
    init: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 1.0)  # rho, u, v, T
    name: str = ""

    @property
    def unstructured(self) -> bool:
        return self.cell_nodes is not None

    @property
    def ni(self) -> int:
        return len(self.cell_nodes) if self.unstructured else self.nodes_x.shape[1] - 1

    @property
    def nj(self) -> int:
        return 1 if self.unstructured else self.nodes_x.shape[0] - 1

    @property
    def ncells(self) -> int:
        return self.ni * self.nj

    @property
    def nvel(self) -> int:
        return self.nvx * self.nvy


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def uniform_nodes(ni: int, nj: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    xs = np.linspace(x0, x1, ni + 1)
    ys = np.linspace(y0, y1, nj + 1)
    X, Y = np.meshgrid(xs, ys)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def tanh_coords(n: int, beta: float) -> np.ndarray:
    """Nodes on [0,1] clustered toward both ends: x_i = (1 + tanh(beta(2i/n-1))/tanh(beta))/2."""
    i = np.arange(n + 1, dtype=np.float64)
    return 0.5 * (1.0 + np.tanh(beta * (2.0 * i / n - 1.0)) / math.tanh(beta))


def tanh_nodes(n: int, beta: float):
    c = tanh_coords(n, beta)
    X, Y = np.meshgrid(c, c)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def ogrid_nodes(ntheta: int, nr: int, q: float = 1.05, rmax: float = 15.0):
    """Body-fitted O-grid around the unit cylinder.

    i runs circumferentially (periodic, counter-clockwise starting at the
    downstream axis), j radially outward with r_j = 1 + (rmax-1)(q^j-1)/(q^nr-1).
    Node column i = ntheta repeats column 0 exactly.  For i increasing
    counter-clockwise and j outward the cells are clockwise-oriented, so the
    angle runs clockwise instead: theta_i = -2 pi i / ntheta.
    """
    j = np.arange(nr + 1, dtype=np.float64)
    r = 1.0 + (rmax - 1.0) * (q ** j - 1.0) / (q ** nr - 1.0)
    i = np.arange(ntheta + 1, dtype=np.float64)
    th = -2.0 * math.pi * i / ntheta
    th[-1] = th[0] - 2.0 * math.pi
    cos_t = np.cos(th)
    sin_t = np.sin(th)
    cos_t[-1], sin_t[-1] = cos_t[0], sin_t[0]
    X = r[:, None] * cos_t[None, :]
    Y = r[:, None] * sin_t[None, :]
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def quads_to_unstructured(X: np.ndarray, Y: np.ndarray, tri=None, wrap_i: bool = False):
    """Cells of a structured node block (X, Y: (nj+1, ni+1)) as an unstructured
    mesh: nodes flattened (node (i, j) -> j (ni+1) + i; with wrap_i, column ni
    is column 0 and i runs periodically), cell (i, j) the quad (i,j), (i+1,j),
    (i+1,j+1), (i,j+1), or -- where tri(i, j) is true -- the two triangles
    split along the diagonal (i,j)-(i+1,j+1).  Cells are numbered row by row
    (quad or first triangle, then second).  Boundary edges: j = 0 -> side 2
    (JMIN), j = nj -> 3 (JMAX), i = 0 -> 0 (IMIN), i = ni -> 1 (IMAX)."""
    nj, ni = X.shape[0] - 1, X.shape[1] - 1
    nc = ni if wrap_i else ni + 1
    if wrap_i:
        nx, ny = X[:, :ni].ravel(), Y[:, :ni].ravel()
    else:
        nx, ny = X.ravel(), Y.ravel()
    node = lambda i, j: j * nc + (i % ni if wrap_i else i)
    cells, sides = [], []
    for j in range(nj):
        for i in range(ni):
            a, b, c, d = node(i, j), node(i + 1, j), node(i + 1, j + 1), node(i, j + 1)
            south = JMIN if j == 0 else -1
            north = JMAX if j == nj - 1 else -1
            west = IMIN if (i == 0 and not wrap_i) else -1
            east = IMAX if (i == ni - 1 and not wrap_i) else -1
            if tri is not None and tri(i, j):
                cells += [[a, b, c, -1], [a, c, d, -1]]
                sides += [[south, east, -1, -1], [-1, north, west, -1]]
            else:
                cells.append([a, b, c, d])
                sides.append([south, east, north, west])
    return (np.ascontiguousarray(nx, dtype=np.float64), np.ascontiguousarray(ny, dtype=np.float64),
            np.ascontiguousarray(np.array(cells, dtype=np.int32)), np.ascontiguousarray(np.array(sides, dtype=np.int32)))


def as_unstructured(prob: Problem, tri=None, wrap_i: bool = False, name: Optional[str] = None) -> Problem:
    """The same problem on the unstructured description of its block (see
    quads_to_unstructured); with wrap_i the periodic i-direction becomes plain
    connectivity and sides IMIN/IMAX are unused."""
    import dataclasses

    nx, ny, cells, sides = quads_to_unstructured(prob.nodes_x, prob.nodes_y, tri, wrap_i)
    bc = list(prob.bc)
    if wrap_i:
        bc[IMIN] = bc[IMAX] = (BC_WALL, 1.0, 0.0, 0.0, 1.0)  # unused
    return dataclasses.replace(prob, nodes_x=nx, nodes_y=ny, bc=bc, cell_nodes=cells, edge_side=sides,
                               name=name or (prob.name + "_unstructured"))


def tri_cavity(n: int = 16, **kw) -> Problem:
    """The lid-driven cavity on n x n squares each split into two triangles
    along the diagonal from its lower left to its upper right corner (2 n^2
    cells)."""
    prob = cavity(n, **kw)
    return as_unstructured(prob, tri=lambda i, j: True, name=f"cavity_tri_{n}x{n}")


def hybrid_cylinder(ntheta: int = 24, nr: int = 12, nr_quad: int = 4, **kw) -> Problem:
    """The cylinder O-grid as a hybrid unstructured mesh: quadrilaterals in the
    nr_quad rings next to the wall, triangles outside, the ring closed by
    connectivity (no periodic boundary)."""
    prob = cylinder(ntheta=ntheta, nr=nr, **kw)
    return as_unstructured(prob, tri=lambda i, j: j >= nr_quad, wrap_i=True,
                           name=f"cylinder_hybrid_{ntheta}x{nr}_q{nr_quad}")


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def couette(ncell: int = 64, U: float = 0.1, Kn: float = 0.1, nv: int = 32, vmax: float = 4.0,
            cfl_imp: float = 100.0, Tw: float = 1.0, Pr: float = 1.0, shakhov: int = 0,
            omega: float = 0.5, name: str = "couette") -> Problem:
    """Plane Couette flow: 1 x ncell cells periodic in x, diffuse walls at y=0 (-U) and y=1 (+U)."""
    X, Y = uniform_nodes(1, ncell, 0.0, 1.0 / ncell, 0.0, 1.0)
    bc = [(BC_PERIODIC, 0, 0, 0, 0), (BC_PERIODIC, 0, 0, 0, 0),
          (BC_WALL, 1.0, -U, 0.0, Tw), (BC_WALL, 1.0, U, 0.0, Tw)]
    return Problem(X, Y, bc, NC_TRAP, nv, nv, (-vmax, vmax, -vmax, vmax), K=1, Pr=Pr,
                   omega=omega, Kn=Kn, shakhov=shakhov, cfl_imp=cfl_imp, init=(1.0, 0.0, 0.0, Tw),
                   name=name)


def couette_c1() -> Problem:
    return couette(64, 0.1, 0.1, 32, 4.0, 100.0, name="couette_64_kn0.1_v32")


def cavity(n: int = 64, Kn: float = 0.075, U: float = 0.15, nv: int = 32, vmax: float = 4.0,
           cfl_imp: float = 1000.0, shakhov: int = 1, Pr: float = 2.0 / 3.0, omega: float = 0.5,
           vrule: int = NC_TRAP, stretch_beta: Optional[float] = None, Tw: float = 1.0,
           name: str = "cavity") -> Problem:
    """Lid-driven square cavity: isothermal diffuse walls, lid at y=1 moving with +U."""
    if stretch_beta is None:
        X, Y = uniform_nodes(n, n)
    else:
        X, Y = tanh_nodes(n, stretch_beta)
    bc = [(BC_WALL, 1.0, 0.0, 0.0, Tw), (BC_WALL, 1.0, 0.0, 0.0, Tw),
          (BC_WALL, 1.0, 0.0, 0.0, Tw), (BC_WALL, 1.0, U, 0.0, Tw)]
    return Problem(X, Y, bc, vrule, nv, nv, (-vmax, vmax, -vmax, vmax), K=1, Pr=Pr,
                   omega=omega, Kn=Kn, shakhov=shakhov, cfl_imp=cfl_imp, init=(1.0, 0.0, 0.0, Tw),
                   name=name)


def cavity_c2() -> Problem:
    return cavity(64, 0.075, 0.15, 32, 4.0, 1000.0, name="cavity_64x64_kn0.075_v32")


# tanh stretching with min/max spacing ratio 0.1 for 128 cells
C3_BETA = 1.83297


def cavity_c3() -> Problem:
    return cavity(128, 1e-3, 0.15, 28, 4.0, 1e4, vrule=GAUSS_HERMITE, stretch_beta=C3_BETA,
                  name="cavity_128x128_tanh_kn1e-3_gh28")


def cylinder(ntheta: int = 121, nr: int = 81, Kn: float = 0.1, Ma: float = 5.0, nv: int = 89,
             vmax: float = 15.0, q: float = 1.05, rmax: float = 15.0, cfl_imp: float = 1000.0,
             Tw: float = 1.0, limiter: int = 1, name: str = "cylinder") -> Problem:
    """Hypersonic flow around the unit cylinder on an O-grid, free stream along +x."""
    X, Y = ogrid_nodes(ntheta, nr, q, rmax)
    gamma = 5.0 / 3.0
    Uinf = Ma * math.sqrt(gamma * 0.5)
    bc = [(BC_PERIODIC, 0, 0, 0, 0), (BC_PERIODIC, 0, 0, 0, 0),
          (BC_WALL, 1.0, 0.0, 0.0, Tw), (BC_FARFIELD, 1.0, Uinf, 0.0, 1.0)]
    return Problem(X, Y, bc, NC_SIMPSON if nv % 2 else NC_TRAP, nv, nv,
                   (-vmax, vmax, -vmax, vmax), K=1, Pr=2.0 / 3.0, omega=0.81, Kn=Kn, shakhov=1,
                   cfl_imp=cfl_imp, limiter=limiter, init=(1.0, Uinf, 0.0, 1.0), name=name)


def cylinder_c5() -> Problem:
    # implicit CFL 30: from the impulsive uniform start 100 and above diverge,
    # 10 converges more slowly (2384 against 1904 iterations to 1e-6)
    return cylinder(cfl_imp=30.0, name="cylinder_121x81_ma5_kn0.1_v89")


C4_SEED = 170901819


def batch_c4(count: int = 64, seed: int = C4_SEED, sizes=(32, 48, 64, 96), nv: int = 32) -> List[Problem]:
    """Seeded batch of cavities: Kn log-uniform in [1e-3, 10], lid speed uniform in
    [0.05, 0.3], grid size drawn from `sizes` (numpy PCG64 generator)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        kn = 10.0 ** rng.uniform(-3.0, 1.0)
        U = rng.uniform(0.05, 0.3)
        n = int(rng.choice(np.asarray(sizes)))
        out.append(cavity(n, kn, U, nv, 4.0, 1000.0, name=f"batch{b}_n{n}"))
    return out


# --------------------------------------------------------------------------
# seeded states for parity tests
# --------------------------------------------------------------------------

def random_state(prob: Problem, seed: int, amp: float = 0.05):
    """A smooth, positive, non-equilibrium test state (G, H, W) in float64.

    G, H are Gaussians in velocity with smoothly varying centres and widths,
    times (1 + amp * noise); W is an arbitrary smooth positive field of the
    right magnitudes.  Nothing here is the scheme's equilibrium: it is just a
    reproducible, physically sized input.
    """
    rng = np.random.default_rng(seed)
    N = prob.ncells
    if prob.unstructured:
        # smooth in space: from the cells' node means, scaled to [0, 1]
        cn = np.asarray(prob.cell_nodes)
        tri = cn[:, 3] < 0
        idx = np.where(cn < 0, cn[:, :1], cn)  # a triangle's 4th entry repeats node 0
        Xn, Yn = np.asarray(prob.nodes_x)[idx], np.asarray(prob.nodes_y)[idx]
        cnt = np.where(tri, 3.0, 4.0)
        cx = (Xn.sum(axis=1) - np.where(tri, Xn[:, 3], 0.0)) / cnt
        cy = (Yn.sum(axis=1) - np.where(tri, Yn[:, 3], 0.0)) / cnt
        s = (cx - cx.min()) / max(np.ptp(cx), 1e-300)
        t = (cy - cy.min()) / max(np.ptp(cy), 1e-300)
    else:
        ni, nj = prob.ni, prob.nj
        jj, ii = np.meshgrid(np.arange(nj), np.arange(ni), indexing="ij")
        s = (ii.ravel() + 0.5) / ni
        t = (jj.ravel() + 0.5) / nj
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * s) * np.cos(np.pi * t)
    u = 0.05 * np.cos(np.pi * t) + prob.init[1]
    v = 0.03 * np.sin(2 * np.pi * s)
    T = prob.init[3] * (1.0 + 0.05 * np.cos(np.pi * s) * np.sin(np.pi * t))
    # velocity nodes only to place the test Gaussians (plain uniform sample points)
    x0, x1, y0, y1 = prob.vrange
    vx = np.linspace(x0, x1, prob.nvx) if prob.vrule != GAUSS_HERMITE else np.linspace(-5, 5, prob.nvx)
    vy = np.linspace(y0, y1, prob.nvy) if prob.vrule != GAUSS_HERMITE else np.linspace(-5, 5, prob.nvy)
    VX, VY = np.meshgrid(vx, vy)
    VX = VX.ravel()[None, :]
    VY = VY.ravel()[None, :]
    RT = 0.5 * T[:, None]
    gauss = rho[:, None] / (2 * np.pi * RT) * np.exp(-((VX - u[:, None]) ** 2 + (VY - v[:, None]) ** 2) / (2 * RT))
    noise = rng.standard_normal(gauss.shape)
    G = gauss * (1.0 + amp * noise)
    H = RT * gauss * (1.0 + amp * rng.standard_normal(gauss.shape))
    W = np.stack([rho, rho * u, rho * v, 0.5 * rho * (u * u + v * v + 3.0 * RT[:, 0])], axis=1)
    return (np.ascontiguousarray(G.reshape(N, -1)), np.ascontiguousarray(H.reshape(N, -1)),
            np.ascontiguousarray(W))


def with_params(prob: Problem, params, values) -> Problem:
    """A copy of prob with the parameters (param() ids) set to values: the
    Knudsen number, or the temperature / x / y velocity of the walls of the
    sides in the id's mask."""
    bc = [list(b) for b in prob.bc]
    kn = prob.Kn
    for pid, val in zip(params, values):
        kind, mask = pid & 0xFF, pid >> 8
        if kind == PAR_KN:
            kn = float(val)
            continue
        slot = {PAR_WALL_T: 4, PAR_WALL_U: 2, PAR_WALL_V: 3}[kind]
        for side in range(4):
            if (mask >> side) & 1:
                if bc[side][0] != BC_WALL:
                    raise ValueError(f"side {side} is not a wall")
                bc[side][slot] = float(val)
    return dataclasses.replace(prob, bc=[tuple(b) for b in bc], Kn=kn)
