"""Writes the stored expected values under tests/golden/ from the FP64 oracle
alone (no library code): the converged plane Couette flow of 64 cells with
32 x 32 trapezoid velocities on [-4, 4]^2 (walls at y = 0 and 1 moving with
-0.1 and +0.1, BGK, Kn 0.1, K = 1), iterated from the uniform Maxwellian
until the residual ||R_W/Omega|| falls below 1e-12 of its first value.

Run from the repository root: python tests/golden/make_golden.py
A change to the oracle's arithmetic that moves these values regenerates the
file in the same commit, which names the passage of the paper behind it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1709_01819_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "couette_64_kn0.1_v32_oracle.txt")
TOL = 1e-12


def converged_couette():
    o = O.Oracle(I.couette_c1())
    o.init_uniform()
    hist = []
    while len(hist) < 100000:
        hist.extend(o.iterate(500))
        if hist[-1] <= TOL * hist[0]:
            break
    return o, len(hist), hist[-1] / hist[0]


def main():
    o, n, rel = converged_couette()
    cx, cy, _ = o.geometry()
    m = o.moments()
    with open(OUT, "w") as f:
        f.write("# plane Couette flow, 64 cells, 32x32 trapezoid velocities on [-4,4]^2, BGK, Kn 0.1,\n")
        f.write("# walls y=0 (u=-0.1) and y=1 (u=+0.1), T_w = 1; FP64 oracle converged to a residual\n")
        f.write(f"# of {rel:.3e} of the first ({n} iterations); written by tests/golden/make_golden.py\n")
        f.write("# columns: y rho u v T qx qy (T in units of T_ref)\n")
        for k in range(len(cy)):
            f.write(" ".join(f"{x:.17e}" for x in (cy[k], *m[k])) + "\n")
    print("wrote", OUT, n, "iterations, residual", rel)


if __name__ == "__main__":
    main()
