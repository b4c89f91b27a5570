"""The local chain rules of the adjoint (csrc/adjoint_math.h) against central
differences of their own forward functions, compiled for the CPU with g++."""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1709_01819_gb300", "csrc")


def test_local_vjps_match_central_differences():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "check")
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                               os.path.join(HERE, "adjoint_math_check.cpp"), "-o", exe])
        out = subprocess.check_output([exe], text=True)
    errs = {line.split()[0]: float(line.split()[1]) for line in out.strip().splitlines()}
    assert set(errs) == {"prim_vjp", "tau_vjp", "eq_vjp_bgk", "eq_vjp_shakhov", "bnd_vjp", "heat_uv_vjp",
                         "venkat_d", "venkat_eps_d", "euler_jacT"}
    for name, e in errs.items():
        # central differences with step 1e-6 on O(1) inputs: ~1e-9 truncation + rounding
        assert e < 1e-6, (name, e)
