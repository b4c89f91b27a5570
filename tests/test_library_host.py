"""CPU-side checks of libidugks: the library loads, exports every entry point
declared in include/idugks.h, validates its arguments, and its host-side
setup (velocity quadrature, face count, time step) agrees with the oracle
and with numpy's Gauss-Hermite rule.  No GPU work is launched here."""
import os
import re

import numpy as np
import pytest

from paper_1709_01819_gb300 import binding as B
from paper_1709_01819_gb300 import build as BUILD
from paper_1709_01819_gb300 import inputs as I
from paper_1709_01819_gb300.solver import configure

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    BUILD.build()


def declared_symbols():
    out = []
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            out += re.findall(r"\b(idg_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(out))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert "idg_iterate" in names and "idg_create" in names
    L = B.lib()
    for n in names:
        assert hasattr(L, n), f"missing export {n}"
    bound = {s[0] for s in B.SIGNATURES}
    assert set(names) <= bound, f"binding lacks {set(names) - bound}"


def test_header_is_c99_and_links_from_c(tmp_path):
    """include/idugks.h is a C header: a strict C99 translation unit that takes
    the address of every declared entry point compiles without warnings and
    links against the built library (C linkage, no C++ in the interface)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = declared_symbols()
    src = tmp_path / "abi.c"
    body = "\n".join(f"    (void *)&{n}," for n in names)
    src.write_text('#include "idugks.h"\n#include <stdio.h>\n'
                   "static void *const entry[] = {\n" + body + "\n};\n"
                   'int main(void) { printf("%u\\n", (unsigned)(sizeof entry / sizeof entry[0])); return 0; }\n')
    libdir = os.path.dirname(BUILD.LIB)
    libname = os.path.basename(BUILD.LIB)
    out = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-Wno-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(out), "-L", libdir,
                        "-l:" + libname, "-Wl,--unresolved-symbols=report-all"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([cc, "-std=c99", "-pedantic", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), "-x", "c", "-"],
                       input='#include "idugks.h"\nint main(void) { return 0; }\n', capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_nm_lists_every_symbol():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", BUILD.LIB], capture_output=True, text=True).stdout
    for n in declared_symbols():
        assert re.search(rf"\bT {n}\b", out), n


def _ctx(prob, precision=B.IDG_FP64):
    ctx = B.idg_create(precision, 0)
    configure(ctx, prob)
    return ctx


def test_argument_validation_returns_status_codes():
    L = B.lib()
    import ctypes as C
    h = C.c_void_p()
    assert L.idg_create(C.byref(h), 7, 0) == B.IDG_ERR_ARG
    ctx = B.idg_create(B.IDG_MIXED, 0)
    with pytest.raises(B.IdgError) as e:
        B.idg_set_velocity_grid(ctx, B.IDG_NC_SIMPSON, 32, 32, -4, 4, -4, 4)  # Simpson needs odd n
    assert e.value.status == B.IDG_ERR_ARG
    with pytest.raises(B.IdgError) as e:
        B.idg_set_gas(ctx, 1, -1.0, 0.5, 0.1, 0.5, B.IDG_BGK)
    assert e.value.status == B.IDG_ERR_ARG
    with pytest.raises(B.IdgError) as e:
        B.idg_workspace_size(ctx)  # nothing configured yet
    assert e.value.status == B.IDG_ERR_STATE
    with pytest.raises(B.IdgError) as e:
        B.idg_iterate(ctx, 1, 0.0)
    assert e.value.status == B.IDG_ERR_STATE
    assert "workspace" in B.idg_last_error(ctx)
    # one-sided periodicity is rejected
    p = I.cavity(4, nv=8)
    p.bc[0] = (I.BC_PERIODIC, 0, 0, 0, 0)
    ctx2 = _ctx(p)
    with pytest.raises(B.IdgError) as e:
        B.idg_workspace_size(ctx2)
    assert e.value.status == B.IDG_ERR_ARG
    # checkpoints need a bound context
    for fn in (B.idg_save, B.idg_load):
        with pytest.raises(B.IdgError) as e:
            fn(ctx, "/nonexistent/ckpt.bin")
        assert e.value.status == B.IDG_ERR_STATE
    B.idg_destroy(ctx)
    B.idg_destroy(ctx2)


def test_inverted_cells_are_rejected():
    p = I.cavity(4, nv=8)
    p.nodes_x = p.nodes_x[:, ::-1].copy()
    ctx = _ctx(p)
    with pytest.raises(B.IdgError) as e:
        B.idg_workspace_size(ctx)
    assert "area" in str(e.value)
    B.idg_destroy(ctx)


@pytest.mark.parametrize("n", [8, 28, 60])
def test_library_gauss_hermite_matches_numpy(n):
    p = I.cavity(4, nv=n, vrule=I.GAUSS_HERMITE)
    ctx = _ctx(p)
    N, Nv, nf = B.idg_get_sizes(ctx)
    ux, uy, w = B.idg_velocity_grid(ctx, Nv)
    xr, wr = np.polynomial.hermite.hermgauss(n)
    x = ux[:n]
    wx = w[:n] / w[0] * 1.0
    assert np.allclose(x, xr, rtol=0, atol=1e-12 * max(1, abs(xr).max()))
    # tensor weights: w[k] = w1[kx] w1[ky]; recover w1 from the first row
    w1 = w[:n] / np.sqrt(w[0])
    assert np.allclose(w1 * np.exp(-x * x), wr, rtol=1e-10)
    B.idg_destroy(ctx)


@pytest.mark.parametrize("case", ["couette", "cavity_tanh_gh", "cylinder"])
def test_host_setup_agrees_with_oracle(case):
    from oracle import oracle as O
    if case == "couette":
        p = I.couette(16, nv=16)
    elif case == "cavity_tanh_gh":
        p = I.cavity(12, nv=14, vrule=I.GAUSS_HERMITE, stretch_beta=1.5)
    else:
        p = I.cylinder(ntheta=20, nr=8, nv=11, vmax=6.0)
    o = O.Oracle(p)
    ctx = _ctx(p)
    N, Nv, nf = B.idg_get_sizes(ctx)
    assert (N, Nv, nf) == (o.N, o.Nv, o.nf)
    ux, uy, w = B.idg_velocity_grid(ctx, Nv)
    oux, ouy, ow = o.velocity_grid()
    assert np.allclose(ux, oux, rtol=0, atol=1e-13)
    assert np.allclose(uy, ouy, rtol=0, atol=1e-13)
    assert np.allclose(w, ow, rtol=1e-12)
    assert abs(B.idg_get_dt(ctx) - o.dt) <= 1e-14 * o.dt
    assert B.idg_workspace_size(ctx) > 0
    B.idg_destroy(ctx)


def test_unstructured_mesh_host_checks_and_sizes():
    """Host-side: the setter refuses bad indices; the builder (run by
    idg_workspace_size) refuses a clockwise cell and an edge shared three
    times, and finds the oracle's face count on a triangle mesh."""
    import dataclasses

    from oracle import oracle as O
    from paper_1709_01819_gb300 import binding as B
    from paper_1709_01819_gb300 import inputs as I
    from paper_1709_01819_gb300.solver import configure

    prob = I.tri_cavity(5, nv=4)

    def sizes(p):
        ctx = B.idg_create(B.IDG_MIXED, 0)
        try:
            configure(ctx, p)
            B.idg_workspace_size(ctx)
            return B.idg_get_sizes(ctx)
        finally:
            B.idg_destroy(ctx)

    N, Nv, nf = sizes(prob)
    assert (N, nf) == (O.Oracle(prob).N, O.Oracle(prob).nf) == (50, 85)
    bad = prob.cell_nodes.copy()
    bad[3, :3] = bad[3, 2::-1]
    with pytest.raises(B.IdgError):
        sizes(dataclasses.replace(prob, cell_nodes=bad))
    bad = prob.cell_nodes.copy()
    bad[0, 1] = 10_000
    with pytest.raises(B.IdgError):
        sizes(dataclasses.replace(prob, cell_nodes=bad))


@pytest.mark.parametrize("precision", [B.IDG_FP64, B.IDG_MIXED])
def test_size_limits_and_empty_inputs(precision):
    """The documented limits, at and just past the edge, and empty sizes,
    checked on the host (no device work): a block with min(ni, nj) = 256 plans
    in either precision (float64 with the 2-hyperplane prefetch of the
    macroscopic sweep), 257 is refused; 16384 velocities are accepted, 16512
    refused; zero cells or velocities are refused."""
    ctx = B.idg_create(precision, 0)
    X, Y = I.uniform_nodes(1, 1)
    for ni, nj in ((0, 1), (1, 0)):  # through the C entry: the binding sizes from the arrays
        assert B.lib().idg_set_mesh_structured(ctx, ni, nj, B.dptr(X), B.dptr(Y)) == B.IDG_ERR_ARG
    for nx, ny in ((0, 8), (8, 0), (129, 128)):
        with pytest.raises(B.IdgError) as e:
            B.idg_set_velocity_grid(ctx, B.IDG_NC_TRAP, nx, ny, -4, 4, -4, 4)
        assert e.value.status == B.IDG_ERR_ARG
    B.idg_set_velocity_grid(ctx, B.IDG_NC_TRAP, 128, 128, -4, 4, -4, 4)
    B.idg_destroy(ctx)
    for n, ok in ((256, True), (257, False)):
        p = I.cavity(n, nv=4)
        p.nodes_x, p.nodes_y = I.uniform_nodes(n, n + 3)
        ctx = _ctx(p, precision)
        if ok:
            assert B.idg_workspace_size(ctx) > 0
        else:
            with pytest.raises(B.IdgError) as e:
                B.idg_workspace_size(ctx)
            assert e.value.status == B.IDG_ERR_ARG and "256" in B.idg_last_error(ctx)
        B.idg_destroy(ctx)
