"""The synthetic inputs against the recipes they are stated with: the seeded
64-cavity batch, the O-grid radii and spacing, the tanh stretching, the
unstructured variants' cell counts and the hypersonic free stream."""
import math

import numpy as np

from paper_1709_01819_gb300 import inputs as I


def test_batch_of_64_cavities_follows_its_recipe_and_seed():
    a, b = I.batch_c4(), I.batch_c4()
    assert len(a) == 64
    key = [(p.Kn, p.bc[3][2], p.ni) for p in a]
    assert key == [(p.Kn, p.bc[3][2], p.ni) for p in b]  # the seed fixes the draw
    kn = np.array([k[0] for k in key])
    U = np.array([k[1] for k in key])
    n = np.array([k[2] for k in key])
    assert kn.min() >= 1e-3 and kn.max() <= 10.0 and kn.min() < 1e-2 and kn.max() > 1.0
    assert U.min() >= 0.05 and U.max() <= 0.3
    assert set(n) == {32, 48, 64, 96}
    assert all(p.nvx == p.nvy == 32 and p.ni == p.nj for p in a)
    assert [p.Kn for p in I.batch_c4(seed=1)] != list(kn)


def test_ogrid_radii_spacing_and_closure():
    X, Y = I.ogrid_nodes(121, 81)
    r = np.hypot(X, Y)
    q = 1.05
    rj = 1.0 + 14.0 * (q ** np.arange(82) - 1.0) / (q ** 81 - 1.0)
    assert np.abs(r - rj[:, None]).max() <= 1e-12 * 15.0
    assert abs((rj[1] - 1.0) - 0.0137) < 1e-4  # first radial spacing ~0.0137 R
    assert abs(r[-1].max() - 15.0) < 1e-12
    assert np.array_equal(X[:, -1], X[:, 0]) and np.array_equal(Y[:, -1], Y[:, 0])


def test_tanh_stretching_min_to_max_spacing_is_a_tenth():
    c = I.tanh_coords(128, I.C3_BETA)
    d = np.diff(c)
    assert abs(c[0]) < 1e-15 and abs(c[-1] - 1.0) < 1e-15
    assert np.allclose(d, d[::-1], rtol=0, atol=1e-15)
    assert abs(d.min() / d.max() - 0.100) < 5e-4


def test_unstructured_variants_cell_counts():
    assert I.tri_cavity(16).cell_nodes.shape[0] == 2 * 16 * 16
    h = I.hybrid_cylinder(ntheta=121, nr=81, nr_quad=41)
    assert h.cell_nodes.shape[0] == 121 * 41 + 2 * 121 * 40 == 14641
    quads = int(np.sum(h.cell_nodes[:, 3] >= 0))
    assert quads == 121 * 41


def test_hypersonic_free_stream():
    p = I.cylinder_c5()
    kinds = [b[0] for b in p.bc]
    far = p.bc[kinds.index(I.BC_FARFIELD)]
    gamma = 5.0 / 3.0  # K = 1
    assert abs(far[2] - 5.0 * math.sqrt(gamma * 0.5)) < 1e-12  # Ma 5 at R T = 1/2
    assert abs(far[2] - 4.564) < 1e-3
    assert p.nvx == p.nvy == 89 and p.vrange == (-15.0, 15.0, -15.0, 15.0)
