"""The seeded input generators build what their recipes state: sizes by construction and by
Euler's formula, vertices on the surfaces they sample, the same arrays for the same seed."""
import numpy as np

import ttie_inputs as ti


def _euler(m):
    e = ti.edge_list(m.tri)
    return m.V - len(e) + m.F


def test_icosphere_and_octasphere():
    s = ti.icosphere(2)
    assert (s.V, s.F) == (162, 320)
    assert np.allclose(np.linalg.norm(s.x, axis=1), 1.0)
    assert _euler(s) == 2
    for level in (0, 1, 3):
        o = ti.octasphere(level)
        assert o.F == 8 * 4 ** level and o.V == o.F // 2 + 2 and _euler(o) == 2
        assert np.allclose(np.linalg.norm(o.x, axis=1), 1.0)


def test_cloth_sizes_and_seed():
    c = ti.cloth(256, seed=2)
    assert (c.V, c.F) == (65536, 130050)                    # 256^2 vertices, 2 x 255^2 triangles
    assert _euler(ti.cloth(17, seed=2)) == 1                 # a disk
    assert np.array_equal(ti.cloth(17, seed=2).x, ti.cloth(17, seed=2).x)
    assert not np.array_equal(ti.cloth(17, seed=2).x, ti.cloth(17, seed=3).x)
    # the literal construction: x, y on the unit square grid, sheared by the height field only
    lit = ti.cloth(17, seed=2, crossing=False)
    assert lit.x[:, 1].min() == 0.0 and lit.x[:, 1].max() == 1.0


def test_torus_and_ellipsoid():
    t = ti.torus(1.0, 0.3, 16, 8)
    assert (t.V, t.F) == (128, 256) and _euler(t) == 0      # genus one
    rho = np.hypot(t.x[:, 0], t.x[:, 1]) - 1.0
    assert np.allclose(np.hypot(rho, t.x[:, 2]), 0.3)
    ax = np.array([0.7, 1.1, 1.4])
    e = ti.ellipsoid(6, ax)
    assert e.F == 2 * 12 * 5 and _euler(e) == 2              # n_lon = 2 n_lat, F = 2 n_lon (n_lat - 1)
    assert np.allclose(np.sum((e.x / ax) ** 2, axis=1), 1.0)


def test_two_icospheres_groups():
    m = ti.two_icospheres()
    assert m.F == 640 and np.array_equal(np.bincount(m.group), [320, 320])
    assert np.allclose(np.linalg.norm(m.x[:162], axis=1), 1.0)
    assert np.allclose(np.linalg.norm(m.x[162:] - [1.2, 0.0, 0.0], axis=1), 1.0)
