"""The seeded generator: reproducible, valid meshes of the stated shapes."""
import numpy as np

import meshgen


def test_streams_are_counter_based():
    a = meshgen.stream_u64(5, "x", 10)
    b = meshgen.stream_u64(5, "x", 4, offset=6)
    assert np.array_equal(a[6:], b)
    assert not np.array_equal(a, meshgen.stream_u64(6, "x", 10))
    u = meshgen.stream_uniform(1, "u", 100000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_hex_grid_shapes_and_boundary():
    m = meshgen.hex_grid(4, 3, 2, jitter=0.25, seed=3, permute_nodes=True, permute_elems=True)
    assert m.X.shape == (5 * 4 * 3, 3) and m.E.shape == (24, 8) and m.E.dtype == np.int32
    assert sorted(np.unique(m.E)) == list(range(m.n_nodes))
    assert all(len(set(row)) == 8 for row in m.E.tolist())
    # boundary nodes stay on the cube faces, so the mesh tiles the unit cube
    onface = (np.isclose(m.X, 0) | np.isclose(m.X, 1)).any(axis=1)
    assert onface.sum() == 5 * 4 * 3 - 3 * 2 * 1
    assert m.X.min() >= 0 and m.X.max() <= 1


def test_reproducible():
    a = meshgen.config_mesh(0)
    b = meshgen.config_mesh(0)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.E, b.E) and np.array_equal(a.c, b.c)
    assert a.n_elems == 8000 and a.n_nodes == 9261


def test_kuhn_tets_orientation():
    m = meshgen.kuhn_tets(3, jitter=0.0)
    x = m.X[m.E]
    det = np.linalg.det(x[:, 1:] - x[:, :1])
    assert np.allclose(det, 1.0 / 27)          # 6 tets of volume h^3/6 per cell, all positive


def test_batch_specs_range():
    specs = meshgen.batch_specs()
    assert len(specs) == 512
    arr = np.array(specs)
    assert arr.min() >= 10 and arr.max() <= 60
    tot = int(np.prod(arr, axis=1).sum())
    assert 1.2e7 < tot < 2.6e7
