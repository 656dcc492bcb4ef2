"""Pins of the oracle's load vector, F_n = sum_e s_e * integral N_a (Section 1, steps
(ii)-(iii): local load vectors f_e assembled into F).

The references are:
- closed forms for single elements;
- the identity F = M 1 when s = c (the shape functions sum to one), checked against
  the mass operator, which is separate code with its own pins;
- the total source.

Planted mistakes must each fail at least one pin.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import meshgen


def single(load, npe, xe, s):
    E = np.arange(npe, dtype=np.int32)[None, :]
    return load(npe, np.asarray(xe, float), E, np.array([s], float))


def brick_corners(F=None, b=None):
    xi = 2.0 * meshgen.HEX_NODE_OFFSETS.astype(float) - 1.0
    F = np.eye(3) if F is None else F
    b = np.zeros(3) if b is None else b
    return xi @ F.T + b


def pin_single_elements(load):
    """Parallelepiped (affine brick): every node gets s vol / 8. Tetrahedron: s |T| / 4."""
    rng = np.random.default_rng(41)
    for _ in range(4):
        F = np.eye(3) * 0.5 + 0.2 * rng.standard_normal((3, 3))
        s = float(np.exp(rng.standard_normal()))
        f = single(load, 8, brick_corners(F, rng.standard_normal(3)), s)
        vol = 8.0 * abs(np.linalg.det(F))
        if np.abs(f - s * vol / 8).max() > 1e-13 * s * vol:
            return False
        xe = rng.standard_normal((4, 3))
        V = abs(np.linalg.det(xe[1:] - xe[0])) / 6.0
        f = single(load, 4, xe, s)
        if np.abs(f - s * V / 4).max() > 1e-13 * s * V:
            return False
    return True


def pin_equals_mass_times_one(load, oracle_lib, npe):
    """With s = c: F = M 1 exactly (sum_b N_b = 1 under the integral), against the
    oracle's assembled mass matrix."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(3, 2, 2, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True)
    F = load(npe, m.X, m.E, m.c)
    M = oracle_lib.build_K(npe, m.X, m.E, m.c, op="mass")
    rp, col, v = M["rowptr"], M["col"], M["vals"]
    Mu = np.zeros(m.n_nodes)
    for i in range(m.n_nodes):
        for k in range(rp[i], rp[i + 1]):
            Mu[i] += v[k]
            if col[k] != i:
                Mu[col[k]] += v[k]
    return np.abs(F - Mu).max() <= 1e-13 * np.abs(Mu).max()


def pin_total(load, npe):
    """The tiled unit cube with s = 1: sum F = 1."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(4, 3, 2, jitter=0.3, seed=9, c_law="one", permute_nodes=True)
    return abs(load(npe, m.X, m.E, np.ones(m.E.shape[0])).sum() - 1.0) <= 1e-13


def run_pins(load, oracle_lib):
    return dict(single=pin_single_elements(load), mass_hex=pin_equals_mass_times_one(load, oracle_lib, 8),
                mass_tet=pin_equals_mass_times_one(load, oracle_lib, 4), total_hex=pin_total(load, 8),
                total_tet=pin_total(load, 4))


def test_load_single_elements(oracle_lib):
    assert pin_single_elements(oracle_lib.load_vector)


@pytest.mark.parametrize("npe", [8, 4])
def test_load_equals_mass_times_one(oracle_lib, npe):
    assert pin_equals_mass_times_one(oracle_lib.load_vector, oracle_lib, npe)


@pytest.mark.parametrize("npe", [8, 4])
def test_load_total(oracle_lib, npe):
    assert pin_total(oracle_lib.load_vector, npe)


MUTATIONS = {
    "tet_share": ("fe[a] += src[e] * (vol / 4.0) * (a == q ? qa : qb);", "fe[a] += src[e] * (vol / 3.0) * (a == q ? qa : qb);"),
    "brick_no_jacobian": ("for (int a = 0; a < 8; ++a) fe[a] += src[e] * fabs(det) * N[a];",
                          "for (int a = 0; a < 8; ++a) fe[a] += src[e] * N[a];"),
    "brick_shape_index": ("for (int a = 0; a < 8; ++a) fe[a] += src[e] * fabs(det) * N[a];",
                          "for (int a = 0; a < 8; ++a) fe[a] += src[e] * fabs(det) * N[7 - a];"),
    "wrong_node": ("for (int a = 0; a < npe; ++a) F[E[e * npe + a]] += fe[a];",
                   "for (int a = 0; a < npe; ++a) F[E[e * npe + (a + 1) % npe]] += fe[a];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_load_planted_mistakes_are_caught(tmp_path, oracle_lib, name):
    src = open(os.path.join(os.path.dirname(oracle_lib.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    L = ctypes.CDLL(str(so))
    L.oracle_load.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 4
    L.oracle_load.restype = ctypes.c_int64

    def load(npe, X, E, s):
        X = np.ascontiguousarray(X, np.float64)
        E = np.ascontiguousarray(E, np.int32)
        s = np.ascontiguousarray(s, np.float64)
        F = np.zeros(X.shape[0])
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        L.oracle_load(npe, E.shape[0], p(E), p(X), p(s), p(F))
        return F

    res = run_pins(load, oracle_lib)
    assert not all(res.values()), f"mutation {name} passed every pin: {res}"


@pytest.mark.parametrize("npe", [8, 4])
def test_body_force_load_components(oracle_lib, npe):
    """The elasticity operator's load of a body force b_e: component i of F is the
    scalar load of b_e,i, so a uniform force on the tiled unit cube totals b, and
    its components sit at DOFs 3n + i."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(3, 2, 2, jitter=0.3, seed=6, c_law="one", permute_nodes=True)
    bvec = np.array([0.5, -2.0, 1.25])
    F = oracle_lib.load_vector(npe, m.X, m.E, np.tile(bvec, (m.n_elems, 1)))
    assert F.shape == (3 * m.n_nodes,)
    assert np.allclose(F.reshape(-1, 3).sum(axis=0), bvec, rtol=0, atol=1e-13)
    w = oracle_lib.load_vector(npe, m.X, m.E, np.ones(m.n_elems))
    assert np.allclose(F.reshape(-1, 3), np.outer(w, bvec), rtol=0, atol=1e-15)
