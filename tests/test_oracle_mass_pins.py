"""Pins of the oracle's mass operator, M_ab = integral c N_a N_b (the other
operator the paper says its construction generalises to, Section 5).

As for the stiffness pins, none re-types the oracle's formula. The references are:
- a closed form built from the node offsets (not from the oracle's tables);
- the affine scaling law;
- the classical integral of products of barycentric coordinates;
- an exact sympy integral of det J over the reference cube;
- invariants of the continuous operator.

Planted mistakes in a copy of ``oracle.c`` must each fail at least one of them.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import meshgen


def brick_corners(F=None, b=None):
    xi = 2.0 * meshgen.HEX_NODE_OFFSETS.astype(float) - 1.0
    F = np.eye(3) if F is None else F
    b = np.zeros(3) if b is None else b
    return xi @ F.T + b


def unit_cube_mass(h, c):
    """Cube of edge h: M_ab = c h^3 / 216 * 2^(3 - d_ab), d_ab = number of axes on
    which nodes a and b differ (the 1D mass matrix h/6 [2 1; 1 2] in each axis)."""
    off = meshgen.HEX_NODE_OFFSETS
    d = np.abs(off[:, None, :] - off[None, :, :]).sum(-1)
    return c * h ** 3 / 216.0 * 2.0 ** (3 - d)


def pin_unit_cube(me):
    h, c = 0.37, 2.5
    m = me(8, brick_corners(h / 2 * np.eye(3), np.array([0.3, -1.1, 2.0])), c)
    ex = unit_cube_mass(h, c)
    return np.abs(m - ex).max() <= 1e-14 * ex.max()


def pin_affine_bricks(me):
    """x = F xi + b: N_a N_b |det J| is a polynomial of degree <= 2 per axis, so the
    2x2x2 rule is exact and M = |det F| / (h^3 / 8) times the cube's matrix."""
    rng = np.random.default_rng(17)
    for _ in range(4):
        F = np.eye(3) * 0.5 + 0.2 * rng.standard_normal((3, 3))
        c = float(np.exp(rng.standard_normal()))
        m = me(8, brick_corners(F, rng.standard_normal(3)), c)
        ex = unit_cube_mass(2.0, c) * abs(np.linalg.det(F))
        if np.abs(m - ex).max() > 1e-13 * ex.max():
            return False
    return True


def pin_tets(me):
    """Linear tetrahedron: integral lambda_a lambda_b = V (1 + delta_ab) / 20."""
    rng = np.random.default_rng(23)
    for _ in range(6):
        xe = rng.standard_normal((4, 3))
        c = float(np.exp(rng.standard_normal()))
        V = abs(np.linalg.det((xe[1:] - xe[0]))) / 6.0
        ex = c * V / 20.0 * (np.ones((4, 4)) + np.eye(4))
        if np.abs(me(4, xe, c) - ex).max() > 1e-13 * ex.max():
            return False
    return True


def pin_total_mass(me, npe):
    """Jittered mesh of the unit cube, c = 1: the mesh tiles the cube, so u^T M u
    for u = 1 is the volume 1. Every element matrix is symmetric positive definite."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(3, 3, 2, jitter=0.25, seed=99, c_law="one", permute_nodes=True)
    total, ok = 0.0, True
    for e in range(m.E.shape[0]):
        M = me(npe, m.X[m.E[e]], 1.0)
        total += M.sum()
        ok &= np.allclose(M, M.T, rtol=0, atol=1e-15 * np.abs(M).max())
        ok &= np.linalg.eigvalsh(M).min() > 0
    return bool(ok and abs(total - 1.0) <= 1e-13)


def pin_trilinear_volume(me):
    """A non-affine brick: sum_ab M_ab = c * volume, the volume being the exact
    integral of det J over the reference cube, by sympy on the trilinear map."""
    sp = pytest.importorskip("sympy")
    r, s, t = sp.symbols("r s t")
    xi = 2 * meshgen.HEX_NODE_OFFSETS - 1
    rng = np.random.default_rng(29)
    xe = brick_corners() * 0.5 + 0.12 * rng.standard_normal((8, 3))
    N = [(1 + r * int(p[0])) * (1 + s * int(p[1])) * (1 + t * int(p[2])) / 8 for p in xi]
    x = [sum(sp.Rational(float(xe[a, j])) * N[a] for a in range(8)) for j in range(3)]
    J = sp.Matrix([[sp.diff(x[j], v) for j in range(3)] for v in (r, s, t)])
    vol = sp.integrate(sp.expand(J.det()), (r, -1, 1), (s, -1, 1), (t, -1, 1))
    c = 1.3
    return abs(me(8, xe, c).sum() - c * float(vol)) <= 1e-13 * c * float(vol)


def run_pins(me):
    return dict(unit_cube=pin_unit_cube(me), affine=pin_affine_bricks(me), tets=pin_tets(me),
                total_hex=pin_total_mass(me, 8), total_tet=pin_total_mass(me, 4))


def mass_of(oracle_lib):
    return lambda npe, xe, c: oracle_lib.ke_dense(npe, xe, c, op="mass")


def test_mass_unit_cube_closed_form(oracle_lib):
    assert pin_unit_cube(mass_of(oracle_lib))


def test_mass_affine_bricks(oracle_lib):
    assert pin_affine_bricks(mass_of(oracle_lib))


def test_mass_tet_closed_form(oracle_lib):
    assert pin_tets(mass_of(oracle_lib))


@pytest.mark.parametrize("npe", [8, 4])
def test_mass_total_and_spd(oracle_lib, npe):
    assert pin_total_mass(mass_of(oracle_lib), npe)


def test_mass_trilinear_volume(oracle_lib):
    assert pin_trilinear_volume(mass_of(oracle_lib))


def test_mass_assembled_total(oracle_lib):
    """The assembled lower CSR M: the full matrix's sum (2 * lower - diagonal) is c * volume."""
    m = meshgen.hex_grid(4, 3, 3, jitter=0.25, seed=3, c_law="one", permute_nodes=True, permute_elems=True)
    out = oracle_lib.build_K(8, m.X, m.E, m.c, op="mass")
    rp, col, v = out["rowptr"], out["col"], out["vals"]
    diag = sum(v[k] for i in range(m.n_nodes) for k in range(rp[i], rp[i + 1]) if col[k] == i)
    assert abs(2 * v.sum() - diag - 1.0) <= 1e-13


MUTATIONS = {
    "tet_rule_points": ("lam[a] = a == q ? qa : qb;", "lam[a] = a == q ? qb : qa;"),
    "tet_weight": ("me[4 * a + b] += c * (vol / 4.0) * lam[a] * lam[b];",
                   "me[4 * a + b] += c * (vol / 6.0) * lam[a] * lam[b];"),
    "brick_shape_index": ("N[a] = 0.125 * (1 + r * ra) * (1 + s * sa) * (1 + t * ta);",
                          "N[a] = 0.125 * (1 + r * ra) * (1 + s * ra) * (1 + t * ta);"),
    "brick_no_jacobian": ("me[8 * a + b] += c * absdet * N[a] * N[b];", "me[8 * a + b] += c * N[a] * N[b];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mass_planted_mistakes_are_caught(tmp_path, name):
    import oracle
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    L = ctypes.CDLL(str(so))
    L.oracle_ke_dense.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]

    def me(npe, xe, c):
        xe = np.ascontiguousarray(xe, dtype=np.float64)
        m = np.zeros((npe, npe))
        L.oracle_ke_dense(1, npe, xe.ctypes.data_as(ctypes.c_void_p), float(c), m.ctypes.data_as(ctypes.c_void_p))
        return m

    res = run_pins(me)
    assert not all(res.values()), f"mutation {name} passed every pin: {res}"


def test_mass_gradient_complex_step_vs_central_differences(oracle_lib):
    """The oracle's gradient of L = sum G_ij M_ij (complex step of its mass routine)
    against central differences of its real mass matrix, in X and c."""
    for npe, gen in ((8, meshgen.hex_grid), (4, meshgen.kuhn_tets)):
        m = gen(2, 2, 2, jitter=0.2, seed=8, permute_nodes=True)
        M = oracle_lib.build_K(npe, m.X, m.E, m.c, op="mass")
        G = np.random.default_rng(2).standard_normal(M["nnz"])
        dX, dc = oracle_lib.vjp_from_G(npe, m.X, m.E, m.c, G, M["slot"], op="mass")

        def L(X, c):
            return float(G @ oracle_lib.build_K(npe, X, m.E, c, op="mass")["vals"])

        h = 1e-6
        fd = np.zeros_like(m.X)
        for i in range(m.n_nodes):
            for j in range(3):
                Xp, Xm = m.X.copy(), m.X.copy()
                Xp[i, j] += h
                Xm[i, j] -= h
                fd[i, j] = (L(Xp, m.c) - L(Xm, m.c)) / (2 * h)
        assert np.abs(dX - fd).max() <= 1e-6 * np.abs(fd).max()
        fdc = np.array([(L(m.X, m.c + h * (np.arange(m.n_elems) == e)) -
                         L(m.X, m.c - h * (np.arange(m.n_elems) == e))) / (2 * h)
                        for e in range(m.n_elems)])
        assert np.abs(dc - fdc).max() <= 1e-6 * np.abs(fdc).max()
