"""Pins of the FP64 oracle to facts fixed by the paper and by the mathematics.

None of these re-types the oracle's formula: each compares it with something
computed another way -- a closed form, an exact integral by a computer-algebra
system, an invariant of the continuous problem that the discrete one inherits,
the paper's own printed counts (Table 1 / Table 2, ``tests/golden``), or brute
force.  ``test_planted_mistakes_are_caught`` compiles deliberately broken copies
of ``oracle.c`` and checks that the same pins reject every one of them.
"""
import ctypes
import itertools
import json
import os
import subprocess

import numpy as np
import pytest

import meshgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- helpers
def brick_corners(F=None, b=None):
    """Brick node coordinates for the map x = F xi + b of the reference cube, node
    order from meshgen's offsets (0/1 per axis -> xi = -1/+1)."""
    xi = 2.0 * meshgen.HEX_NODE_OFFSETS.astype(float) - 1.0
    F = np.eye(3) if F is None else F
    b = np.zeros(3) if b is None else b
    return xi @ F.T + b


def dense_K(ke_dense, npe, X, E, c):
    """Brute-force dense global matrix: add every full k_e into an n x n array."""
    n = X.shape[0]
    K = np.zeros((n, n))
    for e in range(E.shape[0]):
        ke = ke_dense(npe, X[E[e]], c[e])
        for a in range(npe):
            for b in range(npe):
                K[E[e, a], E[e, b]] += ke[a, b]
    return K


def csr_to_dense(n, rowptr, col, vals):
    L = np.zeros((n, n))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            L[i, col[k]] += vals[k]
    return L


def reference_stiffness_integrals():
    """R[i, j, a, b] = exact integral over [-1,1]^3 of dN_a/dxi_i * dN_b/dxi_j, by
    sympy differentiation of the trilinear shape functions and exact monomial
    integration."""
    sp = pytest.importorskip("sympy")
    r, s, t = sp.symbols("r s t")
    xi = 2 * meshgen.HEX_NODE_OFFSETS - 1
    N = [(1 + r * int(p[0])) * (1 + s * int(p[1])) * (1 + t * int(p[2])) / 8 for p in xi]
    grads = [[sp.diff(Na, v) for v in (r, s, t)] for Na in N]

    def integ(expr):
        poly = sp.Poly(sp.expand(expr), r, s, t)
        tot = sp.Rational(0)
        for (i, j, k), coef in poly.terms():
            f = 1
            for p in (i, j, k):
                f *= sp.Rational(2, p + 1) if p % 2 == 0 else 0
            tot += coef * f
        return tot

    R = np.zeros((3, 3, 8, 8))
    for i in range(3):
        for j in range(3):
            for a in range(8):
                for b in range(8):
                    R[i, j, a, b] = float(integ(grads[a][i] * grads[b][j]))
    return R


_R_CACHE = {}


def exact_affine_brick(F, c):
    """k_ab = c |det F| sum_ij (F^-1 F^-T)_ij R_ij(a, b) for x = F xi + b (exact)."""
    if "R" not in _R_CACHE:
        _R_CACHE["R"] = reference_stiffness_integrals()
    R = _R_CACHE["R"]
    Fi = np.linalg.inv(F)
    G = Fi @ Fi.T
    return c * abs(np.linalg.det(F)) * np.einsum("ij,ijab->ab", G, R)


def exact_tet(xe, c):
    """k_ab = c vol grad(lambda_a) . grad(lambda_b) with the barycentric gradients
    read off the inverse of the 4x4 matrix [1, x_a] (textbook P1 element)."""
    A = np.hstack([np.ones((4, 1)), xe])
    grads = np.linalg.inv(A)[1:, :]         # column a = grad lambda_a
    vol = abs(np.linalg.det(A)) / 6.0
    return c * vol * grads.T @ grads


# ------------------------------------------------------------------ the pin suite
def pin_unit_cube(ke_dense):
    """Unit-cube brick: k = c h/12 * {4 (same node), 0 (edge), -1 (face diag), -1 (body diag)}."""
    h, c = 0.37, 2.5
    xe = brick_corners(h / 2 * np.eye(3), np.array([0.3, -1.1, 2.0]))
    k = ke_dense(8, xe, c)
    off = meshgen.HEX_NODE_OFFSETS
    ham = np.abs(off[:, None, :] - off[None, :, :]).sum(-1)
    expect = c * h / 12.0 * np.choose(ham, [4.0, 0.0, -1.0, -1.0])
    return np.abs(k - expect).max() <= 1e-14 * c * h


def pin_affine_bricks(ke_dense):
    """Parallelepipeds: 2x2x2 Gauss is exact; compare with the exact integral."""
    rng = np.random.default_rng(7)
    for _ in range(4):
        F = np.eye(3) * 0.5 + 0.2 * rng.standard_normal((3, 3))
        if np.linalg.det(F) < 0:
            F[:, 0] *= -1
        c = float(np.exp(rng.standard_normal()))
        k = ke_dense(8, brick_corners(F, rng.standard_normal(3)), c)
        ex = exact_affine_brick(F, c)
        if np.abs(k - ex).max() > 1e-13 * np.abs(ex).max():
            return False
    return True


def pin_tets(ke_dense):
    rng = np.random.default_rng(11)
    for _ in range(6):
        xe = rng.standard_normal((4, 3))
        c = float(np.exp(rng.standard_normal()))
        k = ke_dense(4, xe, c)
        ex = exact_tet(xe, c)
        if np.abs(k - ex).max() > 1e-12 * np.abs(ex).max():
            return False
    return True


def pin_patch_and_energy(ke_dense, npe):
    """On a jittered mesh of the unit cube with c = 1 and u = a.x + d:
    K u = 0 at interior nodes (patch test) and u^T K u = |a|^2 * vol(cube) = |a|^2
    (the mesh tiles the cube exactly; 2x2x2 Gauss integrates det J of a
    trilinear map exactly)."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(3, 3, 2, jitter=0.25, seed=99, c_law="one", permute_nodes=True)
    K = dense_K(ke_dense, npe, m.X, m.E, m.c)
    a = np.array([0.7, -1.3, 0.4])
    u = m.X @ a + 0.9
    Ku = K @ u
    interior = ((m.X > 1e-12) & (m.X < 1 - 1e-12)).all(axis=1)
    ok_patch = np.abs(Ku[interior]).max() <= 1e-12 * np.abs(K).max()
    ok_energy = abs(u @ K @ u - a @ a) <= 1e-12 * (a @ a)
    ok_rowsum = np.abs(K.sum(axis=1)).max() <= 1e-12 * np.abs(K).max()
    return bool(ok_patch and ok_energy and ok_rowsum)


def run_pins(ke_dense):
    return dict(unit_cube=pin_unit_cube(ke_dense), affine=pin_affine_bricks(ke_dense),
                tets=pin_tets(ke_dense), patch_hex=pin_patch_and_energy(ke_dense, 8),
                patch_tet=pin_patch_and_energy(ke_dense, 4))


# ----------------------------------------------------------------------- the tests
def test_unit_cube_closed_form(oracle_lib):
    assert pin_unit_cube(oracle_lib.ke_dense)


def test_affine_bricks_exact_integral(oracle_lib):
    assert pin_affine_bricks(oracle_lib.ke_dense)


def test_tet_closed_form(oracle_lib):
    assert pin_tets(oracle_lib.ke_dense)


@pytest.mark.parametrize("npe", [8, 4])
def test_patch_energy_rowsum(oracle_lib, npe):
    assert pin_patch_and_energy(oracle_lib.ke_dense, npe)


def test_trilinear_brick_high_precision():
    """A non-affine brick against a 40-digit evaluation of Eq. 9 whose shape-function
    derivatives come from sympy differentiation (not from the oracle's table)."""
    sp = pytest.importorskip("sympy")
    import mpmath as mp
    import oracle
    mp.mp.dps = 40
    r, s, t = sp.symbols("r s t")
    xi = 2 * meshgen.HEX_NODE_OFFSETS - 1
    N = [(1 + r * int(p[0])) * (1 + s * int(p[1])) * (1 + t * int(p[2])) / 8 for p in xi]
    dN = sp.lambdify((r, s, t), sp.Matrix([[sp.diff(Na, v) for Na in N] for v in (r, s, t)]), "mpmath")
    rng = np.random.default_rng(5)
    xe = brick_corners() * 0.5 + 0.12 * rng.standard_normal((8, 3))
    c = 1.7
    k = mp.zeros(8, 8)
    g = 1 / mp.sqrt(3)
    Xe = mp.matrix(xe.tolist())
    for pr, ps, pt in itertools.product((-g, g), repeat=3):
        D = mp.matrix(dN(pr, ps, pt))
        J = D * Xe
        B = mp.inverse(J) * D
        k += c * abs(mp.det(J)) * B.T * B
    ref = np.array(k.tolist(), dtype=float)
    got = oracle.ke_dense(8, xe, c)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_symmetry_and_psd(oracle_lib):
    rng = np.random.default_rng(3)
    for npe in (8, 4):
        xe = (brick_corners() * 0.5 if npe == 8 else np.eye(4, 3)) + 0.1 * rng.standard_normal((npe, 3))
        k = oracle_lib.ke_dense(npe, xe, 1.3)
        assert np.abs(k - k.T).max() <= 1e-15 * np.abs(k).max()
        w = np.linalg.eigvalsh(k)
        assert w.min() >= -1e-13 * w.max()
        assert np.sum(w > 1e-10 * w.max()) == npe - 1      # kernel = constants


def test_nnz_matches_table1_and_closed_form(oracle_lib):
    """Table 1's NNZ in CSC (lower triangle) for n = 10, 20, 40 and the triplet
    count 36 * n_elems; the closed form ((3n+1)^3 + (n+1)^3) / 2 reproduces every
    column of the table; Table 2's matrix sizes are (n+1)^3."""
    t1 = json.load(open(os.path.join(GOLDEN, "table1_nnz.json")))
    t2 = json.load(open(os.path.join(GOLDEN, "table2_sizes.json")))
    for ne, nt, nc in zip(t1["n_elems"], t1["nnz_triplet"], t1["nnz_csc"]):
        n = round(ne ** (1 / 3))
        assert n ** 3 == ne and nt == 36 * ne
        assert ((3 * n + 1) ** 3 + (n + 1) ** 3) // 2 == nc
    for ne, ms in zip(t2["n_elems"], t2["matrix_size"]):
        n = round(ne ** (1 / 3))
        assert (n + 1) ** 3 == ms
    for n, nc in zip((10, 20, 40), t1["nnz_csc"][:3]):
        m = meshgen.hex_grid(n, jitter=0.2, seed=n, permute_nodes=True, permute_elems=True)
        K = oracle_lib.build_K(8, m.X, m.E, m.c)
        assert K["nnz"] == nc
        assert K["rowptr"][-1] == nc and len(K["slot"]) == 36 * n ** 3


def test_table1_memory_formula():
    """Table 1's memory rows follow 16 B per triplet and 16 B per CSC nonzero plus
    8 B per column pointer (a check of how the table is read, not of K)."""
    t1 = json.load(open(os.path.join(GOLDEN, "table1_nnz.json")))
    for ne, nt, nc, mt, mc in zip(t1["n_elems"], t1["nnz_triplet"], t1["nnz_csc"],
                                  t1["mem_triplet_MB"], t1["mem_csc_MB"]):
        n = round(ne ** (1 / 3))
        assert abs(nt * 16 / 1e6 - mt) <= 0.006 * mt + 0.01
        assert abs((nc * 16 + ((n + 1) ** 3 + 1) * 8) / 1e6 - mc) <= 0.006 * mc + 0.01


@pytest.mark.parametrize("n", [1, 3, 10])
def test_kuhn_nnz_closed_form(oracle_lib, n):
    """Kuhn split: each node couples with itself, 3 axis edges, 3 face diagonals
    and one body diagonal per cell: nnz = N + 3n(n+1)^2 + 3n^2(n+1) + n^3."""
    m = meshgen.kuhn_tets(n, jitter=0.2, seed=n, permute_nodes=True, permute_elems=True)
    K = oracle_lib.build_K(4, m.X, m.E, m.c)
    assert K["nnz"] == (n + 1) ** 3 + 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3


@pytest.mark.parametrize("shape,npe", [((1, 1, 1), 8), ((2, 1, 1), 8), ((2, 2, 2), 8), ((2, 2, 1), 4)])
def test_brute_force_dense(oracle_lib, shape, npe):
    """CSR -> dense equals tril of the brute-force dense sum of full k_e."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(*shape, jitter=0.2, seed=4, permute_nodes=True, permute_elems=True)
    K = oracle_lib.build_K(npe, m.X, m.E, m.c)
    L = csr_to_dense(m.n_nodes, K["rowptr"], K["col"], K["vals"])
    D = dense_K(oracle_lib.ke_dense, npe, m.X, m.E, m.c)
    assert np.abs(L - np.tril(D)).max() <= 1e-14 * np.abs(D).max()
    # columns ascending and unique within each row, diagonal last
    for i in range(m.n_nodes):
        cols = K["col"][K["rowptr"][i]:K["rowptr"][i + 1]]
        assert np.all(np.diff(cols) > 0) and cols[-1] == i


def test_permutation_covariance(oracle_lib):
    """Renumbering nodes and elements permutes K and changes nothing else."""
    base = meshgen.hex_grid(5, 4, 3, jitter=0.2, seed=21)
    perm = meshgen.hex_grid(5, 4, 3, jitter=0.2, seed=21, permute_nodes=True, permute_elems=True)
    p = meshgen.stream_permutation(21, "node_perm", base.n_nodes)   # new id of old node
    Kb = oracle_lib.build_K(8, base.X, base.E, base.c)
    Kp = oracle_lib.build_K(8, perm.X, perm.E, perm.c)
    assert Kb["nnz"] == Kp["nnz"]
    Db = csr_to_dense(base.n_nodes, Kb["rowptr"], Kb["col"], Kb["vals"])
    Dp = csr_to_dense(perm.n_nodes, Kp["rowptr"], Kp["col"], Kp["vals"])
    Db, Dp = Db + np.tril(Db, -1).T, Dp + np.tril(Dp, -1).T
    assert np.abs(Dp[np.ix_(p, p)] - Db).max() <= 1e-14 * np.abs(Db).max()


def test_gradient_complex_step_vs_central_differences(oracle_lib):
    """The oracle's VJP of L = sum G_ij K_ij against central differences of the
    oracle's own K in X and c (two independent derivatives of one function)."""
    for npe, gen in ((8, meshgen.hex_grid), (4, meshgen.kuhn_tets)):
        m = gen(2, 2, 2, jitter=0.2, seed=8, permute_nodes=True)
        K = oracle_lib.build_K(npe, m.X, m.E, m.c)
        G = np.random.default_rng(1).standard_normal(K["nnz"])
        dX, dc = oracle_lib.vjp_from_G(npe, m.X, m.E, m.c, G, K["slot"])

        def L(X, c):
            return float(G @ oracle_lib.build_K(npe, X, m.E, c)["vals"])

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


# ----------------------------------------------------- planted mistakes must be caught
MUTATIONS = {
    "transposed_inverse": ("acc += inv[i][k] * dN[k][a];", "acc += inv[k][i] * dN[k][a];"),
    "missing_jacobian": ("T absdet = RE(det) < 0 ? -det : det;", "T absdet = RE(det) < 0 ? -1.0 : 1.0;"),
    "gauss_point": ("const double g = 1.0 / sqrt(3.0);", "const double g = 0.5;"),
    "dN_index": ("dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);",
                 "dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + s * ta);"),
    "cofactor_sign": ("T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];",
                      "T c01 = J[1][0] * J[2][2] - J[1][2] * J[2][0];"),
    "tet_volume": ("T vol = (RE(det) < 0 ? -det : det) / 6.0;", "T vol = (RE(det) < 0 ? -det : det) / 2.0;"),
    "tet_gradient": ("static const double TET_DL[3][4] = {{-1, 1, 0, 0}, {-1, 0, 1, 0}, {-1, 0, 0, 1}};",
                     "static const double TET_DL[3][4] = {{-1, 1, 0, 0}, {-1, 0, 1, 0}, {0, 0, 0, 1}};"),
    "dropped_term": ("for (int i = 0; i < 3; ++i) acc += B[i][a] * B[i][b];",
                     "for (int i = 0; i < 2; ++i) acc += B[i][a] * B[i][b];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(tmp_path, name):
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

    def ke_dense(npe, xe, c):
        xe = np.ascontiguousarray(xe, dtype=np.float64)
        ke = np.zeros((npe, npe))
        L.oracle_ke_dense(0, npe, xe.ctypes.data_as(ctypes.c_void_p), float(c), ke.ctypes.data_as(ctypes.c_void_p))
        return ke

    res = run_pins(ke_dense)
    assert not all(res.values()), f"mutation {name} passed every pin: {res}"
