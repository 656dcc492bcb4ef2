"""Pins of the oracle's elasticity operator: three DOFs per node (Algorithm 1's
DOFxn), k_e = integral Be^T D Be with the Lame parameters (lambda_e, mu_e).

None re-types the oracle's Voigt formulation.  The references are:
- the strain-energy route: W(u) = integral lambda/2 (tr eps)^2 + mu eps:eps with
  eps = sym(grad u), grad u = (du/dxi)(dx/dxi)^-1, the xi-derivatives of the
  interpolated fields taken by the complex step of the shape functions N (not of
  any derivative formula), and k_AB recovered by polarisation,
  W(e_A + e_B) - W(e_A) - W(e_B); on affine bricks with an exact 3x3x3 rule;
- rigid-body motions, which must lie in the null space of every k_e;
- the block trace identity sum_i K[3a+i, 3b+i] = (lambda + 4 mu) k_ab against
  the scalar operator of Eq. 9, which has its own pins;
- the patch test and the total strain energy of an affine displacement on a
  jittered mesh of the unit cube, through the assembled 3N x 3N matrix;
- rotation covariance of k_e.

Planted mistakes in a copy of ``oracle.c`` must each fail at least one pin.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import meshgen

SIGN = 2.0 * meshgen.HEX_NODE_OFFSETS.astype(float) - 1.0


def shape_hex(xi):
    """N_a(xi) of the trilinear brick, for real or complex xi [3]."""
    return np.prod((1.0 + SIGN * xi[None, :]) / 2.0, axis=1)


def shape_tet(xi):
    return np.array([1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]], dtype=complex)


def dshape(shape, xi):
    """dN_a/dxi_i [npe, 3] by the complex step of N itself."""
    h = 1e-30
    cols = []
    for i in range(3):
        z = xi.astype(complex)
        z[i] += 1j * h
        cols.append(np.imag(shape(z)) / h)
    return np.stack(cols, axis=1)


def energy_stiffness(npe, xe, lam, mu, rule):
    """k_e by polarisation of the strain energy, summed over quadrature points."""
    shape = shape_hex if npe == 8 else shape_tet
    nk = 3 * npe
    K = np.zeros((nk, nk))
    for xi, w in rule:
        dN = dshape(shape, np.asarray(xi, float))       # [npe, 3] d N / d xi
        dx = xe.T @ dN                                   # dx_i / dxi_j
        detJ = abs(np.linalg.det(dx))
        inv = np.linalg.inv(dx)

        def W(u):
            H = u.reshape(npe, 3).T @ dN @ inv           # du_i / dx_j
            eps = 0.5 * (H + H.T)
            return w * detJ * (0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps))

        We = np.array([W(np.eye(nk)[A]) for A in range(nk)])
        for A in range(nk):
            for B in range(A + 1):
                u = np.zeros(nk)
                u[A] += 1.0
                u[B] += 1.0
                K[A, B] += W(u) - We[A] - We[B] if A != B else 2.0 * We[A]
    return np.tril(K) + np.tril(K, -1).T


def gauss_rule(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return [((a, b, c), wa * wb * wc) for a, wa in zip(x, w) for b, wb in zip(x, w) for c, wc in zip(x, w)]


TET_RULE = [((0.25, 0.25, 0.25), 1.0 / 6.0)]


def brick_corners(F=None, b=None):
    F = np.eye(3) if F is None else F
    b = np.zeros(3) if b is None else b
    return SIGN @ F.T + b


def random_brick(rng, affine):
    F = np.eye(3) * 0.5 + 0.15 * rng.standard_normal((3, 3))
    xe = brick_corners(F, rng.standard_normal(3))
    if not affine:
        xe = xe + 0.08 * rng.standard_normal((8, 3))
    return xe


def random_tet(rng):
    while True:
        xe = rng.standard_normal((4, 3))
        if np.linalg.det(xe[1:] - xe[0]) > 0.05:
            return xe


def random_lame(rng):
    mu = float(np.exp(rng.standard_normal()))
    return float(mu * rng.uniform(0.2, 3.0)), mu


def close(A, B, tol):
    return np.abs(A - B).max() <= tol * np.abs(B).max()


def pin_energy_affine_bricks(ke_el):
    rng = np.random.default_rng(101)
    rule = gauss_rule(3)  # exact: the integrand is a polynomial of degree <= 2 per axis
    for _ in range(2):
        xe = random_brick(rng, affine=True)
        lam, mu = random_lame(rng)
        if not close(ke_el(8, xe, lam, mu), energy_stiffness(8, xe, lam, mu, rule), 1e-12):
            return False
    return True


def pin_energy_distorted_brick(ke_el):
    """Non-affine brick: the 2x2x2 rule of Eq. 9 is the definition; the energy
    route with the same rule must agree."""
    rng = np.random.default_rng(102)
    xe = random_brick(rng, affine=False)
    lam, mu = random_lame(rng)
    return close(ke_el(8, xe, lam, mu), energy_stiffness(8, xe, lam, mu, gauss_rule(2)), 1e-12)


def pin_energy_tets(ke_el):
    rng = np.random.default_rng(103)
    for _ in range(3):
        xe = random_tet(rng)
        lam, mu = random_lame(rng)
        if not close(ke_el(4, xe, lam, mu), energy_stiffness(4, xe, lam, mu, TET_RULE), 1e-12):
            return False
    return True


def rigid_modes(xe):
    """6 rigid-body motions of the nodes xe: translations and u = w x (x - x0)."""
    n = xe.shape[0]
    modes = []
    for i in range(3):
        u = np.zeros((n, 3))
        u[:, i] = 1.0
        modes.append(u.ravel())
    x = xe - xe.mean(axis=0)
    for i in range(3):
        w = np.zeros(3)
        w[i] = 1.0
        modes.append(np.cross(w, x).ravel())
    return np.stack(modes, axis=1)


def pin_rigid_modes(ke_el):
    rng = np.random.default_rng(104)
    for npe in (8, 4):
        for _ in range(3):
            xe = random_brick(rng, affine=False) if npe == 8 else random_tet(rng)
            lam, mu = random_lame(rng)
            K = ke_el(npe, xe, lam, mu)
            R = rigid_modes(xe)
            if np.abs(K @ R).max() > 1e-12 * np.abs(K).max() * np.abs(R).max():
                return False
            if np.linalg.eigvalsh(K)[6] <= 1e-9 * np.abs(K).max():  # only 6 zero modes
                return False
    return True


def pin_trace_identity(ke_el, ke_scalar):
    rng = np.random.default_rng(105)
    for npe in (8, 4):
        xe = random_brick(rng, affine=False) if npe == 8 else random_tet(rng)
        lam, mu = random_lame(rng)
        K = ke_el(npe, xe, lam, mu)
        tr = np.einsum("aibi->ab", K.reshape(npe, 3, npe, 3))
        if not close(tr, (lam + 4.0 * mu) * ke_scalar(npe, xe, 1.0), 1e-12):
            return False
    return True


def pin_rotation(ke_el):
    rng = np.random.default_rng(106)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    for npe in (8, 4):
        xe = random_brick(rng, affine=False) if npe == 8 else random_tet(rng)
        lam, mu = random_lame(rng)
        K = ke_el(npe, xe, lam, mu)
        Kr = ke_el(npe, xe @ Q.T, lam, mu)
        T = np.kron(np.eye(npe), Q)
        if not close(Kr, T @ K @ T.T, 1e-12):
            return False
    return True


def full_from_lower(out, n):
    import scipy.sparse as sp
    rp, col, v = out["rowptr"], out["col"], out["vals"]
    rows = np.repeat(np.arange(n), np.diff(rp))
    L = sp.csr_matrix((v, (rows, col)), shape=(n, n))
    return (L + L.T - sp.diags(L.diagonal())).tocsr()


def pin_patch_test(build, npe):
    """u = A x + b on a jittered mesh of the unit cube: the internal forces K U
    vanish at interior nodes, and U^T K U / 2 equals the energy density of the
    constant strain sym(A) times the volume 1, for uniform (lambda, mu)."""
    gen = meshgen.hex_grid if npe == 8 else meshgen.kuhn_tets
    m = gen(3, 3, 2, jitter=0.25, seed=7, c_law="one", permute_nodes=True, permute_elems=True)
    lam, mu = 1.7, 0.6
    c = np.tile([lam, mu], (m.n_elems, 1))
    out = build(npe, m.X, m.E, c)
    K = full_from_lower(out, 3 * m.n_nodes)
    rng = np.random.default_rng(107)
    A = rng.standard_normal((3, 3))
    U = (m.X @ A.T + rng.standard_normal(3)).ravel()
    f = (K @ U).reshape(-1, 3)
    lo, hi = m.X.min(axis=0), m.X.max(axis=0)
    interior = np.all((m.X > lo + 1e-9) & (m.X < hi - 1e-9), axis=1)
    eps = 0.5 * (A + A.T)
    psi = 0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps)
    ok_forces = np.abs(f[interior]).max() <= 1e-12 * np.abs(f).max()
    ok_energy = abs(0.5 * U @ (K @ U) - psi) <= 1e-12 * psi
    return bool(interior.any() and ok_forces and ok_energy)


def run_pins(ke_el, ke_scalar, build):
    return dict(energy_affine=pin_energy_affine_bricks(ke_el), energy_distorted=pin_energy_distorted_brick(ke_el),
                energy_tets=pin_energy_tets(ke_el), rigid=pin_rigid_modes(ke_el),
                trace=pin_trace_identity(ke_el, ke_scalar), rotation=pin_rotation(ke_el),
                patch_hex=pin_patch_test(build, 8), patch_tet=pin_patch_test(build, 4))


def elastic_of(oracle_lib):
    return oracle_lib.ke_elastic_dense


def scalar_of(oracle_lib):
    return lambda npe, xe, c: oracle_lib.ke_dense(npe, xe, c)


def builder_of(oracle_lib):
    return lambda npe, X, E, c: oracle_lib.build_K(npe, X, E, c, op="elasticity")


def test_elastic_energy_affine_bricks(oracle_lib):
    assert pin_energy_affine_bricks(elastic_of(oracle_lib))


def test_elastic_energy_distorted_brick(oracle_lib):
    assert pin_energy_distorted_brick(elastic_of(oracle_lib))


def test_elastic_energy_tets(oracle_lib):
    assert pin_energy_tets(elastic_of(oracle_lib))


def test_elastic_rigid_modes(oracle_lib):
    assert pin_rigid_modes(elastic_of(oracle_lib))


def test_elastic_trace_identity(oracle_lib):
    assert pin_trace_identity(elastic_of(oracle_lib), scalar_of(oracle_lib))


def test_elastic_rotation(oracle_lib):
    assert pin_rotation(elastic_of(oracle_lib))


@pytest.mark.parametrize("npe", [8, 4])
def test_elastic_patch_test(oracle_lib, npe):
    pytest.importorskip("scipy")
    assert pin_patch_test(builder_of(oracle_lib), npe)


def test_elastic_packed_matches_dense(oracle_lib):
    """Packed order p = A(A+1)/2 + B over local DOFs A = 3a + i, and the (lambda, mu)
    columns of c, as the CUDA path reads them."""
    m = meshgen.kuhn_tets(2, 1, 1, jitter=0.2, seed=3)
    c = meshgen.lame(m)
    ke, cs, bad = oracle_lib.ke_packed(4, m.X, m.E, c, op="elasticity")
    assert ke.shape == (m.n_elems, 78) and bad == 0
    for e in range(m.n_elems):
        K = oracle_lib.ke_elastic_dense(4, m.X[m.E[e]], c[e, 0], c[e, 1])
        assert np.array_equal(ke[e], K[np.tril_indices(12)])


MUTATIONS = {
    "voigt_shear_component": ("Be[4][3 * a + 1] = B[2][a]; Be[4][3 * a + 2] = B[1][a];",
                              "Be[4][3 * a + 1] = B[1][a]; Be[4][3 * a + 2] = B[2][a];"),
    "tensor_shear_modulus": ("D[k + 3][k + 3] = mu;", "D[k + 3][k + 3] = 2.0 * mu;"),
    "lambda_diagonal_only": ("for (int l = 0; l < 3; ++l) D[k][l] = lam;",
                             "for (int l = 0; l < 3; ++l) D[k][l] = 0.0;"),
    "tet_weight": ("elastic_add(4, B, fabs(det) / 6.0, lam, mu, ke);",
                   "elastic_add(4, B, fabs(det) / 2.0, lam, mu, ke);"),
    "brick_no_jacobian": ("elastic_add(8, B, fabs(det), lam, mu, ke);", "elastic_add(8, B, 1.0, lam, mu, ke);"),
    "dof_component": ("const int32_t ga = dofxn * E[e * npe + a / dofxn] + a % dofxn;",
                      "const int32_t ga = dofxn * E[e * npe + a / dofxn] + (dofxn - 1 - a % dofxn);"),
    "dof_node_major": ("const int32_t gb = dofxn * E[e * npe + b / dofxn] + b % dofxn;",
                       "const int32_t gb = dofxn * E[e * npe + b % npe] + b / npe;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_elastic_planted_mistakes_are_caught(tmp_path, oracle_lib, monkeypatch, name):
    pytest.importorskip("scipy")
    src = open(os.path.join(os.path.dirname(oracle_lib.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, name  # the complex copy of the routine repeats some lines
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so),
                           str(path), "-lm"])
    monkeypatch.setattr(oracle_lib, "_lib", oracle_lib.declare(ctypes.CDLL(str(so))))
    res = run_pins(elastic_of(oracle_lib), scalar_of(oracle_lib), builder_of(oracle_lib))
    assert not all(res.values()), f"mutation {name} passed every pin: {res}"


def test_elastic_gradient_complex_step_vs_central_differences(oracle_lib):
    """The oracle's gradient of L = sum G_ij K_ij for elasticity (complex step of its
    complex element routine) against central differences of its real matrix, in X,
    lambda and mu."""
    for npe, gen in ((8, meshgen.hex_grid), (4, meshgen.kuhn_tets)):
        m = gen(2, 1, 1, jitter=0.2, seed=8, permute_nodes=True)
        c = meshgen.lame(m)
        K = oracle_lib.build_K(npe, m.X, m.E, c, op="elasticity")
        G = np.random.default_rng(3).standard_normal(K["nnz"])
        dX, dc = oracle_lib.vjp_from_G(npe, m.X, m.E, c, G, K["slot"], op="elasticity")

        def L(X, cc):
            return float(G @ oracle_lib.build_K(npe, X, m.E, cc, op="elasticity")["vals"])

        h = 1e-6
        fd = np.zeros_like(m.X)
        for i in range(m.n_nodes):
            for j in range(3):
                Xp, Xm = m.X.copy(), m.X.copy()
                Xp[i, j] += h
                Xm[i, j] -= h
                fd[i, j] = (L(Xp, c) - L(Xm, c)) / (2 * h)
        assert np.abs(dX - fd).max() <= 1e-6 * np.abs(fd).max()
        fdc = np.zeros_like(c)
        for e in range(m.n_elems):
            for k in range(2):
                cp, cm = c.copy(), c.copy()
                cp[e, k] += h
                cm[e, k] -= h
                fdc[e, k] = (L(m.X, cp) - L(m.X, cm)) / (2 * h)
        assert np.abs(dc - fdc).max() <= 1e-6 * np.abs(fdc).max()
