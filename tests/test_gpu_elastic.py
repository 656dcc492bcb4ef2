"""Parity of the CUDA elasticity operator (three DOFs per node, operator_kind 2)
with the FP64 oracle, through the C ABI.

The DOF pattern must be bit-exact; values within 1e-12 (FP64) or 1e-5 (mixed)
of the oracle relative to each entry's Cauchy-Schwarz scale, as for the scalar
operators.  Tiny patch capacities force many patches and ragged batches on small
meshes; the full-size cases check sampled DOF rows against the oracle and the
rigid-body null space of the whole matrix.
"""
import numpy as np
import pytest

import meshgen
import oracle
from helpers import TOL_FP64, TOL_MIXED, TOL_VJP_FP64, TOL_VJP_MIXED, rel_err, vjp_err, vjp_scales

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ELASTIC = 2


@pytest.fixture(scope="module")
def fem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_04784_gb300 import _build
    _build.build()
    from paper_1501_04784_gb300 import fem as F
    return F


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype)


def make(fem, m, **opts):
    return fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), operator_kind=ELASTIC, **opts)


def inputs(m, prec):
    lame = meshgen.lame(m)
    if prec == "mixed":
        X, c = m.X.astype(np.float32), lame.astype(np.float32)
    else:
        X, c = m.X, lame
    dt = torch.float64 if prec == "fp64" else torch.float32
    return dev(X, dt), dev(c, dt), np.asarray(X, np.float64), np.asarray(c, np.float64)


def oracle_el(m, X, c):
    return oracle.build_K(m.npe, X, m.E, c, op="elasticity")


MESHES = {
    "hex_6x5x4_perm": lambda: meshgen.hex_grid(6, 5, 4, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True),
    "hex_1x1x1": lambda: meshgen.hex_grid(1, 1, 1, jitter=0.0, seed=1),
    "tet_5x4x3_perm": lambda: meshgen.kuhn_tets(5, 4, 3, jitter=0.3, seed=2, permute_nodes=True, permute_elems=True),
}
PATCH_CAPS = {"default": 0, "tiny": 48}


@pytest.mark.parametrize("cap", list(PATCH_CAPS))
@pytest.mark.parametrize("name", list(MESHES))
def test_elastic_pattern_bit_exact(fem, name, cap):
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=PATCH_CAPS[cap])
    X, c = m.X, meshgen.lame(m)
    ref = oracle_el(m, X, c)
    assert mesh.pattern() == ref["nnz"]
    rowptr, col = mesh.get_pattern()
    assert np.array_equal(rowptr.cpu().numpy(), ref["rowptr"])
    assert np.array_equal(col.cpu().numpy(), ref["col"])


@pytest.mark.parametrize("cap", list(PATCH_CAPS))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_elastic_build_K(fem, name, prec, cap):
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=PATCH_CAPS[cap])
    Xd, cd, X, c = inputs(m, prec)
    ref = oracle_el(m, X, c)
    vals = mesh.build_K(Xd, cd, prec)
    mesh.sync()
    err = rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"])
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex_6x5x4_perm", "tet_5x4x3_perm"])
def test_elastic_integrate_and_assemble(fem, name, prec):
    """The staged path: packed element matrices (p = A(A+1)/2 + B over local DOFs)
    against the oracle's, then their assembly against the oracle's K."""
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=64)
    Xd, cd, X, c = inputs(m, prec)
    ke = mesh.integrate_local(Xd, cd, prec)
    ref_ke, cs, _ = oracle.ke_packed(m.npe, X, m.E, c, op="elasticity")
    assert ke.shape == ref_ke.shape
    tol = TOL_FP64 if prec == "fp64" else TOL_MIXED
    assert rel_err(ke.cpu().numpy().ravel(), ref_ke.ravel(), cs.ravel()) <= tol
    vals = mesh.assemble_csr(ke, prec)
    mesh.sync()
    ref = oracle_el(m, X, c)
    assert rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"]) <= tol


def test_elastic_assemble_oracle_ke(fem):
    """Assembly alone, of the oracle's own element matrices in FP64: only the
    summation order differs from the oracle's sparse conversion."""
    m = MESHES["tet_5x4x3_perm"]()
    mesh = make(fem, m, patch_entries=64)
    c = meshgen.lame(m)
    ke, _, _ = oracle.ke_packed(m.npe, m.X, m.E, c, op="elasticity")
    vals = mesh.assemble_csr(dev(ke, torch.float64), "fp64").cpu().numpy()
    ref = oracle_el(m, m.X, c)
    assert rel_err(vals, ref["vals"], ref["cs"]) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_elastic_reproducible_and_host_path(fem, prec):
    m = MESHES["hex_6x5x4_perm"]()
    Xd, cd, X, c = inputs(m, prec)
    outs = []
    for threads, bps in ((256, 0), (256, 0), (128, 1), (64, 2)):
        mesh = make(fem, m, block_threads=threads, blocks_per_sm=bps, patch_entries=256)
        outs.append(mesh.build_K(Xd, cd, prec).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint8), outs[0].view(np.uint8))
    mesh = make(fem, m, patch_entries=256)
    hv = mesh.build_K_host(Xd.cpu().pin_memory(), cd.cpu().pin_memory(), prec).numpy()
    assert np.array_equal(hv.view(np.uint8), outs[0].view(np.uint8))


def dof_matvec(rp, col, vals, u):
    """y = K u for the symmetric K stored as its lower triangle (on the GPU)."""
    n = rp.numel() - 1
    rows = torch.repeat_interleave(torch.arange(n, device=rp.device), rp[1:] - rp[:-1])
    colL = col.long()
    y = torch.zeros(n, dtype=vals.dtype, device=vals.device)
    y.index_add_(0, rows, vals * u[colL])
    off = rows != colL
    y.index_add_(0, colL[off], vals[off] * u[rows[off]])
    return y


def rigid_modes(X):
    n = X.shape[0]
    modes = []
    for i in range(3):
        u = np.zeros((n, 3))
        u[:, i] = 1.0
        modes.append(u.ravel())
    x = X - X.mean(axis=0)
    for i in range(3):
        w = np.zeros(3)
        w[i] = 1.0
        modes.append(np.cross(w, x).ravel())
    return modes


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_elastic_full_size_sampled(fem, kind):
    """Large meshes (40^3 bricks, 24^3 cells of tetrahedra, permuted, jittered) in
    mixed precision: DOF rows of sampled nodes against the oracle, and the six
    rigid-body motions in the null space of the assembled matrix."""
    if kind == "hex":
        m = meshgen.hex_grid(40, jitter=0.25, seed=11, permute_nodes=True, permute_elems=True, c_sigma=1.0)
    else:
        m = meshgen.kuhn_tets(24, jitter=0.3, seed=12, permute_nodes=True, permute_elems=True)
    mesh = make(fem, m)
    Xd, cd, X, c = inputs(m, "mixed")
    vals = mesh.build_K(Xd, cd, "mixed")
    mesh.sync()
    rowptr, col = mesh.get_pattern()
    rp, cl, v = rowptr.cpu().numpy(), col.cpu().numpy(), vals.cpu().numpy()
    rng = np.random.default_rng(21)
    nodes = rng.choice(m.n_nodes, 400, replace=False)
    touch = np.isin(m.E, nodes).any(axis=1)
    sub = oracle.build_K(m.npe, X, m.E[touch], c[touch], op="elasticity")
    worst = 0.0
    for n in nodes:
        for r in range(3 * n, 3 * n + 3):
            a, b = sub["rowptr"][r], sub["rowptr"][r + 1]
            assert np.array_equal(cl[rp[r]:rp[r + 1]], sub["col"][a:b])
            worst = max(worst, rel_err(v[rp[r]:rp[r + 1]], sub["vals"][a:b], sub["cs"][a:b]))
    assert worst <= TOL_MIXED, worst
    # residual of each DOF relative to sum_j sqrt(K_ii K_jj) |u_j| (the
    # Cauchy-Schwarz scale of its terms; entries themselves may cancel)
    K64 = vals.double()
    n = rowptr.numel() - 1
    rows = torch.repeat_interleave(torch.arange(n, device="cuda"), rowptr[1:] - rowptr[:-1])
    diag = torch.zeros(n, dtype=torch.float64, device="cuda")
    on = rows == col.long()
    diag[rows[on]] = K64[on].abs()
    S = torch.sqrt(diag[rows] * diag[col.long()])
    for u in rigid_modes(X):
        ud = torch.as_tensor(u, device="cuda")
        y = dof_matvec(rowptr, col, K64, ud)
        scale = dof_matvec(rowptr, col, S, ud.abs())
        assert float((y.abs() / scale.clamp_min(1e-300)).max()) <= 1e-5


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_elastic_zero_volume_element_is_reported(fem, prec):
    from paper_1501_04784_gb300 import abi
    m = MESHES["hex_6x5x4_perm"]()
    X = m.X.copy()
    X[m.E[0], 2] = X[m.E[0][0], 2]
    bad = make(fem, m)
    dt = torch.float32 if prec == "mixed" else torch.float64
    bad.build_K(dev(X, dt), dev(meshgen.lame(m), dt), prec)
    with pytest.raises(abi.FemError, match="FEM_ERR_DEGENERATE"):
        bad.sync()
    bad.sync()
    # the backward pass reports it the same way
    G = torch.ones(bad.nnz, dtype=dt, device="cuda")
    bad.vjp(dev(X, dt), dev(meshgen.lame(m), dt), G, prec)
    with pytest.raises(abi.FemError, match="FEM_ERR_DEGENERATE"):
        bad.sync()
    bad.sync()


@pytest.mark.parametrize("cap", list(PATCH_CAPS))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_elastic_backward(fem, name, prec, cap):
    """The backward pass of the elasticity operator: dL/dX and (dL/dlambda, dL/dmu)
    of L = sum over stored DOF entries G_ij K_ij against the oracle's complex-step
    gradient; the tiny patch capacity makes many patches and ragged batches."""
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=PATCH_CAPS[cap])
    Xd, cd, X, c = inputs(m, prec)
    ref = oracle_el(m, X, c)
    G = np.random.default_rng(11).standard_normal(ref["nnz"])
    if prec == "mixed":
        G = G.astype(np.float32)
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, X, m.E, c, G.astype(np.float64), ref["slot"], op="elasticity")
    dt = torch.float64 if prec == "fp64" else torch.float32
    mesh.pattern()
    assert mesh.nnz == ref["nnz"]
    dX, dc = mesh.vjp(Xd, cd, dev(G, dt), prec)
    assert dc.shape == (m.n_elems, 2)
    dX, dc = dX.cpu().numpy().astype(np.float64), dc.cpu().numpy().astype(np.float64)
    sx, sc = vjp_scales(m, X, c, np.asarray(G, np.float64)[ref["slot"]], op="elasticity")
    tol = TOL_VJP_FP64 if prec == "fp64" else TOL_VJP_MIXED
    assert vjp_err(dX, dX_ref, sx) <= tol, vjp_err(dX, dX_ref, sx)
    assert vjp_err(dc, dc_ref, sc) <= tol, vjp_err(dc, dc_ref, sc)
    # bitwise reproducible: owner-computes accumulation in a fixed colour order
    dX2, dc2 = mesh.vjp(Xd, cd, dev(G, dt), prec)
    assert np.array_equal(dX2.cpu().numpy().astype(np.float64), dX)
    assert np.array_equal(dc2.cpu().numpy().astype(np.float64), dc)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex_6x5x4_perm", "tet_5x4x3_perm"])
def test_elastic_backward_staged_and_fused_agree(fem, name, prec):
    """The staged elasticity backward (element pass into library memory, then the
    gather) against the fused one, up to the rounding of the element arithmetic."""
    m = MESHES[name]()
    Xd, cd, _, _ = inputs(m, prec)
    staged, fused = make(fem, m, patch_entries=48), make(fem, m, patch_entries=48, vjp_fused=1)
    nnz = staged.pattern()
    fused.pattern()
    dt = torch.float64 if prec == "fp64" else torch.float32
    G = dev(np.random.default_rng(13).standard_normal(nnz), dt)
    a, b = staged.vjp(Xd, cd, G, prec), fused.vjp(Xd, cd, G, prec)
    tol = 1e-13 if prec == "fp64" else 2e-6
    for u, v in zip(a, b):
        assert (u - v).abs().max().item() <= tol * v.abs().max().item()
    assert staged.info()["live_bytes"] > fused.info()["live_bytes"]


def test_elastic_autograd(fem):
    """torch.autograd through build_K: the gradient of a scalar function of K's
    values reaches X and the Lame parameters [n_elems, 2]."""
    from paper_1501_04784_gb300 import autograd
    m = MESHES["hex_6x5x4_perm"]()
    mesh = make(fem, m)
    Xd, cd, X, c = inputs(m, "fp64")
    Xd.requires_grad_(True)
    cd.requires_grad_(True)
    vals = autograd.build_K(mesh, Xd, cd, "fp64")
    G = np.random.default_rng(12).standard_normal(mesh.nnz)
    (vals * dev(G, torch.float64)).sum().backward()
    ref = oracle_el(m, X, c)
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, X, m.E, c, G, ref["slot"], op="elasticity")
    assert Xd.grad.shape == (m.n_nodes, 3) and cd.grad.shape == (m.n_elems, 2)
    assert np.abs(Xd.grad.cpu().numpy() - dX_ref).max() <= 1e-11 * np.abs(dX_ref).max()
    assert np.abs(cd.grad.cpu().numpy() - dc_ref).max() <= 1e-11 * np.abs(dc_ref).max()


@pytest.mark.parametrize("prec,opts", [("mixed", dict(patch_entries=8192)), ("fp64", {}),
                                       ("fp64", dict(fp64_fused=1))])
def test_elastic_row_windows(fem, prec, opts):
    """Patches whose 3x3 blocks outgrow shared memory (FP64 at the default patch
    size; FP32 planned at 8192 node pairs) are accumulated in row windows, one
    pass over the closure each: the FP64 build stages element matrices by default
    (fp64_fused=1 integrates in every pass instead)."""
    m = meshgen.hex_grid(20, 20, 12, jitter=0.25, seed=8, permute_nodes=True, permute_elems=True)
    mesh = make(fem, m, **opts)
    mesh.pattern()
    assert mesh.info()["max_patch_entries"] > (3000 if prec == "fp64" else 6000)
    Xd, cd, X, c = inputs(m, prec)
    vals = mesh.build_K(Xd, cd, prec)
    mesh.sync()
    ref = oracle_el(m, X, c)
    assert rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"]) <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_elastic_budget_groups_bitwise_equal(fem, prec):
    """Under a budget too small for all closures the plan runs in patch groups
    (Eq. 10): the elasticity build and its backward pass give exactly the
    unbudgeted values."""
    m = meshgen.hex_grid(16, jitter=0.2, seed=77, permute_nodes=True, permute_elems=True)
    Xd, cd, _, _ = inputs(m, prec)
    free = make(fem, m, patch_entries=256, fp64_fused=1)
    ref = free.build_K(Xd, cd, prec)
    need = free.info()["plan_bytes"]
    tight = make(fem, m, patch_entries=256, mem_budget_bytes=int(need * 0.75), fp64_fused=1)
    got = tight.build_K(Xd, cd, prec)
    tight.sync()
    assert tight.info()["n_groups"] > 1
    assert torch.equal(got, ref)
    # the backward pass in patch groups (always the fused kernel there) equals the
    # unbudgeted fused pass bit for bit
    dt = torch.float64 if prec == "fp64" else torch.float32
    G = torch.randn(free.nnz, generator=torch.Generator(device="cuda").manual_seed(15), device="cuda").to(dt)
    fused = make(fem, m, patch_entries=256, fp64_fused=1, vjp_fused=1)
    fused.pattern()
    a, b = fused.vjp(Xd, cd, G, prec), tight.vjp(Xd, cd, G, prec)
    tight.sync()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_elastic_autotune(fem):
    m = MESHES["hex_6x5x4_perm"]()
    mesh = make(fem, m)
    Xd, cd, X, c = inputs(m, "mixed")
    t = mesh.autotune(Xd, cd, "mixed")
    assert t["tried"] >= 3 and t["patch_entries"] in (1536, 2048, 3072, 4096, 5120)
    vals = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
    ref = oracle_el(m, X, c)
    assert rel_err(vals, ref["vals"], ref["cs"]) <= TOL_MIXED


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex_6x5x4_perm", "tet_5x4x3_perm"])
def test_elastic_body_force_load(fem, name, prec):
    """The elasticity load vector: F[3n + i] = sum_e b_e,i integral N_a against the
    oracle's scalar load of each component, and the total force sum_e b_e vol_e."""
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=64)
    mesh.pattern()
    b = np.random.default_rng(4).standard_normal((m.n_elems, 3))
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = m.X if prec == "fp64" else m.X.astype(np.float32)
    bb = b if prec == "fp64" else b.astype(np.float32)
    F = mesh.load_vector(dev(X, dt), dev(bb, dt), prec)
    mesh.sync()
    F = F.cpu().numpy().astype(np.float64)
    ref = oracle.load_vector(m.npe, np.asarray(X, np.float64), m.E, np.asarray(bb, np.float64))
    scale = oracle.load_vector(m.npe, np.asarray(X, np.float64), m.E, np.abs(np.asarray(bb, np.float64)))
    tol = TOL_FP64 if prec == "fp64" else TOL_MIXED
    assert F.shape == (3 * m.n_nodes,)
    assert np.max(np.abs(F - ref) / np.maximum(scale, 1e-300)) <= tol


@pytest.mark.parametrize("kind,prec", [("hex", "mixed"), ("tet", "mixed"), ("hex", "fp64")])
def test_elastic_batched(fem, kind, prec):
    """Many elasticity meshes in one persistent launch (graph replay on the second
    call): mixed builds equal the single builds bit for bit; FP64 (fused, in row
    windows, where the single build stages element matrices) matches the oracle."""
    gen = meshgen.hex_grid if kind == "hex" else meshgen.kuhn_tets
    ms = [gen(3 + i % 4, 2 + i % 3, 2 + i % 5, jitter=0.2, seed=300 + i, permute_nodes=True) for i in range(9)]
    dt = torch.float32 if prec == "mixed" else torch.float64
    meshes = [make(fem, m) for m in ms]
    Xs = [dev(m.X, dt) for m in ms]
    cs = [dev(meshgen.lame(m), dt) for m in ms]
    single = [mesh.build_K(X, c, prec).clone() for mesh, X, c in zip(meshes, Xs, cs)]
    for rep in range(2):
        got = fem.build_K_batched(meshes, Xs, cs, prec)
        meshes[0].sync()
        for m, g, sref in zip(ms, got, single):
            if prec == "mixed":
                assert torch.equal(g, sref)
            else:
                ref = oracle_el(m, m.X, meshgen.lame(m))
                assert rel_err(g.cpu().numpy(), ref["vals"], ref["cs"]) <= TOL_FP64


@pytest.mark.parametrize("fp64_dets", [0, 1])
def test_elastic_sliver_tets(fem, fp64_dets):
    """Slivers (a fourth node 1e-4 above a unit triangle, rotated and shifted): the
    elasticity kernel takes the scalar operator's FP64-accurate determinant and face
    vectors, so the mixed build still meets the tolerance against the oracle."""
    rng = np.random.default_rng(7)
    P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.3, 1e-4]], float)
    X, E = [], []
    for t in range(48):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        X.append(P @ Q.T + rng.normal(size=3))
        E.append([4 * t, 4 * t + 1, 4 * t + 2, 4 * t + 3])
    m = meshgen.Mesh(X=np.vstack(X), E=np.asarray(E, np.int32), c=rng.lognormal(0, 0.5, 48), npe=4, shape=(48, 1, 1))
    mesh = make(fem, m, fp64_dets=fp64_dets)
    Xd, cd, X64, c64 = inputs(m, "mixed")
    vals = mesh.build_K(Xd, cd, "mixed")
    mesh.sync()
    ref = oracle_el(m, X64, c64)
    assert rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"]) <= TOL_MIXED
