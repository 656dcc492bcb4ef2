"""Backward pass: the GPU vector-Jacobian product against the oracle's
complex-step gradient, and against central finite differences of the GPU build
on the 10^3 sub-mesh of the large streamed workload."""
import numpy as np
import pytest

import meshgen
import oracle
from helpers import TOL_VJP_FP64, TOL_VJP_MIXED, rounded_inputs, vjp_err, vjp_scales

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


CASES = {
    "hex_4x3x3": lambda: meshgen.hex_grid(4, 3, 3, jitter=0.25, seed=31, permute_nodes=True, permute_elems=True),
    "tet_3x3x2": lambda: meshgen.kuhn_tets(3, 3, 2, jitter=0.25, seed=32, permute_nodes=True, permute_elems=True),
    "hex20_perm": lambda: meshgen.config_mesh(0),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_vjp_matches_oracle_gradient(fem, name, prec):
    m = CASES[name]()
    X, c = rounded_inputs(m, prec)
    ref = oracle.build_K(m.npe, X.astype(np.float64), m.E, c.astype(np.float64))
    G = np.random.default_rng(4).standard_normal(ref["nnz"])
    if prec == "mixed":
        G = G.astype(np.float32)
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, X.astype(np.float64), m.E, c.astype(np.float64),
                                       G.astype(np.float64), ref["slot"])
    dt = torch.float64 if prec == "fp64" else torch.float32
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512)
    mesh.pattern()
    dX, dc = mesh.vjp(dev(X, dt), dev(c, dt), dev(G, dt), prec)
    dX, dc = dX.cpu().numpy().astype(np.float64), dc.cpu().numpy().astype(np.float64)
    # per component, against the scale of the terms that make it up
    sx, sc = vjp_scales(m, X, c, np.asarray(G, np.float64)[ref["slot"]])
    tol = TOL_VJP_FP64 if prec == "fp64" else TOL_VJP_MIXED
    assert vjp_err(dX, dX_ref, sx) <= tol, vjp_err(dX, dX_ref, sx)
    assert vjp_err(dc, dc_ref, sc) <= tol, vjp_err(dc, dc_ref, sc)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex_4x3x3", "tet_3x3x2", "hex20_perm"])
def test_vjp_staged_and_fused_agree(fem, name, prec):
    """The staged backward (every element once into library memory, then a gather in
    colour order) and the fused one (recomputed in every closure holding the
    element) give the same gradients up to the rounding of the element arithmetic.
    (A plan built per patch group always takes the fused pass: test_gpu_batch_budget.)"""
    m = CASES[name]()
    X, c = rounded_inputs(m, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd, cd = dev(X, dt), dev(c, dt)
    staged = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512)
    fused = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512, vjp_fused=1)
    nnz = staged.pattern()
    fused.pattern()
    G = dev(np.random.default_rng(8).standard_normal(nnz), dt)
    a, b = staged.vjp(Xd, cd, G, prec), fused.vjp(Xd, cd, G, prec)
    tol = 1e-13 if prec == "fp64" else 2e-6
    for u, v in zip(a, b):
        assert (u - v).abs().max().item() <= tol * v.abs().max().item()
    scratch = m.n_elems * m.npe * 3 * (8 if prec == "fp64" else 4)
    assert staged.info()["live_bytes"] >= fused.info()["live_bytes"] + scratch


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vjp_zero_volume_element_is_reported(fem, prec, fused):
    """A brick flattened to zero volume has no finite gradient: the backward pass
    finishes, fem_sync reports FEM_ERR_DEGENERATE once, and a valid backward pass
    on the same mesh afterwards matches the oracle."""
    from paper_1501_04784_gb300 import abi
    m = CASES["hex_4x3x3"]()
    Xv, c = rounded_inputs(m, prec)
    X = Xv.copy()
    X[m.E[0], 2] = X[m.E[0][0], 2]  # all 8 nodes of element 0 in one z plane
    dt = torch.float64 if prec == "fp64" else torch.float32
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512, vjp_fused=fused)
    nnz = mesh.pattern()
    G = np.random.default_rng(14).standard_normal(nnz)
    if prec == "mixed":
        G = G.astype(np.float32)
    mesh.vjp(dev(X, dt), dev(c, dt), dev(G, dt), prec)
    with pytest.raises(abi.FemError, match="FEM_ERR_DEGENERATE"):
        mesh.sync()
    mesh.sync()
    dX, dc = mesh.vjp(dev(Xv, dt), dev(c, dt), dev(G, dt), prec)
    mesh.sync()
    ref = oracle.build_K(m.npe, Xv.astype(np.float64), m.E, c.astype(np.float64))
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, Xv.astype(np.float64), m.E, c.astype(np.float64),
                                       G.astype(np.float64), ref["slot"])
    sx, sc = vjp_scales(m, Xv, c, np.asarray(G, np.float64)[ref["slot"]])
    tol = TOL_VJP_FP64 if prec == "fp64" else TOL_VJP_MIXED
    assert vjp_err(dX.cpu().numpy(), dX_ref, sx) <= tol
    assert vjp_err(dc.cpu().numpy(), dc_ref, sc) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vjp_thin_element_stays_finite(fem, prec):
    """A brick squeezed to 1e-7 of its height (tiny but nonzero Jacobian
    determinants) has a finite gradient: no FEM_ERR_DEGENERATE, every component
    finite, and the oracle's gradient matched."""
    m = meshgen.hex_grid(2, 2, 1, jitter=0.0, seed=3)
    Xv, c = rounded_inputs(m, prec)
    X = Xv.copy()
    X[:, 2] *= 1e-7
    dt = torch.float64 if prec == "fp64" else torch.float32
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(X, torch.float64))
    nnz = mesh.pattern()
    G = np.random.default_rng(15).standard_normal(nnz)
    if prec == "mixed":
        G = G.astype(np.float32)
    dX, dc = mesh.vjp(dev(X, dt), dev(c, dt), dev(G, dt), prec)
    mesh.sync()
    dX, dc = dX.cpu().numpy().astype(np.float64), dc.cpu().numpy().astype(np.float64)
    assert np.isfinite(dX).all() and np.isfinite(dc).all()
    ref = oracle.build_K(m.npe, X.astype(np.float64), m.E, c.astype(np.float64))
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, X.astype(np.float64), m.E, c.astype(np.float64),
                                       G.astype(np.float64), ref["slot"])
    sx, sc = vjp_scales(m, X, c, np.asarray(G, np.float64)[ref["slot"]])
    tol = TOL_VJP_FP64 if prec == "fp64" else TOL_VJP_MIXED
    assert vjp_err(dX, dX_ref, sx) <= tol and vjp_err(dc, dc_ref, sc) <= tol


def test_vjp_bitwise_reproducible(fem):
    m = CASES["hex20_perm"]()
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    nnz = mesh.pattern()
    G = dev(np.random.default_rng(5).standard_normal(nnz), torch.float64)
    X, c = dev(m.X, torch.float64), dev(m.c, torch.float64)
    a = mesh.vjp(X, c, G, "fp64")
    b = mesh.vjp(X, c, G, "fp64")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_autograd_central_differences_10cube(fem):
    """The large workload's recipe (jitter 0.2h, c ~ lognormal(0, 0.5)) on its
    10^3 sub-mesh: torch.autograd through BuildK against central differences of
    the GPU build itself, for sampled coordinates and coefficients (FP64)."""
    from paper_1501_04784_gb300.autograd import build_K
    m = meshgen.config_mesh(4, nx=10)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    nnz = mesh.pattern()
    G = dev(np.random.default_rng(6).standard_normal(nnz), torch.float64)
    X = dev(m.X, torch.float64).requires_grad_(True)
    c = dev(m.c, torch.float64).requires_grad_(True)
    L = (build_K(mesh, X, c, "fp64") * G).sum()
    L.backward()
    rng = np.random.default_rng(7)
    h = 1e-6

    def Lval(Xv, cv):
        return float((mesh.build_K(Xv, cv, "fp64") * G).sum())

    Xd, cd = X.detach(), c.detach()
    for _ in range(25):
        i, j = int(rng.integers(m.n_nodes)), int(rng.integers(3))
        Xp, Xm = Xd.clone(), Xd.clone()
        Xp[i, j] += h
        Xm[i, j] -= h
        fd = (Lval(Xp, cd) - Lval(Xm, cd)) / (2 * h)
        assert abs(fd - float(X.grad[i, j])) <= 1e-6 * (abs(fd) + 1e-3)
    for _ in range(25):
        e = int(rng.integers(m.n_elems))
        cp, cm = cd.clone(), cd.clone()
        cp[e] += h
        cm[e] -= h
        fd = (Lval(Xd, cp) - Lval(Xd, cm)) / (2 * h)
        assert abs(fd - float(c.grad[e])) <= 1e-6 * (abs(fd) + 1e-3)


@pytest.mark.parametrize("name", ["hex_4x3x3", "tet_3x3x2"])
def test_positions_added_by_first_backward(fem, name):
    """A mesh that only builds K holds no in-row positions (they serve the backward
    pass only): the first backward pass adds them to the cached closures (the plan
    grows by 4 bytes per packed pair, padded, per closure element), its gradient
    matches the oracle, and the builds before and after it are bitwise equal."""
    m = CASES[name]()
    X, c = rounded_inputs(m, "mixed")
    Xd, cd = dev(X, torch.float32), dev(c, torch.float32)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512)
    nnz = mesh.pattern()
    before = mesh.build_K(Xd, cd, "mixed").clone()
    info0 = mesh.info()
    ref = oracle.build_K(m.npe, X.astype(np.float64), m.E, c.astype(np.float64))
    G = np.random.default_rng(9).standard_normal(nnz).astype(np.float32)
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, X.astype(np.float64), m.E, c.astype(np.float64),
                                       G.astype(np.float64), ref["slot"])
    dX, dc = mesh.vjp(Xd, cd, dev(G, torch.float32), "mixed")
    mesh.sync()
    npairs = m.npe * (m.npe + 1) // 2
    grown = mesh.info()["plan_bytes"] - info0["plan_bytes"]
    assert grown == info0["closure_elems"] * ((npairs + 3) // 4 * 4)
    sx, sc = vjp_scales(m, X, c, G[ref["slot"]])
    assert vjp_err(dX.cpu().numpy(), dX_ref, sx) <= TOL_VJP_MIXED
    assert vjp_err(dc.cpu().numpy(), dc_ref, sc) <= TOL_VJP_MIXED
    assert torch.equal(mesh.build_K(Xd, cd, "mixed"), before)
