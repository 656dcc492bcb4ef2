"""The mass operator (fem_options.operator_kind = 1): M = sum_e c_e int N^T N, the
other operator the paper's construction generalises to (Section 5), through the same
kernels, plan and assembly as the stiffness matrix, against the oracle's mass
operator (itself pinned in test_oracle_mass_pins.py)."""
import numpy as np
import pytest

import meshgen
import oracle
from helpers import (TOL_FP64, TOL_MIXED, TOL_VJP_FP64, TOL_VJP_MIXED, oracle_K, oracle_ke, oracle_rows, rel_err,
                     rounded_inputs, vjp_err, vjp_scales)

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


def inputs(m, prec):
    X, c = rounded_inputs(m, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    return dev(X, dt), dev(c, dt), X, c


MESHES = {
    "hex20_perm": lambda: meshgen.config_mesh(0),
    "tet10_perm": lambda: meshgen.config_mesh(2, nx=10),
    "hex_7x5x3": lambda: meshgen.hex_grid(7, 5, 3, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True),
}


def mass_mesh(fem, m, **opts):
    return fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), operator_kind=1, **opts)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_mass_build_against_oracle(fem, name, prec):
    m = MESHES[name]()
    for cap in (0, 64):
        mesh = mass_mesh(fem, m, patch_entries=cap)
        Xd, cd, X, c = inputs(m, prec)
        ref = oracle_K(m, X, c, op="mass")
        assert mesh.pattern() == ref["nnz"]
        vals = mesh.build_K(Xd, cd, prec).cpu().numpy()
        err = rel_err(vals, ref["vals"], ref["cs"])
        assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), (cap, err)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex20_perm", "tet10_perm"])
def test_mass_integrate_local(fem, name, prec):
    m = MESHES[name]()
    mesh = mass_mesh(fem, m)
    Xd, cd, X, c = inputs(m, prec)
    me = mesh.integrate_local(Xd, cd, prec).cpu().numpy()
    ref, cs, _ = oracle_ke(m, X, c, op="mass")
    assert rel_err(me.ravel(), ref.ravel(), cs.ravel()) <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)


def test_mass_total_is_volume(fem):
    """u^T M u for u = 1 with c = 1 is the volume of the unit cube that the jittered
    mesh tiles: the full matrix's sum, 2 * lower - diagonal."""
    m = meshgen.hex_grid(12, 9, 7, jitter=0.25, seed=8, c_law="one", permute_nodes=True, permute_elems=True)
    mesh = mass_mesh(fem, m)
    Xd, cd, X, c = inputs(m, "fp64")
    vals = mesh.build_K(Xd, cd, "fp64").cpu().numpy()
    rowptr, col = mesh.get_pattern()
    rp, cl = rowptr.cpu().numpy(), col.cpu().numpy()
    diag = vals[rp[1:] - 1]
    assert np.array_equal(cl[rp[1:] - 1], np.arange(m.n_nodes))
    assert abs(2 * vals.sum() - diag.sum() - 1.0) <= 1e-12


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_mass_batched_equals_single(fem, kind):
    ms = [meshgen.hex_grid(3 + i, 4, 2 + i % 3, jitter=0.2, seed=40 + i, permute_nodes=True) if kind == "hex"
          else meshgen.kuhn_tets(3 + i, 3, 2 + i % 2, jitter=0.25, seed=60 + i, permute_nodes=True)
          for i in range(6)]
    meshes = [mass_mesh(fem, m, patch_entries=256) for m in ms]
    Xs = [dev(m.X, torch.float32) for m in ms]
    cs = [dev(m.c, torch.float32) for m in ms]
    single = [mesh.build_K(X, c, "mixed").clone() for mesh, X, c in zip(meshes, Xs, cs)]
    got = fem.build_K_batched(meshes, Xs, cs, "mixed")
    for a, b in zip(got, single):
        assert torch.equal(a, b)


def test_mass_full_size_sampled(fem):
    """The 1M-brick workload's mass matrix in mixed precision, sampled rows against the oracle."""
    m = meshgen.config_mesh(1)
    mesh = mass_mesh(fem, m)
    nnz = mesh.pattern()
    rowptr, col = mesh.get_pattern()
    rp = rowptr.cpu().numpy()
    Xd, cd, X, c = inputs(m, "mixed")
    vals = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
    sample = np.random.default_rng(31).choice(m.n_nodes, 1500, replace=False)
    worst = 0.0
    for r, (cols, v, sc) in oracle_rows(m, sample, X, c, op="mass").items():
        worst = max(worst, rel_err(vals[rp[r]:rp[r + 1]], v, sc))
    assert nnz == 14150601 and worst <= TOL_MIXED, worst


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex_7x5x3", "tet10_perm"])
def test_mass_backward(fem, name, prec):
    """The backward pass of the mass operator: dL/dX and dL/dc of L = sum G_ij M_ij
    against the oracle's complex-step gradient."""
    m = MESHES[name]()
    mesh = mass_mesh(fem, m)
    Xd, cd, X, c = inputs(m, prec)
    ref = oracle.build_K(m.npe, X, m.E, c, op="mass")
    G = np.random.default_rng(9).standard_normal(ref["nnz"])
    if prec == "mixed":
        G = G.astype(np.float32)
    dX_ref, dc_ref = oracle.vjp_from_G(m.npe, X, m.E, c, G.astype(np.float64), ref["slot"], op="mass")
    dt = torch.float64 if prec == "fp64" else torch.float32
    mesh.pattern()
    dX, dc = mesh.vjp(Xd, cd, dev(G, dt), prec)
    dX, dc = dX.cpu().numpy().astype(np.float64), dc.cpu().numpy().astype(np.float64)
    sx, sc = vjp_scales(m, X, c, np.asarray(G, np.float64)[ref["slot"]], op="mass")
    tol = TOL_VJP_FP64 if prec == "fp64" else TOL_VJP_MIXED
    assert vjp_err(dX, dX_ref, sx) <= tol, vjp_err(dX, dX_ref, sx)
    assert vjp_err(dc, dc_ref, sc) <= tol, vjp_err(dc, dc_ref, sc)
