"""Batched builds (one persistent launch + CUDA graph over uneven meshes), builds
under a memory budget (patch groups), and the tuner.  Each must give exactly the
values of the plain per-mesh build of the same plan, and those stay within
tolerance of the oracle."""
import numpy as np
import pytest

import meshgen
from helpers import TOL_FP64, TOL_MIXED, oracle_K, rel_err

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


def small_batch(n, kind="hex"):
    out = []
    for i in range(n):
        nx, ny, nz = 3 + i % 5, 4 + (i * 7) % 6, 2 + (i * 3) % 7
        if kind == "hex":
            out.append(meshgen.hex_grid(nx, ny, nz, jitter=0.2, seed=1000 + i, permute_nodes=True, permute_elems=True))
        else:
            out.append(meshgen.kuhn_tets(nx, ny, nz, jitter=0.25, seed=2000 + i, permute_nodes=True))
    return out


@pytest.mark.parametrize("assembly", [0, 1], ids=["patches", "tiles"])
@pytest.mark.parametrize("kind,prec", [("hex", "mixed"), ("tet", "mixed"), ("hex", "fp64")])
def test_batched_equals_single_builds(fem, kind, prec, assembly):
    ms = small_batch(17, kind)
    dt = torch.float32 if prec == "mixed" else torch.float64
    meshes = [fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512,
                       tile_elems=64, assembly=assembly) for m in ms]
    Xs = [dev(m.X, dt) for m in ms]
    cs = [dev(m.c, dt) for m in ms]
    single = [mesh.build_K(X, c, prec).clone() for mesh, X, c in zip(meshes, Xs, cs)]
    for rep in range(3):   # first call tunes and captures, later calls replay the graph
        got = fem.build_K_batched(meshes, Xs, cs, prec)
        for a, b in zip(got, single):
            assert torch.equal(a, b)
    cfg = fem.batched_config(meshes, prec)
    assert cfg["block_threads"] in (128, 256, 512) and cfg["grid"] > 0
    # new input buffers: the graph replays with the refreshed descriptor table
    Xs2 = [(X * 1.01).contiguous() for X in Xs]
    got = fem.build_K_batched(meshes, Xs2, cs, prec)
    for mesh, X, c, g in zip(meshes, Xs2, cs, got):
        assert torch.equal(g, mesh.build_K(X, c, prec))
    # values against the oracle for a few meshes
    tol = TOL_MIXED if prec == "mixed" else TOL_FP64
    for i in (0, 5, 16):
        m = ms[i]
        X = m.X.astype(np.float32).astype(np.float64) if prec == "mixed" else m.X
        c = m.c.astype(np.float32).astype(np.float64) if prec == "mixed" else m.c
        ref = oracle_K(m, X * (1.0 if rep < 0 else 1.0), c)
        assert rel_err(single[i].cpu().numpy(), ref["vals"], ref["cs"]) <= tol
    for mesh in meshes:
        mesh.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_budget_groups_bitwise_equal(fem, prec):
    """A budget too small for all closures at once: the plan runs in patch groups
    (Eq. 10) and gives exactly the values of the unbudgeted build."""
    m = meshgen.hex_grid(24, jitter=0.2, seed=77, permute_nodes=True, permute_elems=True)
    dt = torch.float32 if prec == "mixed" else torch.float64
    X, c = dev(m.X, dt), dev(m.c, dt)
    # FP64 builds and backward passes fuse here on both sides (a plan built per
    # patch group always fuses them), so the two differ only in the grouping
    free = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=1024, fp64_fused=1,
                    vjp_fused=1)
    ref = free.build_K(X, c, prec)
    need = free.info()["plan_bytes"]
    tight = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=1024,
                     mem_budget_bytes=int(need * 0.75), fp64_fused=1)
    got = tight.build_K(X, c, prec)
    info = tight.info()
    assert info["n_groups"] > 1
    assert info["closure_elems"] == free.info()["closure_elems"]
    assert torch.equal(got, ref)
    G = dev(np.random.default_rng(3).standard_normal(free.nnz), dt)
    a = free.vjp(X, c, G, prec)
    b = tight.vjp(X, c, G, prec)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_fp64_staged_and_fused_agree(fem):
    """FEM_FP64 integrates once into staged element matrices by default; the fused
    form recomputes them per closure.  Both match the oracle to FP64 tolerance."""
    m = meshgen.config_mesh(0)
    X, c = dev(m.X, torch.float64), dev(m.c, torch.float64)
    staged = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=X).build_K(X, c, "fp64").cpu().numpy()
    fused = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=X, fp64_fused=1).build_K(X, c, "fp64").cpu().numpy()
    ref = oracle_K(m)
    assert rel_err(staged, ref["vals"], ref["cs"]) <= TOL_FP64
    assert rel_err(fused, ref["vals"], ref["cs"]) <= TOL_FP64
    assert np.abs(staged - fused).max() <= 1e-14 * np.abs(ref["cs"]).max()


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_group_cache_equals_rebuilt_groups(fem, kind):
    """Patch groups copied back from the host copies of their closures (group_cache,
    the default; their accumulator targets derived on the device from the in-row
    positions) give the values of groups built again at every call
    (group_cache = 0) and of the unbudgeted build, bitwise, on repeated calls; the
    backward pass agrees too, and the builds after it still do.  Both match the
    oracle."""
    if kind == "hex":
        m = meshgen.hex_grid(24, jitter=0.2, seed=78, permute_nodes=True, permute_elems=True)
    else:
        m = meshgen.kuhn_tets(14, jitter=0.25, seed=79, permute_nodes=True, permute_elems=True)
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    E, X64 = dev(m.E, torch.int32), dev(m.X, torch.float64)
    free = fem.Mesh(E, m.n_nodes, X=X64, patch_entries=1024, vjp_fused=1)
    ref = free.build_K(X, c, "mixed")
    budget = int(free.info()["plan_bytes"] * 0.75)
    cached = fem.Mesh(E, m.n_nodes, X=X64, patch_entries=1024, mem_budget_bytes=budget)
    rebuilt = fem.Mesh(E, m.n_nodes, X=X64, patch_entries=1024, mem_budget_bytes=budget, group_cache=0)
    for _ in range(2):
        assert torch.equal(cached.build_K(X, c, "mixed"), ref)
        assert torch.equal(rebuilt.build_K(X, c, "mixed"), ref)
    assert cached.info()["n_groups"] > 1 and rebuilt.info()["n_groups"] > 1
    o = oracle_K(m, m.X.astype(np.float32), m.c.astype(np.float32))
    assert rel_err(ref.cpu().numpy(), o["vals"], o["cs"]) <= TOL_MIXED
    G = dev(np.random.default_rng(5).standard_normal(free.nnz), torch.float32)
    a, b, r = cached.vjp(X, c, G, "mixed"), rebuilt.vjp(X, c, G, "mixed"), free.vjp(X, c, G, "mixed")
    for u, v, w in zip(a, b, r):
        assert torch.equal(u, v) and torch.equal(u, w)
    assert torch.equal(cached.build_K(X, c, "mixed"), ref)
    cached.sync()
    rebuilt.sync()


def test_autotune_tiles(fem):
    """The tuner on a mesh that builds on element tiles picks a tile size."""
    m = meshgen.config_mesh(0)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), assembly=1)
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    t = mesh.autotune(X, c, "mixed")
    assert t["assembly"] == 1 and t["tried"] >= 3 and t["patch_entries"] in (256, 384, 512, 768, 1024)
    assert mesh.info()["assembly"] == 1
    vals = mesh.build_K(X, c, "mixed").cpu().numpy()
    ref = oracle_K(m, m.X.astype(np.float32), m.c.astype(np.float32))
    assert rel_err(vals, ref["vals"], ref["cs"]) <= TOL_MIXED


def test_budget_too_small_for_one_patch(fem):
    from paper_1501_04784_gb300 import abi
    m = meshgen.hex_grid(12, jitter=0.2, seed=5)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, mem_budget_bytes=200_000)
    with pytest.raises(abi.FemError, match="FEM_ERR_BUDGET"):
        mesh.pattern()


def test_autotune_keeps_values_in_tolerance(fem):
    m = meshgen.config_mesh(0)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    t = mesh.autotune(X, c, "mixed")
    assert t["assembly"] == 0 and t["tried"] >= 3 and t["patch_entries"] in (4096, 6144, 8192, 12288, 16384)
    vals = mesh.build_K(X, c, "mixed").cpu().numpy()
    ref = oracle_K(m, m.X.astype(np.float32), m.c.astype(np.float32))
    assert rel_err(vals, ref["vals"], ref["cs"]) <= TOL_MIXED


def test_autotune_cache(fem, tmp_path):
    """The tuner cache: the first call times the candidates and stores the choice
    keyed by GPU, element type, precision, operator and size class; a second mesh
    of the same kind applies it without timing and builds the same values."""
    m = meshgen.config_mesh(0)
    X, c = dev(m.X, torch.float32), dev(m.c, torch.float32)
    cache = str(tmp_path / "tune.json")
    a = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    ta = a.autotune(X, c, "mixed", cache=cache)
    assert ta["tried"] >= 3
    b = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    tb = b.autotune(X, c, "mixed", cache=cache)
    assert tb["tried"] == 0 and (tb["patch_entries"], tb["block_threads"]) == (ta["patch_entries"], ta["block_threads"])
    assert b.info()["n_patches"] == a.info()["n_patches"]
    assert torch.equal(a.build_K(X, c, "mixed"), b.build_K(X, c, "mixed"))
