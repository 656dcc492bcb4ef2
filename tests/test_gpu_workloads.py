"""The two large workloads at full size.

* 512 uneven brick meshes (about 15M elements) built in one persistent launch
  replayed from a CUDA graph, after the tuner picks the patch size on the largest
  mesh: every mesh bitwise equal to its own single build, sampled meshes within
  tolerance of the oracle.
* 300^3 bricks (27M elements, 27.27M nodes) under a 16 GB device budget for the
  library's memory: nnz equal to the closed form, sampled rows against the oracle
  in FP64 and mixed precision.
"""
import numpy as np
import pytest

import meshgen
from helpers import TOL_FP64, TOL_MIXED, oracle_K, oracle_rows, rel_err

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


def test_batch_of_512_uneven_meshes(fem):
    ms = meshgen.batch_meshes()
    assert len(ms) == 512
    total = sum(m.n_elems for m in ms)
    assert 1.2e7 < total < 2.6e7
    big = max(range(len(ms)), key=lambda i: ms[i].n_elems)
    mb = ms[big]
    probe = fem.Mesh(dev(mb.E, torch.int32), mb.n_nodes, X=dev(mb.X, torch.float64))
    tune = probe.autotune(dev(mb.X, torch.float32), dev(mb.c, torch.float32), "mixed")
    probe.close()
    meshes = [fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64),
                       patch_entries=tune["patch_entries"]) for m in ms]
    Xs = [dev(m.X, torch.float32) for m in ms]
    cs = [dev(m.c, torch.float32) for m in ms]
    got = fem.build_K_batched(meshes, Xs, cs, "mixed")
    got = fem.build_K_batched(meshes, Xs, cs, "mixed")      # graph replay
    for mesh, X, c, g in zip(meshes, Xs, cs, got):
        assert torch.equal(g, mesh.build_K(X, c, "mixed"))
    small = sorted(range(len(ms)), key=lambda i: ms[i].n_elems)[:3]
    for i in small:
        m = ms[i]
        ref = oracle_K(m, m.X.astype(np.float32), m.c.astype(np.float32))
        assert rel_err(got[i].cpu().numpy(), ref["vals"], ref["cs"]) <= TOL_MIXED
    for mesh in meshes:
        mesh.close()


def test_27M_bricks_under_16GB_budget(fem):
    m = meshgen.config_mesh(4)
    assert m.n_elems == 27_000_000 and m.n_nodes == 27_270_901
    budget = 16 << 30
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), mem_budget_bytes=budget)
    nnz = mesh.pattern()
    assert nnz == ((3 * 300 + 1) ** 3 + 301 ** 3) // 2 == 379_351_801
    info = mesh.info()
    assert info["budget_bytes"] == budget
    rowptr, col = mesh.get_pattern()
    rp = rowptr.cpu().numpy()
    cl = col.cpu().numpy()
    rng = np.random.default_rng(27)
    sample = rng.choice(m.n_nodes, 2000, replace=False)
    for prec, dt, tol in (("mixed", torch.float32, TOL_MIXED), ("fp64", torch.float64, TOL_FP64)):
        Xh = m.X.astype(np.float32) if prec == "mixed" else m.X
        ch = m.c.astype(np.float32) if prec == "mixed" else m.c
        vals = mesh.build_K(dev(Xh, dt), dev(ch, dt), prec).cpu().numpy()
        ref = oracle_rows(m, sample, Xh, ch)
        worst = 0.0
        for r, (cols, v, cs) in ref.items():
            a, b = rp[r], rp[r + 1]
            assert np.array_equal(cl[a:b], cols)
            worst = max(worst, rel_err(vals[a:b], v, cs))
        assert worst <= tol, (prec, worst)
        del vals
    mesh.close()


def test_27M_bricks_in_groups_under_7GB(fem):
    """The 27M-brick workload under a 7 GB library budget, too small for the whole
    plan: the numeric build runs in two or more patch groups one after the other
    (Eq. 10), and sampled rows match the oracle."""
    m = meshgen.config_mesh(4)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), mem_budget_bytes=7 << 30)
    nnz = mesh.pattern()
    assert nnz == 379_351_801
    Xh, ch = m.X.astype(np.float32), m.c.astype(np.float32)
    vals = mesh.build_K(dev(Xh, torch.float32), dev(ch, torch.float32), "mixed")
    mesh.sync()
    info = mesh.info()
    assert info["n_groups"] >= 2 and info["peak_bytes"] <= 7 << 30
    vals = vals.cpu().numpy()
    rowptr, col = mesh.get_pattern()
    rp, cl = rowptr.cpu().numpy(), col.cpu().numpy()
    sample = np.random.default_rng(28).choice(m.n_nodes, 2000, replace=False)
    worst = 0.0
    for r, (cols, v, cs) in oracle_rows(m, sample, Xh, ch).items():
        a, b = rp[r], rp[r + 1]
        assert np.array_equal(cl[a:b], cols)
        worst = max(worst, rel_err(vals[a:b], v, cs))
    assert worst <= TOL_MIXED, worst
    mesh.close()
