"""Full-size parity against the oracle: the 1M-brick workload (mixed and FP64)
and the 3.07M-tetrahedron workload (mixed), every row pointer, every column
index and every value of the lower CSR compared with the oracle's complete build
(Algorithm 1 with the sparse conversion of Section 3, in FP64).  The oracle runs
on the host in about 12 s per workload and precision.

Also the other paths to K's values against the oracle: builds under a memory
budget too small for the whole plan (the Eq. 10 groups) and builds that write K
straight into page-locked host memory, in both precisions."""
import numpy as np
import pytest

import meshgen
from helpers import TOL_FP64, TOL_MIXED, oracle_K, rel_err, rounded_inputs

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


def plain_rel(got, ref, scale, floor=1e-3):
    """Plain relative error on the entries that do not cancel (|K*| >= floor * scale)."""
    keep = np.abs(ref) >= floor * scale
    got = np.asarray(got, np.float64)
    return float(np.max(np.abs(got[keep] - ref[keep]) / np.abs(ref[keep]))) if keep.any() else 0.0


@pytest.mark.parametrize("cfg,precs", [(1, ("mixed", "fp64")), (2, ("mixed",))],
                         ids=["1M_bricks", "3.07M_tets"])
def test_full_size_pattern_and_values(fem, cfg, precs):
    m = meshgen.config_mesh(cfg)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64))
    tiles = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), assembly=1)
    nnz = mesh.pattern()
    assert tiles.pattern() == nnz and tiles.info()["assembly"] == 1
    rowptr, col = mesh.get_pattern()
    rowptr, col = rowptr.cpu().numpy(), col.cpu().numpy()
    for prec in precs:
        X, c = rounded_inputs(m, prec)
        ref = oracle_K(m, X, c)
        assert nnz == ref["nnz"]
        assert np.array_equal(rowptr, ref["rowptr"])          # every row pointer
        assert np.array_equal(col, ref["col"])                # every column index
        dt = torch.float64 if prec == "fp64" else torch.float32
        # the element-tile assembly of the same mesh, every value
        tv = tiles.build_K(dev(X, dt), dev(c, dt), prec)
        tiles.sync()
        terr = rel_err(tv.cpu().numpy(), ref["vals"], ref["cs"])
        assert terr <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), (prec, "tiles", terr)
        del tv
        vals = mesh.build_K(dev(X, dt), dev(c, dt), prec)
        mesh.sync()
        vals = vals.cpu().numpy()
        err = rel_err(vals, ref["vals"], ref["cs"])           # every value
        assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), (prec, err)
        # 2,000 sampled rows, each row checked on its own
        rng = np.random.default_rng(300 + cfg)
        worst = 0.0
        for r in rng.choice(m.n_nodes, 2000, replace=False):
            a, b = rowptr[r], rowptr[r + 1]
            worst = max(worst, rel_err(vals[a:b], ref["vals"][a:b], ref["cs"][a:b]))
        assert worst <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)
        # the plain relative error of the entries that do not cancel, and the error
        # against the sum of |contributions| of each entry, are reported
        print(f"cfg{cfg} {prec}: scaled {err:.3e}  vs |contrib| "
              f"{rel_err(vals, ref['vals'], ref['abs']):.3e}  plain (|K| >= 1e-3 scale) "
              f"{plain_rel(vals, ref['vals'], ref['cs']):.3e}")
        del ref, vals
    mesh.close()
    tiles.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_budget_groups_match_oracle(fem, prec):
    """A budget too small for all patch closures at once: the build runs on
    patches in groups (Eq. 10), one group after the other, and matches the
    oracle."""
    m = meshgen.hex_grid(24, jitter=0.2, seed=77, permute_nodes=True, permute_elems=True)
    X, c = rounded_inputs(m, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    free = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=1024)
    free.pattern()
    need = free.info()["plan_bytes"]
    tight = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=1024,
                     mem_budget_bytes=int(need * 0.75), fp64_fused=1)
    vals = tight.build_K(dev(X, dt), dev(c, dt), prec)
    tight.sync()
    info = tight.info()
    assert info["n_groups"] > 1 and info["assembly"] == 0
    ref = oracle_K(m, X, c)
    err = rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"])
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err


@pytest.mark.parametrize("assembly", [0, 1], ids=["patches", "tiles"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["hex20_perm", "tet10_perm"])
def test_host_resident_matches_oracle(fem, name, prec, assembly):
    """K written by the kernels straight into page-locked host memory
    (host_direct): every value against the oracle."""
    m = meshgen.config_mesh(0) if name == "hex20_perm" else meshgen.config_mesh(2, nx=10)
    X, c = rounded_inputs(m, prec)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), host_direct=1, assembly=assembly)
    mesh.pattern()
    assert mesh.info()["assembly"] == assembly
    hv = mesh.build_K_host(torch.from_numpy(np.ascontiguousarray(X)).pin_memory(),
                           torch.from_numpy(np.ascontiguousarray(c)).pin_memory(), prec).numpy()
    ref = oracle_K(m, X, c)
    err = rel_err(hv, ref["vals"], ref["cs"])
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err
