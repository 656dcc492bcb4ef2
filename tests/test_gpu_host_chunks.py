"""Host pipeline over row ranges (fem_options.host_chunks): the rows are split into
contiguous ranges, the node patches are planned inside them, and each range's
values leave the device while the next range is built (Section 4.3's overlap of
one group's transfer with the next group's integration).

Checked: the pipelined host build equals the device build of the same plan bit
for bit and the oracle within tolerance, for bricks and tetrahedra, both
precisions, the mass operator, more ranges than a small mesh has rows, under a
budget that also splits each range into patch groups (Eq. 10), through the
asynchronous entry point, and on a large brick mesh, where the library holds two
ranges of values on the device instead of K."""
import numpy as np
import pytest

import meshgen
from helpers import TOL_FP64, TOL_MIXED, oracle_K, oracle_rows, rel_err, rounded_inputs

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


def make(fem, m, **opts):
    return fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), **opts)


MESHES = {
    "hex_16x12x10": lambda: meshgen.hex_grid(16, 12, 10, jitter=0.25, seed=41, permute_nodes=True,
                                             permute_elems=True),
    "tet_8x7x6": lambda: meshgen.kuhn_tets(8, 7, 6, jitter=0.3, seed=42, permute_nodes=True, permute_elems=True),
}


def host_inputs(m, prec):
    X, c = rounded_inputs(m, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    return (torch.as_tensor(np.ascontiguousarray(X)).to(dt).pin_memory(),
            torch.as_tensor(np.ascontiguousarray(c)).to(dt).pin_memory(), X, c)


@pytest.mark.parametrize("chunks", [2, 7])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_pipelined_host_build(fem, name, prec, chunks):
    m = MESHES[name]()
    Xh, ch, X, c = host_inputs(m, prec)
    mesh = make(fem, m, host_chunks=chunks, patch_entries=512)
    nnz = mesh.pattern()
    got = mesh.build_K_host(Xh, ch, prec)
    info = mesh.info()
    assert info["n_chunks"] == chunks
    assert torch.equal(got, mesh.build_K(Xh.cuda(), ch.cuda(), prec).cpu())
    ref = oracle_K(m, X, c)
    assert nnz == ref["nnz"]
    assert rel_err(got.numpy(), ref["vals"], ref["cs"]) <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)


def test_pipelined_mass_matrix(fem):
    m = MESHES["hex_16x12x10"]()
    Xh, ch, X, c = host_inputs(m, "mixed")
    mesh = make(fem, m, host_chunks=3, operator_kind=1)
    mesh.pattern()
    got = mesh.build_K_host(Xh, ch, "mixed")
    ref = oracle_K(m, X, c, op="mass")
    assert rel_err(got.numpy(), ref["vals"], ref["cs"]) <= TOL_MIXED


def test_more_ranges_than_rows(fem):
    """A one-brick mesh (8 rows) asked for 50 ranges gets one range per row."""
    m = meshgen.hex_grid(1, 1, 1, jitter=0.1, seed=3)
    Xh, ch, X, c = host_inputs(m, "fp64")
    mesh = make(fem, m, host_chunks=50)
    mesh.pattern()
    got = mesh.build_K_host(Xh, ch, "fp64")
    assert mesh.info()["n_chunks"] == 8
    ref = oracle_K(m, X, c)
    assert rel_err(got.numpy(), ref["vals"], ref["cs"]) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pipelined_under_budget_in_groups(fem, prec):
    """A budget too small for every closure at once: each range runs in patch
    groups whose closures are built per call; values still match the oracle and
    the device build of the same mesh, and the peak stays within the budget."""
    m = meshgen.hex_grid(24, 20, 16, jitter=0.25, seed=43, permute_nodes=True, permute_elems=True)
    Xh, ch, X, c = host_inputs(m, prec)
    free = make(fem, m, host_chunks=4, patch_entries=512)
    nnz = free.pattern()
    need = free.info()["plan_bytes"]
    free.close()
    w = 8 if prec == "fp64" else 4
    budget = int(need * 0.6) + Xh.numel() * w + ch.numel() * w + nnz * w // 2 + (64 << 10)
    mesh = make(fem, m, host_chunks=4, patch_entries=512, mem_budget_bytes=budget)
    mesh.pattern()
    got = mesh.build_K_host(Xh, ch, prec)
    info = mesh.info()
    assert info["n_groups"] >= 2 and info["n_chunks"] == 4
    assert info["peak_bytes"] <= budget
    assert torch.equal(got, mesh.build_K(Xh.cuda(), ch.cuda(), prec).cpu())
    ref = oracle_K(m, X, c)
    assert rel_err(got.numpy(), ref["vals"], ref["cs"]) <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)


def test_pipelined_async_calls(fem):
    """Consecutive asynchronous pipelined builds with different coefficients on two
    streams taken in turn: each output equals its own synchronous build."""
    m = MESHES["tet_8x7x6"]()
    Xh, ch, X, c = host_inputs(m, "mixed")
    mesh = make(fem, m, host_chunks=5)
    nnz = mesh.pattern()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cs = [(ch * (1.0 + 0.25 * k)).pin_memory() for k in range(4)]
    outs = [torch.empty(nnz, dtype=torch.float32).pin_memory() for _ in cs]
    for k, (cc, o) in enumerate(zip(cs, outs)):
        mesh.build_K_host_async(Xh, cc, "mixed", out=o, stream=streams[k % 2])
    for st in streams:
        st.synchronize()
    mesh.sync()
    for cc, o in zip(cs, outs):
        assert torch.equal(o, mesh.build_K_host(Xh, cc, "mixed"))


def test_large_bricks_two_ranges_of_values_on_device(fem):
    """80^3 bricks (the 27M-brick recipe at 512k elements), 8 ranges: the pipelined
    host build adds the inputs and two ranges of FP32 values to the library's
    device memory, where the plain host build adds the inputs and all of K's
    values; sampled rows match the oracle, and the result equals the device build
    of the same plan."""
    m = meshgen.config_mesh(4, nx=80)
    Xh, ch, X, c = host_inputs(m, "mixed")
    inputs = Xh.numel() * 4 + ch.numel() * 4
    whole = make(fem, m)
    nnz = whole.pattern()
    before = whole.info()["live_bytes"]
    whole.build_K_host(Xh, ch, "mixed")
    assert whole.info()["live_bytes"] - before >= inputs + nnz * 4
    whole.close()
    mesh = make(fem, m, host_chunks=8)
    mesh.pattern()
    before = mesh.info()["live_bytes"]
    got = mesh.build_K_host(Xh, ch, "mixed")
    assert mesh.info()["live_bytes"] - before <= inputs + nnz * 4 // 3 + 4096
    assert torch.equal(got, mesh.build_K(Xh.cuda(), ch.cuda(), "mixed").cpu())
    rowptr, col = mesh.get_pattern()
    rp, cl = rowptr.cpu().numpy(), col.cpu().numpy()
    sample = np.random.default_rng(44).choice(m.n_nodes, 500, replace=False)
    vals = got.numpy()
    worst = 0.0
    for r, (cols, v, cs) in oracle_rows(m, sample, X, c).items():
        a, b = rp[r], rp[r + 1]
        assert np.array_equal(cl[a:b], cols)
        worst = max(worst, rel_err(vals[a:b], v, cs))
    assert worst <= TOL_MIXED, worst
