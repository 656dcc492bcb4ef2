"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Pattern and row pointers must be bit-exact; values within 1e-12 (FP64) or
1e-5 (mixed) of the oracle, relative to each entry's Cauchy-Schwarz scale (see
helpers.py).  Sizes span many thread-block patches and ragged tails; small
patch capacities force hundreds of patches on small meshes.
"""
import numpy as np
import pytest

import meshgen
from helpers import TOL_FP64, TOL_MIXED, oracle_K, oracle_ke, oracle_rows, rel_err, rounded_inputs

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
    E = dev(m.E, torch.int32)
    mesh = fem.Mesh(E, m.n_nodes, X=dev(m.X, torch.float64), **opts)
    return mesh


def inputs(m, prec):
    X, c = rounded_inputs(m, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    return dev(X, dt), dev(c, dt), X, c


MESHES = {
    "hex20_perm": lambda: meshgen.config_mesh(0),
    "hex_7x5x3": lambda: meshgen.hex_grid(7, 5, 3, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True),
    "hex_1x1x1": lambda: meshgen.hex_grid(1, 1, 1, jitter=0.0, seed=1),
    "tet10_perm": lambda: meshgen.config_mesh(2, nx=10),
    "tet_6x4x3": lambda: meshgen.kuhn_tets(6, 4, 3, jitter=0.3, seed=2, permute_nodes=True, permute_elems=True),
}
PATCH_CAPS = {"default": 0, "tiny": 64}
# the two assemblies of the scalar operators: node patches (default) and element
# tiles (each element integrated once, border rows summed from tile partials);
# tiny tiles make most rows border rows
ASSEMBLIES = {"patches": {}, "tiles": dict(assembly=1), "tiles_tiny": dict(assembly=1, tile_elems=8)}


@pytest.mark.parametrize("cap", list(PATCH_CAPS))
@pytest.mark.parametrize("name", list(MESHES))
def test_pattern_bit_exact(fem, name, cap):
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=PATCH_CAPS[cap])
    ref = oracle_K(m)
    nnz = mesh.pattern()
    assert nnz == ref["nnz"]
    rowptr, col = mesh.get_pattern()
    assert np.array_equal(rowptr.cpu().numpy(), ref["rowptr"])
    assert np.array_equal(col.cpu().numpy(), ref["col"])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex20_perm", "tet10_perm", "hex_7x5x3"])
def test_integrate_local(fem, name, prec):
    m = MESHES[name]()
    mesh = make(fem, m)
    Xd, cd, X, c = inputs(m, prec)
    ke = mesh.integrate_local(Xd, cd, prec).cpu().numpy()
    ref, cs, _ = oracle_ke(m, X, c)
    err = rel_err(ke.ravel(), ref.ravel(), cs.ravel())
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err


@pytest.mark.parametrize("cap", list(PATCH_CAPS))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_build_K(fem, name, prec, cap):
    m = MESHES[name]()
    mesh = make(fem, m, patch_entries=PATCH_CAPS[cap])
    Xd, cd, X, c = inputs(m, prec)
    ref = oracle_K(m, X, c)
    vals = mesh.build_K(Xd, cd, prec).cpu().numpy()
    err = rel_err(vals, ref["vals"], ref["cs"])
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err


@pytest.mark.parametrize("asm", ["tiles", "tiles_tiny"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_build_K_tiles(fem, name, prec, asm):
    """The element-tile assembly: every value against the oracle, the same build
    twice bitwise equal, and the same values from any block size (the plan fixes
    every sum's order)."""
    m = MESHES[name]()
    mesh = make(fem, m, **ASSEMBLIES[asm])
    Xd, cd, X, c = inputs(m, prec)
    ref = oracle_K(m, X, c)
    nnz = mesh.pattern()
    assert mesh.info()["assembly"] == 1
    assert nnz == ref["nnz"]
    vals = mesh.build_K(Xd, cd, prec)
    err = rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"])
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err
    assert torch.equal(vals, mesh.build_K(Xd, cd, prec))
    other = make(fem, m, block_threads=128, **ASSEMBLIES[asm])
    assert torch.equal(vals, other.build_K(Xd, cd, prec))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["hex20_perm", "tet10_perm"])
def test_assemble_given_ke(fem, name, prec):
    """fem_assemble_csr of the oracle's own element matrices: only the summation
    order differs from the oracle's sparse conversion."""
    m = MESHES[name]()
    mesh = make(fem, m)
    mesh.pattern()
    ke, cs, _ = oracle_ke(m)
    dt = torch.float64 if prec == "fp64" else torch.float32
    vals = mesh.assemble_csr(dev(ke, dt), prec).cpu().numpy()
    ref = oracle_K(m)
    tol = 1e-14 if prec == "fp64" else 3e-7
    assert rel_err(vals, ref["vals"], ref["cs"]) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bitwise_reproducible_across_launch_shapes(fem, prec):
    m = MESHES["hex20_perm"]()
    Xd, cd, _, _ = inputs(m, prec)
    outs = []
    for threads, bps in ((256, 0), (256, 0), (128, 1), (512, 1), (64, 3)):
        mesh = make(fem, m, block_threads=threads, blocks_per_sm=bps, patch_entries=2048)
        outs.append(mesh.build_K(Xd, cd, prec).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint8), outs[0].view(np.uint8))


def test_host_entry_point_matches_device(fem):
    m = MESHES["tet10_perm"]()
    mesh = make(fem, m)
    Xd, cd, X, c = inputs(m, "mixed")
    dv = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
    hv = mesh.build_K_host(torch.from_numpy(np.ascontiguousarray(X)).pin_memory(),
                           torch.from_numpy(np.ascontiguousarray(c)).pin_memory(), "mixed").numpy()
    assert np.array_equal(dv, hv)


def test_isolated_nodes_and_single_element(fem):
    m = meshgen.hex_grid(1, 1, 1, seed=3)
    E = dev(m.E, torch.int32)
    mesh = fem.Mesh(E, m.n_nodes + 5)           # 5 nodes that no element uses
    nnz = mesh.pattern()
    assert nnz == 36
    rowptr, col = mesh.get_pattern()
    assert np.array_equal(rowptr.cpu().numpy()[-6:], np.full(6, 36))
    X = np.vstack([m.X, np.zeros((5, 3))])
    vals = mesh.build_K(dev(X, torch.float64), dev(m.c, torch.float64), "fp64").cpu().numpy()
    ref = oracle_K(m)
    assert rel_err(vals, ref["vals"], ref["cs"]) <= TOL_FP64


def test_error_statuses(fem):
    from paper_1501_04784_gb300 import abi
    m = meshgen.hex_grid(2, seed=3)
    E = m.E.copy()
    E[1, 3] = m.n_nodes + 7
    with pytest.raises(abi.FemError, match="FEM_ERR_INDEX"):
        fem.Mesh(dev(E, torch.int32), m.n_nodes)
    E = m.E.copy()
    E[2, 5] = E[2, 1]
    with pytest.raises(abi.FemError, match="FEM_ERR_DEGENERATE"):
        fem.Mesh(dev(E, torch.int32), m.n_nodes)
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes)
    vals = torch.empty(1000, dtype=torch.float64, device="cuda")
    L = abi.load()
    import ctypes
    st = L.fem_build_K(mesh.handle, 0, ctypes.c_void_p(dev(m.X, torch.float64).data_ptr()), 1,
                       ctypes.c_void_p(dev(m.c, torch.float64).data_ptr()), 1, ctypes.c_void_p(vals.data_ptr()), None)
    assert abi.STATUS[st] == "FEM_ERR_STATE"
    small = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, mem_budget_bytes=1024)
    with pytest.raises(abi.FemError, match="FEM_ERR_BUDGET"):
        small.pattern()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_1M_bricks_sampled(fem, prec):
    """The 1M-brick workload at full size: pattern checked against the closed-form
    nnz and structural invariants, values of sampled rows against the oracle."""
    m = meshgen.config_mesh(1)
    mesh = make(fem, m)
    nnz = mesh.pattern()
    assert nnz == ((3 * 100 + 1) ** 3 + 101 ** 3) // 2 == 14150601
    rowptr, col = mesh.get_pattern()
    rp = rowptr.cpu().numpy()
    cl = col.cpu().numpy()
    assert np.all(np.diff(rp) >= 1)
    last = cl[rp[1:] - 1]
    assert np.array_equal(last, np.arange(m.n_nodes))      # diagonal is the last entry of each row
    Xd, cd, X, c = inputs(m, prec)
    vals = mesh.build_K(Xd, cd, prec).cpu().numpy()
    rng = np.random.default_rng(12)
    sample = rng.choice(m.n_nodes, 3000, replace=False)
    ref = oracle_rows(m, sample, X, c)
    worst = 0.0
    for r, (cols, v, cs) in ref.items():
        a, b = rp[r], rp[r + 1]
        assert np.array_equal(cl[a:b], cols)
        worst = max(worst, rel_err(vals[a:b], v, cs))
    assert worst <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), worst


def sliver_tets(n=64, lift=1e-4, seed=7):
    """n separate slivers: a unit right triangle and a fourth node `lift` above a
    point inside it, each randomly rotated and shifted, so that the Jacobian
    determinant is a heavily cancelling sum of products of the FP32 edge
    vectors (a plain FP32 evaluation is off by ~1e-4 relative)."""
    rng = np.random.default_rng(seed)
    P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.3, lift]], float)
    X, E = [], []
    for t in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        X.append(P @ Q.T + rng.normal(size=3))
        E.append([4 * t, 4 * t + 1, 4 * t + 2, 4 * t + 3])
    return meshgen.Mesh(X=np.vstack(X), E=np.asarray(E, np.int32), c=rng.lognormal(0, 0.5, n), npe=4,
                        shape=(n, 1, 1))


@pytest.mark.parametrize("fp64_dets", [0, 1])
def test_distorted_tet_determinant_modes(fem, fp64_dets):
    """Distorted tetrahedra take an FP64-accurate determinant, in double-single
    FP32 arithmetic (default) or in FP64: slivers far beyond a plain FP32
    determinant's reach still meet the mixed tolerance, element by element and
    assembled, and so does the 80^3-cell tetrahedron recipe at 10^3 cells."""
    m = sliver_tets()
    mesh = make(fem, m, fp64_dets=fp64_dets)
    Xd, cd, X, c = inputs(m, "mixed")
    ke = mesh.integrate_local(Xd, cd, "mixed").cpu().numpy()
    ref, cs, _ = oracle_ke(m, X, c)
    assert rel_err(ke.ravel(), ref.ravel(), cs.ravel()) <= TOL_MIXED
    refK = oracle_K(m, X, c)
    vals = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
    assert rel_err(vals, refK["vals"], refK["cs"]) <= TOL_MIXED
    m = MESHES["tet10_perm"]()
    mesh = make(fem, m, fp64_dets=fp64_dets)
    Xd, cd, X, c = inputs(m, "mixed")
    refK = oracle_K(m, X, c)
    vals = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
    assert rel_err(vals, refK["vals"], refK["cs"]) <= TOL_MIXED


def test_device_wait_timeout_is_reported(fem):
    """Failure detection without a fault: with debug_stall, warp 0 of every block
    waits (at most wait_spins polls) for a colour phase that cannot complete.
    The wait gives up, the kernel still finishes, fem_sync reports
    FEM_ERR_TIMEOUT once, and the context stays usable: a later build is
    correct."""
    from paper_1501_04784_gb300 import abi
    m = MESHES["hex_7x5x3"]()
    Xd, cd, X, c = inputs(m, "mixed")
    stalled = make(fem, m, debug_stall=1, wait_spins=64)
    stalled.build_K(Xd, cd, "mixed")
    with pytest.raises(abi.FemError, match="FEM_ERR_TIMEOUT"):
        stalled.sync()
    stalled.sync()   # the status word was cleared
    ok = make(fem, m)
    vals = ok.build_K(Xd, cd, "mixed")
    ok.sync()
    ref = oracle_K(m, X, c)
    assert rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"]) <= TOL_MIXED


@pytest.mark.parametrize("fp64_sums", [0, 1])
def test_high_valence_summation_modes(fem, fp64_sums):
    """Tet diagonals (up to 24 contributions) are summed FP64-accurately either by
    FP32 TwoSum pairs (default) or by FP64 adds; both round once to FP32."""
    m = MESHES["tet10_perm"]()
    mesh = make(fem, m, fp64_sums=fp64_sums)
    Xd, cd, X, c = inputs(m, "mixed")
    ref = oracle_K(m, X, c)
    vals = mesh.build_K(Xd, cd, "mixed").cpu().numpy()
    assert rel_err(vals, ref["vals"], ref["cs"]) <= TOL_MIXED
    rp = ref["rowptr"]
    diag = rp[1:] - 1
    # the diagonal sum itself: within a few FP32 roundings of the exact sum
    d_err = np.abs(vals[diag].astype(np.float64) - ref["vals"][diag]) / ref["cs"][diag]
    assert d_err.max() <= 4e-7


@pytest.mark.parametrize("n_streams", [1, 2, 3, 4])
def test_host_async_streams(fem, n_streams):
    """fem_build_K_host_async on streams taken in turn, through the mesh's three
    staging slots (more steps than slots, so every slot is reused): every step's
    values equal the device build's, and pageable buffers are refused."""
    from paper_1501_04784_gb300 import abi
    m = MESHES["hex_7x5x3"]()
    mesh = make(fem, m)
    Xd, cd, X, c = inputs(m, "mixed")
    ref = mesh.build_K(Xd, cd, "mixed").cpu()
    Xh, ch = Xd.cpu().pin_memory(), cd.cpu().pin_memory()
    scale = [1.0, 1.5, 2.0, 0.5, 3.0, 0.25, 1.25]
    outs = [torch.empty(mesh.nnz, dtype=torch.float32).pin_memory() for _ in scale]
    cs = [(ch * s).pin_memory() for s in scale]
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    for k, s in enumerate(scale):
        mesh.build_K_host_async(Xh, cs[k], "mixed", out=outs[k], stream=streams[k % n_streams])
    torch.cuda.synchronize()
    mesh.sync()
    for k, s in enumerate(scale):
        want = mesh.build_K(Xd, (cd * s).contiguous(), "mixed").cpu()
        assert torch.equal(outs[k], want)
    assert torch.equal(outs[0], ref)
    with pytest.raises(abi.FemError, match="FEM_ERR_ARG"):
        mesh.build_K_host_async(Xd.cpu(), cd.cpu(), "mixed")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_zero_volume_element_is_reported(fem, prec):
    """A brick flattened to zero volume has no finite element matrix: the build
    finishes, fem_sync reports FEM_ERR_DEGENERATE once (status cleared), and a
    valid build on the same context afterwards is correct."""
    from paper_1501_04784_gb300 import abi
    m = MESHES["hex_7x5x3"]()
    X = m.X.copy()
    e0 = m.E[0]
    X[e0, 2] = X[e0[0], 2]             # all 8 nodes of element 0 in one z plane
    bad = make(fem, m)
    dt = torch.float32 if prec == "mixed" else torch.float64
    bad.build_K(dev(X, dt), dev(m.c, dt), prec)
    with pytest.raises(abi.FemError, match="FEM_ERR_DEGENERATE"):
        bad.sync()
    bad.sync()
    Xd, cd, Xr, c = inputs(m, prec)
    vals = bad.build_K(Xd, cd, prec)
    bad.sync()
    ref = oracle_K(m, Xr, c)
    assert rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"]) <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_host_resident_K(fem, prec):
    """K written by the kernel straight into page-locked host memory (host_direct):
    equal to the device build bit for bit; a pageable output is refused."""
    from paper_1501_04784_gb300 import abi
    m = meshgen.hex_grid(24, 20, 16, jitter=0.25, seed=31, permute_nodes=True, permute_elems=True)
    Xd, cd, X, c = inputs(m, prec)
    ref = make(fem, m, fp64_fused=1).build_K(Xd, cd, prec)
    Xh, ch = Xd.cpu().pin_memory(), cd.cpu().pin_memory()
    direct = make(fem, m, host_direct=1, fp64_fused=1)
    out = torch.empty(ref.numel(), dtype=ref.dtype).pin_memory()
    assert torch.equal(direct.build_K_host(Xh, ch, prec, out=out), ref.cpu())
    with pytest.raises(abi.FemError, match="FEM_ERR_ARG"):
        direct.build_K_host(Xh, ch, prec, out=torch.empty(ref.numel(), dtype=ref.dtype))   # pageable


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_host_resident_K_under_budget(fem, prec):
    """A memory budget with room for the symbolic phase, the plan and the inputs
    but not for K's values (the 3N x 3N elasticity matrix, whose values outweigh the
    symbolic phase's scratch): fem_build_K_host writes them straight into the
    page-locked host buffer by itself, never exceeds the budget, and equals the
    device build."""
    m = meshgen.hex_grid(24, 20, 16, jitter=0.25, seed=31, permute_nodes=True, permute_elems=True)
    dt = torch.float32 if prec == "mixed" else torch.float64
    lame = meshgen.lame(m)
    Xd, cd = dev(m.X, dt), dev(lame, dt)

    def el(**o):
        return fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), operator_kind=2,
                        fp64_fused=1, **o)
    ref = el().build_K(Xd, cd, prec)
    probe = el()
    probe.pattern()
    info = probe.info()
    vbytes = ref.numel() * ref.element_size()
    inputs_bytes = Xd.numel() * Xd.element_size() + cd.numel() * cd.element_size() + 512
    budget = max(info["peak_bytes"], info["live_bytes"] + inputs_bytes) + vbytes // 4
    assert info["live_bytes"] + inputs_bytes + vbytes > budget
    tight = el(mem_budget_bytes=budget)
    out = torch.empty(ref.numel(), dtype=ref.dtype).pin_memory()
    got = tight.build_K_host(Xd.cpu().pin_memory(), cd.cpu().pin_memory(), prec, out=out)
    assert torch.equal(got, ref.cpu())
    assert tight.info()["peak_bytes"] <= budget
