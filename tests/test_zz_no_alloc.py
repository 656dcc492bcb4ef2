"""fem_pattern_noalloc: the pattern for callers that cannot allocate device memory.

Those callers (code under an external device-memory manager, plugins limited to
the buffers they are handed, streams that must stay free of allocation) get the
lower-CSR pattern from a call whose working memory is a fixed array inside the
library.  This file runs last (its name sorts last) so that a failure here
leaves every other test already run.  The checks compare the allocation-free
call with the handle-based fem_pattern / fem_get_pattern, bit for bit, on two
calls in a row (the second reuses the scratch left by the first)."""
import ctypes

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_04784_gb300 import _build, abi
    _build.build()
    return abi.load()


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


CASES = {
    "hex20_perm": lambda: meshgen.config_mesh(0),
    "tet10_perm": lambda: meshgen.config_mesh(2, nx=10),
    "hex_7x5x3": lambda: meshgen.hex_grid(7, 5, 3, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_pattern_matches_handle_pattern_twice(lib, name):
    from paper_1501_04784_gb300 import fem
    m = CASES[name]()
    E = torch.from_numpy(np.ascontiguousarray(m.E)).cuda()
    mesh = fem.Mesh(E, m.n_nodes)
    nnz = mesh.pattern()
    rp_ref, col_ref = mesh.get_pattern()
    torch.cuda.synchronize()
    for _ in range(2):
        rowptr = torch.full((m.n_nodes + 1,), -7, dtype=torch.int64, device="cuda")
        col = torch.full((nnz + 5,), -7, dtype=torch.int32, device="cuda")
        got = ctypes.c_int64(-1)
        st = lib.fem_pattern_noalloc(m.npe, m.n_nodes, m.n_elems, ptr(E), ptr(rowptr), ptr(col), nnz + 5,
                                     ctypes.byref(got), stream())
        assert st == 0, lib.fem_last_error()
        assert got.value == nnz
        assert torch.equal(rowptr, rp_ref)
        assert torch.equal(col[:nnz], col_ref)
        assert int(col[nnz:].eq(-7).sum()) == 5      # nothing written past nnz
    mesh.close()


def test_noalloc_reports_limits(lib):
    m = CASES["hex20_perm"]()
    E = torch.from_numpy(np.ascontiguousarray(m.E)).cuda()
    rowptr = torch.empty(m.n_nodes + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(16, dtype=torch.int32, device="cuda")
    got = ctypes.c_int64(-1)
    st = lib.fem_pattern_noalloc(8, m.n_nodes, m.n_elems, ptr(E), ptr(rowptr), ptr(col), 16, ctypes.byref(got),
                                 stream())
    assert st == 1 and got.value == 118121            # FEM_ERR_ARG, nnz still reported
    big = ctypes.c_int64(-1)
    st = lib.fem_pattern_noalloc(8, 10_000_000, 10_000_000, ptr(E), ptr(rowptr), ptr(col), 16, ctypes.byref(big),
                                 stream())
    assert st == 5 and b"scratch" in lib.fem_last_error()   # FEM_ERR_BUDGET, checked before any GPU work


@pytest.mark.parametrize("n,fits", [(64, True), (66, False)])
def test_noalloc_documented_size_limit(lib, n, fits):
    """The documented limit: a 64^3 brick grid fits the 16 MiB scratch, a 66^3 grid
    is refused with FEM_ERR_BUDGET before any GPU work."""
    m = meshgen.hex_grid(n, jitter=0.0, seed=1)
    E = torch.from_numpy(np.ascontiguousarray(m.E)).cuda()
    nnz_closed = ((3 * n + 1) ** 3 + (n + 1) ** 3) // 2
    rowptr = torch.empty(m.n_nodes + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(nnz_closed if fits else 16, dtype=torch.int32, device="cuda")
    got = ctypes.c_int64(-1)
    st = lib.fem_pattern_noalloc(8, m.n_nodes, m.n_elems, ptr(E), ptr(rowptr), ptr(col), col.numel(),
                                 ctypes.byref(got), stream())
    if fits:
        assert st == 0, lib.fem_last_error()
        assert got.value == nnz_closed
        assert int(rowptr[-1]) == nnz_closed
    else:
        assert st == 5 and b"scratch" in lib.fem_last_error()
