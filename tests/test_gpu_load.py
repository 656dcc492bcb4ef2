"""Global load vector F = sum_e src_e int N (Section 1's f_e and F) on the GPU against
the oracle's load vector (pinned in test_oracle_load_pins.py), and against the GPU's
own mass matrix (F = M 1 when src = c)."""
import numpy as np
import pytest

import meshgen
from helpers import TOL_FP64, TOL_MIXED, rounded_inputs

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


MESHES = {
    "hex20_perm": lambda: meshgen.config_mesh(0),
    "tet10_perm": lambda: meshgen.config_mesh(2, nx=10),
    "hex_7x5x3": lambda: meshgen.hex_grid(7, 5, 3, jitter=0.25, seed=5, permute_nodes=True, permute_elems=True),
}


def source(m, seed=3):
    """A signed per-element source (so that entries can cancel)."""
    return np.random.default_rng(seed).standard_normal(m.E.shape[0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_load_vector_against_oracle(fem, oracle_lib, name, prec):
    m = MESHES[name]()
    s = source(m)
    X, _ = rounded_inputs(m, prec)
    s_in = s.astype(np.float32) if prec == "mixed" else s
    dt = torch.float32 if prec == "mixed" else torch.float64
    ref = oracle_lib.load_vector(m.npe, X, m.E, s_in)
    scale = oracle_lib.load_vector(m.npe, X, m.E, np.abs(s_in))   # sum of |contributions| per node
    for cap in (0, 64):
        mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), patch_entries=cap)
        F = mesh.load_vector(dev(X, dt), dev(s_in, dt), prec).cpu().numpy()
        err = np.max(np.abs(F - ref) / scale)
        assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), (cap, err)


def test_load_vector_equals_mass_row_sums(fem):
    """src = c: F = M 1 with M the GPU's own mass matrix (both FP64)."""
    m = MESHES["hex_7x5x3"]()
    Xd, cd = dev(m.X, torch.float64), dev(m.c, torch.float64)
    E = dev(m.E, torch.int32)
    F = fem.Mesh(E, m.n_nodes, X=Xd).load_vector(Xd, cd, "fp64").cpu().numpy()
    mm = fem.Mesh(E, m.n_nodes, X=Xd, operator_kind=1)
    vals = mm.build_K(Xd, cd, "fp64").cpu().numpy()
    rp, col = (t.cpu().numpy() for t in mm.get_pattern())
    Mu = np.zeros(m.n_nodes)
    rows = np.repeat(np.arange(m.n_nodes), np.diff(rp))
    np.add.at(Mu, rows, vals)
    off = col != rows
    np.add.at(Mu, col[off], vals[off])
    assert np.max(np.abs(F - Mu)) <= 1e-13 * np.max(np.abs(Mu))


def test_load_vector_budget_groups_bitwise(fem):
    """Patch groups under a memory budget (Eq. 10) give the same F bit for bit."""
    m = meshgen.config_mesh(0)
    Xd, sd = dev(m.X.astype(np.float32), torch.float32), dev(source(m).astype(np.float32), torch.float32)
    E = dev(m.E, torch.int32)
    full = fem.Mesh(E, m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512)
    a = full.load_vector(Xd, sd, "mixed")
    need = full.info()["plan_bytes"]
    small = fem.Mesh(E, m.n_nodes, X=dev(m.X, torch.float64), patch_entries=512, mem_budget_bytes=int(need * 0.75))
    b = small.load_vector(Xd, sd, "mixed")
    assert small.info()["n_groups"] > 1
    assert torch.equal(a, b)
