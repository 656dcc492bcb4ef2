"""Genuinely unstructured inputs (the abstract's and Section 3's "unstructured
meshes"): Delaunay tetrahedralisations of seeded random points, whose node
valence, row lengths and colour counts vary from node to node, and brick grids
with geometrically graded spacing (cell sizes over a 50x range), at 10^4 to 10^5
elements, every value against the oracle in both precisions and both assemblies.
Also the library's limits on such meshes: the longest lower row (255 entries)
and the colour count (255) are reported against what these meshes reach, and a
mesh beyond them is refused cleanly."""
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


MESHES = {
    "delaunay_1e4": lambda: meshgen.delaunay_tets(1600),
    "delaunay_1e5": lambda: meshgen.delaunay_tets(15000, seed=meshgen.BASE_SEED + 12),
    "graded_24": lambda: meshgen.graded_bricks(24),
    "graded_40": lambda: meshgen.graded_bricks(40, ratio=100.0, seed=meshgen.BASE_SEED + 13),
}


@pytest.mark.parametrize("assembly", [0, 1], ids=["patches", "tiles"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(MESHES))
def test_unstructured_against_oracle(fem, name, prec, assembly):
    m = MESHES[name]()
    assert 1e4 <= m.n_elems <= 1.5e5
    mesh = fem.Mesh(dev(m.E, torch.int32), m.n_nodes, X=dev(m.X, torch.float64), assembly=assembly)
    X, c = rounded_inputs(m, prec)
    ref = oracle_K(m, X, c)
    nnz = mesh.pattern()
    assert nnz == ref["nnz"]
    rowptr, col = mesh.get_pattern()
    assert np.array_equal(rowptr.cpu().numpy(), ref["rowptr"])
    assert np.array_equal(col.cpu().numpy(), ref["col"])
    dt = torch.float64 if prec == "fp64" else torch.float32
    vals = mesh.build_K(dev(X, dt), dev(c, dt), prec)
    mesh.sync()
    err = rel_err(vals.cpu().numpy(), ref["vals"], ref["cs"])
    assert err <= (TOL_FP64 if prec == "fp64" else TOL_MIXED), err
    info = mesh.info()
    # how close these meshes come to the library's limits
    assert info["max_row_len"] <= 255 and info["n_colors"] <= 255
    print(f"{name} {prec} asm={assembly}: max lower row {info['max_row_len']} of 255, "
          f"colours {info['n_colors']} of 255, error {err:.2e}")


def fan(n_rim, seed=5):
    """Tetrahedra fanned around one centre node (the highest id): the Delaunay
    tetrahedralisation of n_rim seeded points on a sphere and its centre.  The
    centre's lower row holds n_rim + 1 entries and about 2 n_rim elements touch it."""
    from scipy.spatial import Delaunay
    u = meshgen.stream_uniform(seed, "fan", 2 * n_rim).reshape(-1, 2)
    z, phi = 2 * u[:, 0] - 1, 2 * np.pi * u[:, 1]
    r = np.sqrt(1 - z * z)
    P = np.vstack([np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1), np.zeros((1, 3))])
    E = Delaunay(P).simplices.astype(np.int32)
    return P, np.ascontiguousarray(E)


@pytest.mark.parametrize("n_rim,what", [(258, "row"), (300, "elements"), (140, "colours")])
def test_beyond_the_limits_is_refused(fem, n_rim, what):
    """A node whose lower row outgrows 255 entries, that more than 512 tetrahedra
    touch, or whose elements need more than 255 colours (more than 255 elements
    on one node), is refused with FEM_ERR_UNSUPPORTED and a message; nothing
    faults."""
    from paper_1501_04784_gb300 import abi
    P, E = fan(n_rim)
    center = P.shape[0] - 1
    assert (E == center).any(axis=1).sum() > 255
    mesh = fem.Mesh(dev(E, torch.int32), P.shape[0], X=dev(P, torch.float64))
    with pytest.raises(abi.FemError, match="FEM_ERR_UNSUPPORTED"):
        mesh.pattern()
    msg = abi.load().fem_last_error().decode()
    assert {"row": "255", "elements": "elements", "colours": "colours"}[what] in msg, msg


def test_fan_within_the_limits_matches_oracle(fem):
    """The same fan with 120 rim points (a 121-entry row, 236 elements at one node,
    236 colours) is inside the limits: pattern and values against the oracle."""
    P, E = fan(120)
    from types import SimpleNamespace
    m = SimpleNamespace(X=P, E=E, c=np.ones(E.shape[0]), npe=4, n_nodes=P.shape[0], n_elems=E.shape[0])
    mesh = fem.Mesh(dev(E, torch.int32), P.shape[0], X=dev(P, torch.float64))
    ref = oracle_K(m)
    assert mesh.pattern() == ref["nnz"]
    vals = mesh.build_K(dev(P, torch.float64), dev(m.c, torch.float64), "fp64").cpu().numpy()
    assert rel_err(vals, ref["vals"], ref["cs"]) <= TOL_FP64
    assert mesh.info()["max_row_len"] == 121
