"""Seeded synthetic meshes for the global stiffness-matrix build.

This module produces the inputs of the method -- node coordinates X, element
connectivity E and the per-element coefficient c (the arrays C, E and MP of
Section 3) -- and nothing else.  It holds none of the method's arithmetic: no
shape functions, Jacobians, element matrices or assembly.  Both the oracle
tests and the CUDA tests draw their inputs from here.

Workloads follow the paper's cubic-domain meshes (Section 3, Table 2: an
n x n x n grid of 8-node bricks on the unit cube) with the distortions and
orderings of the benchmark configurations:

* ``hex_grid``  -- structured brick grid, interior-node jitter, optional random
  node / element numbering, c_e laws;
* ``kuhn_tets`` -- the same grid with every cell split into 6 tetrahedra along
  its main diagonal;
* ``delaunay_tets`` -- genuinely unstructured tetrahedra: the Delaunay
  tetrahedralisation of seeded uniform random points in the unit cube;
* ``graded_bricks`` -- a brick grid whose spacing grows geometrically along each
  axis (cell sizes spanning a stated ratio), with interior-node jitter;
* ``batch_specs`` -- grid shapes for a batch of uneven meshes;
* ``lame`` -- per-element Lame parameters (lambda, mu) for the elasticity
  operator: Young's modulus c_e and a seeded Poisson ratio per element.

Randomness is counter-based SplitMix64 (Steele, Lea & Flood 2014): value i of
stream (seed, name) is mix(key + (i + 1) * 0x9E3779B97F4A7C15), so every draw
is reproducible from (seed, name, i) alone, on any platform.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 150104784
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Natural coordinates of the 8 brick nodes: nodes 0-3 on the face t = -1,
# counter-clockwise from (-1,-1,-1); nodes 4-7 the same on t = +1.
HEX_NODE_OFFSETS = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _name_key(name: str) -> np.uint64:
    h = 0xCBF29CE484222325  # FNV-1a 64 over the stream name
    for ch in name.encode():
        h = ((h ^ ch) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(h)


def stream_u64(seed: int, name: str, n: int, offset: int = 0) -> np.ndarray:
    """n raw 64-bit draws of stream (seed, name), starting at draw ``offset``."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([np.uint64(seed) ^ _name_key(name)], dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(key + ctr * GOLDEN)


def stream_uniform(seed: int, name: str, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (stream_u64(seed, name, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def stream_normal(seed: int, name: str, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on two uniform streams."""
    u1 = ((stream_u64(seed, name + "/u1", n) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = stream_uniform(seed, name + "/u2", n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def stream_permutation(seed: int, name: str, n: int) -> np.ndarray:
    """A uniformly random permutation of range(n) (stable sort of random keys)."""
    return np.argsort(stream_u64(seed, name, n), kind="stable").astype(np.int64)


@dataclass
class Mesh:
    """A mesh as the method consumes it (Section 3: arrays C, E, MP)."""
    X: np.ndarray            # [n_nodes, 3] float64 node coordinates
    E: np.ndarray            # [n_elems, npe] int32 connectivity (global node ids)
    c: np.ndarray            # [n_elems] float64 per-element coefficient
    npe: int                 # nodes per element: 8 (brick) or 4 (tetrahedron)
    shape: tuple             # grid cells (nx, ny, nz)
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.E.shape[0])


def _grid_nodes(nx: int, ny: int, nz: int) -> np.ndarray:
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # node id = i + (nx+1) * (j + (ny+1) * k)
    ijk = np.stack([i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")], axis=1)
    return ijk.astype(np.int64)


def _node_id(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def _jittered_coords(nx, ny, nz, jitter, seed):
    ijk = _grid_nodes(nx, ny, nz)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    X = ijk.astype(np.float64) * h
    if jitter > 0.0:
        interior = ((ijk > 0) & (ijk < np.array([nx, ny, nz]))).all(axis=1)
        u = stream_uniform(seed, "jitter", 3 * X.shape[0]).reshape(-1, 3)
        X = X + np.where(interior[:, None], (2.0 * u - 1.0) * jitter * h, 0.0)
    return X


def _cells(nx, ny, nz):
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return np.stack([ci.ravel(order="F"), cj.ravel(order="F"), ck.ravel(order="F")], axis=1).astype(np.int64)


def _c_lognormal(seed, n, sigma):
    return np.exp(sigma * stream_normal(seed, "c", n))


def _c_subboxes(seed, centroids, lo=1e-2, hi=1e2):
    """c piecewise constant over 8 boxes cut at seeded planes in [0.25, 0.75]."""
    planes = 0.25 + 0.5 * stream_uniform(seed, "c/planes", 3)
    vals = np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * stream_uniform(seed, "c/boxes", 8))
    b = (centroids > planes).astype(np.int64)
    return vals[b[:, 0] + 2 * b[:, 1] + 4 * b[:, 2]]


def _renumber(X, E, c, seed, permute_nodes, permute_elems):
    if permute_nodes:
        p = stream_permutation(seed, "node_perm", X.shape[0])  # new id of old node
        Xn = np.empty_like(X)
        Xn[p] = X
        X, E = Xn, p[E]
    if permute_elems:
        q = stream_permutation(seed, "elem_perm", E.shape[0])  # old element at new slot
        E, c = E[q], c[q]
    return X, np.ascontiguousarray(E, dtype=np.int32), np.ascontiguousarray(c, dtype=np.float64)


def hex_grid(nx: int, ny: int | None = None, nz: int | None = None, *, jitter: float = 0.0,
             seed: int = BASE_SEED, permute_nodes: bool = False, permute_elems: bool = False,
             c_law: str = "lognormal", c_sigma: float = 0.5) -> Mesh:
    """Unit-cube grid of 8-node bricks (Section 3's cubic domain)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    X = _jittered_coords(nx, ny, nz, jitter, seed)
    cells = _cells(nx, ny, nz)
    corners = cells[:, None, :] + HEX_NODE_OFFSETS[None, :, :]
    E = _node_id(corners[..., 0], corners[..., 1], corners[..., 2], nx, ny)
    if c_law == "lognormal":
        c = _c_lognormal(seed, E.shape[0], c_sigma)
    elif c_law == "subboxes":
        c = _c_subboxes(seed, X[E].mean(axis=1))
    elif c_law == "one":
        c = np.ones(E.shape[0])
    else:
        raise ValueError(c_law)
    X, E, c = _renumber(X, E, c, seed, permute_nodes, permute_elems)
    return Mesh(X, E, c, 8, (nx, ny, nz), dict(kind="hex8", jitter=jitter, seed=seed))


def kuhn_tets(nx: int, ny: int | None = None, nz: int | None = None, *, jitter: float = 0.0,
              seed: int = BASE_SEED, permute_nodes: bool = False, permute_elems: bool = False,
              c_law: str = "subboxes", c_sigma: float = 0.5) -> Mesh:
    """Unit-cube grid with each cell split into 6 tetrahedra (Kuhn split).

    Tet pi of a cell follows the path (0,0,0) -> e_pi0 -> e_pi0 + e_pi1 -> (1,1,1)
    for the 6 axis permutations pi; for odd pi nodes 1 and 2 are swapped so that
    every tetrahedron is positively oriented before jitter.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    X = _jittered_coords(nx, ny, nz, jitter, seed)
    cells = _cells(nx, ny, nz)
    tets = []
    eye = np.eye(3, dtype=np.int64)
    for perm in itertools.permutations(range(3)):
        v0 = np.zeros(3, np.int64)
        v1 = eye[perm[0]]
        v2 = v1 + eye[perm[1]]
        v3 = np.ones(3, np.int64)
        odd = sum(1 for i in range(3) for j in range(i + 1, 3) if perm[i] > perm[j]) % 2 == 1
        tets.append([v0, v2, v1, v3] if odd else [v0, v1, v2, v3])
    offs = np.array(tets, dtype=np.int64)                       # [6, 4, 3]
    corners = cells[:, None, None, :] + offs[None, :, :, :]      # [ncell, 6, 4, 3]
    E = _node_id(corners[..., 0], corners[..., 1], corners[..., 2], nx, ny).reshape(-1, 4)
    if c_law == "subboxes":
        c = _c_subboxes(seed, X[E].mean(axis=1))
    elif c_law == "lognormal":
        c = _c_lognormal(seed, E.shape[0], c_sigma)
    elif c_law == "one":
        c = np.ones(E.shape[0])
    else:
        raise ValueError(c_law)
    X, E, c = _renumber(X, E, c, seed, permute_nodes, permute_elems)
    return Mesh(X, E, c, 4, (nx, ny, nz), dict(kind="tet4", jitter=jitter, seed=seed))


def delaunay_tets(n_points: int, *, seed: int = BASE_SEED + 10, permute_nodes: bool = True,
                  permute_elems: bool = True, c_law: str = "lognormal", c_sigma: float = 0.5) -> Mesh:
    """Delaunay tetrahedralisation (Qhull, through scipy) of n_points seeded uniform
    random points in the unit cube.  Node valence, row lengths and colour counts
    vary from node to node as in a mesher's output, unlike the structured grids;
    simplices come in either orientation (the method uses |det J|)."""
    from scipy.spatial import Delaunay
    X = stream_uniform(seed, "points", 3 * n_points).reshape(-1, 3)
    E = np.ascontiguousarray(Delaunay(X).simplices, dtype=np.int64)
    if c_law == "lognormal":
        c = _c_lognormal(seed, E.shape[0], c_sigma)
    elif c_law == "subboxes":
        c = _c_subboxes(seed, X[E].mean(axis=1))
    elif c_law == "one":
        c = np.ones(E.shape[0])
    else:
        raise ValueError(c_law)
    X, E, c = _renumber(X, E, c, seed, permute_nodes, permute_elems)
    return Mesh(X, E, c, 4, (n_points,), dict(kind="tet4-delaunay", seed=seed))


def graded_bricks(n: int, *, ratio: float = 50.0, jitter: float = 0.2, seed: int = BASE_SEED + 11,
                  permute_nodes: bool = True, permute_elems: bool = True, c_sigma: float = 0.5) -> Mesh:
    """n^3 bricks on the unit cube with geometrically graded spacing: along every
    axis the cell widths grow by a constant factor from the first cell to the last,
    whose width is `ratio` times the first's.  Interior nodes are jittered by up to
    `jitter` times the smaller of their two neighbouring widths on each axis."""
    w = ratio ** (np.arange(n) / max(n - 1, 1))
    t = np.concatenate([[0.0], np.cumsum(w)]) / w.sum()           # node positions along an axis
    ijk = _grid_nodes(n, n, n)
    X = t[ijk]
    if jitter > 0.0:
        gap = np.minimum(np.diff(t, prepend=np.inf)[ijk], np.diff(t, append=np.inf)[ijk])
        interior = ((ijk > 0) & (ijk < n)).all(axis=1)
        u = stream_uniform(seed, "jitter", 3 * X.shape[0]).reshape(-1, 3)
        X = X + np.where(interior[:, None], (2.0 * u - 1.0) * jitter * gap, 0.0)
    cells = _cells(n, n, n)
    corners = cells[:, None, :] + HEX_NODE_OFFSETS[None, :, :]
    E = _node_id(corners[..., 0], corners[..., 1], corners[..., 2], n, n)
    c = _c_lognormal(seed, E.shape[0], c_sigma)
    X, E, c = _renumber(X, E, c, seed, permute_nodes, permute_elems)
    return Mesh(X, E, c, 8, (n, n, n), dict(kind="hex8-graded", ratio=ratio, jitter=jitter, seed=seed))


def batch_specs(n_meshes: int = 512, seed: int = BASE_SEED + 3, lo: float = 1e3, hi: float = 2e5,
                nmin: int = 10, nmax: int = 60):
    """Grid shapes for a batch of uneven meshes.

    Target element counts are log-uniform in [lo, hi]; nx and ny are uniform in
    [nmin, nmax] and nz = round(target / (nx * ny)) clipped to [nmin, nmax].
    """
    t = np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * stream_uniform(seed, "batch/target", n_meshes))
    span = nmax - nmin + 1
    nx = nmin + (stream_u64(seed, "batch/nx", n_meshes) % np.uint64(span)).astype(np.int64)
    ny = nmin + (stream_u64(seed, "batch/ny", n_meshes) % np.uint64(span)).astype(np.int64)
    nz = np.clip(np.rint(t / (nx * ny)), nmin, nmax).astype(np.int64)
    return [(int(a), int(b), int(cc)) for a, b, cc in zip(nx, ny, nz)]


# Configurations of the benchmark workloads (seed = BASE_SEED + index).
def config_mesh(index: int, **over) -> Mesh:
    """The synthetic mesh of workload ``index`` (0..4), optionally re-sized."""
    seed = BASE_SEED + index
    if index == 0:   # 20^3 bricks, jitter 0.2h, permuted, c ~ lognormal(0, 0.5)
        kw = dict(nx=20, jitter=0.2, seed=seed, permute_nodes=True, permute_elems=True, c_sigma=0.5)
        kw.update(over)
        return hex_grid(**kw)
    if index == 1:   # 100^3 bricks, jitter 0.25h, permuted, c ~ lognormal(0, 1)
        kw = dict(nx=100, jitter=0.25, seed=seed, permute_nodes=True, permute_elems=True, c_sigma=1.0)
        kw.update(over)
        return hex_grid(**kw)
    if index == 2:   # 80^3 cells x 6 Kuhn tets, jitter 0.3h, permuted, c on 8 sub-boxes
        kw = dict(nx=80, jitter=0.3, seed=seed, permute_nodes=True, permute_elems=True, c_law="subboxes")
        kw.update(over)
        return kuhn_tets(**kw)
    if index == 4:   # 300^3 bricks, jitter 0.2h, c ~ lognormal(0, 0.5)
        kw = dict(nx=300, jitter=0.2, seed=seed, c_sigma=0.5)
        kw.update(over)
        return hex_grid(**kw)
    raise ValueError("workload 3 is a batch: use batch_meshes()")


def batch_meshes(n_meshes: int = 512, seed: int = BASE_SEED + 3, jitter: float = 0.2, sigma: float = 0.5):
    """The uneven batch: one jittered brick grid per shape of ``batch_specs``."""
    specs = batch_specs(n_meshes, seed=seed)
    return [hex_grid(nx, ny, nz, jitter=jitter, seed=seed * 1000 + m, c_sigma=sigma)
            for m, (nx, ny, nz) in enumerate(specs)]


def lame(m: "Mesh", seed: int | None = None, nu_lo: float = 0.1, nu_hi: float = 0.45) -> np.ndarray:
    """[n_elems, 2] Lame parameters (lambda_e, mu_e) of an isotropic material with
    Young's modulus c_e and Poisson ratio nu_e ~ U[nu_lo, nu_hi] (stream "nu"):
    lambda = E nu / ((1 + nu)(1 - 2 nu)), mu = E / (2 (1 + nu))."""
    seed = m.meta.get("seed", BASE_SEED) if seed is None else seed
    nu = nu_lo + (nu_hi - nu_lo) * stream_uniform(seed, "nu", m.E.shape[0])
    E = np.asarray(m.c, np.float64)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return np.ascontiguousarray(np.stack([lam, mu], axis=1))
