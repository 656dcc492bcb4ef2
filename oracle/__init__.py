"""Python face of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE, NOT THE PRODUCT.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` import this package.  It never imports
the CUDA package and the CUDA package never imports it; the two share only the
seeded input generator ``meshgen``.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``.
Every function here is argument marshalling around one C routine; the
arithmetic, its citations and its readings of the paper are in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_int = ctypes.c_int
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no fast-math) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def declare(L):
    """Declares the argument types of the oracle's C routines on a loaded library
    (this one, or a test's copy built from a modified source)."""
    L.oracle_ke_dense.argtypes = [_int, _int, _p, ctypes.c_double, _p]
    L.oracle_ke_dense.restype = _int
    L.oracle_ke_elastic_dense.argtypes = [_int, _p, ctypes.c_double, ctypes.c_double, _p]
    L.oracle_ke_elastic_dense.restype = _int
    L.oracle_ke_packed.argtypes = [_int, _int, _i64, _p, _p, _p, _p, _p]
    L.oracle_ke_packed.restype = _i64
    L.oracle_triplets.argtypes = [_int, _int, _i64, _p, _p, _p, _p, _p, _p, _p]
    L.oracle_triplets.restype = _i64
    L.oracle_compress.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]
    L.oracle_compress.restype = _i64
    L.oracle_vjp.argtypes = [_int, _i64, _p, _p, _p, _p, _p, _p]
    L.oracle_vjp.restype = None
    L.oracle_vjp_op.argtypes = [_int, _int, _i64, _p, _p, _p, _p, _p, _p]
    L.oracle_vjp_op.restype = None
    L.oracle_load.argtypes = [_int, _i64, _p, _p, _p, _p]
    L.oracle_load.restype = _i64
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _inputs(X, E, c):
    X = np.ascontiguousarray(X, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.float64)
    return X, E, c


# Operators: the stiffness matrix of Eq. 9, the mass matrix (Section 5) and
# linear elasticity (three DOFs per node; c is then [n_elems, 2] = (lambda, mu)).
OPS = {"stiffness": 0, "mass": 1, "elasticity": 2}


def dofs(op: str = "stiffness") -> int:
    """Degrees of freedom per node (Algorithm 1's DOFxn)."""
    return 3 if op == "elasticity" else 1


def npairs(npe: int, op: str = "stiffness") -> int:
    nk = dofs(op) * npe
    return nk * (nk + 1) // 2


def ke_dense(npe: int, xe, c: float, op: str = "stiffness") -> np.ndarray:
    """Full npe x npe element matrix of one element with node coordinates xe [npe, 3]."""
    xe = np.ascontiguousarray(xe, dtype=np.float64).reshape(npe, 3)
    ke = np.zeros((npe, npe))
    lib().oracle_ke_dense(OPS[op], npe, _ptr(xe), float(c), _ptr(ke))
    return ke


def ke_elastic_dense(npe: int, xe, lam: float, mu: float) -> np.ndarray:
    """Dense (3 npe) x (3 npe) elasticity matrix of one element (DOF 3a + i)."""
    xe = np.ascontiguousarray(xe, dtype=np.float64).reshape(npe, 3)
    ke = np.zeros((3 * npe, 3 * npe))
    lib().oracle_ke_elastic_dense(npe, _ptr(xe), float(lam), float(mu), _ptr(ke))
    return ke


def ke_packed(npe: int, X, E, c, op: str = "stiffness"):
    """Packed lower k_e [n_elems, nk(nk+1)/2] (p = A(A+1)/2 + B over the nk local
    DOFs), the Cauchy-Schwarz scales sqrt(k_AA k_BB) of each entry, and the number
    of elements with det J <= 0."""
    X, E, c = _inputs(X, E, c)
    n = E.shape[0]
    ke = np.zeros((n, npairs(npe, op)))
    cs = np.zeros((n, npairs(npe, op)))
    bad = lib().oracle_ke_packed(OPS[op], npe, n, _ptr(E), _ptr(X), _ptr(c), _ptr(ke), _ptr(cs))
    return ke, cs, int(bad)


def triplets(npe: int, X, E, c, op: str = "stiffness"):
    """Algorithm 1's triplet arrays (rows, cols, vals) plus per-triplet scales."""
    X, E, c = _inputs(X, E, c)
    nt = E.shape[0] * npairs(npe, op)
    rows = np.zeros(nt, np.int64)
    cols = np.zeros(nt, np.int32)
    vals = np.zeros(nt)
    cs = np.zeros(nt)
    bad = lib().oracle_triplets(OPS[op], npe, E.shape[0], _ptr(E), _ptr(X), _ptr(c), _ptr(rows),
                                _ptr(cols), _ptr(vals), _ptr(cs))
    return rows, cols, vals, cs, int(bad)


def compress(n_nodes: int, rows, cols, vals, cs):
    """The sparse conversion: lower CSR with per-entry sums of |val| and of scales,
    and the CSR slot of every triplet (n_nodes = number of rows: nodes times DOFs
    per node)."""
    nt = rows.shape[0]
    rowptr = np.zeros(n_nodes + 1, np.int64)
    col = np.zeros(max(nt, 1), np.int32)
    val = np.zeros(max(nt, 1))
    ab = np.zeros(max(nt, 1))
    sc = np.zeros(max(nt, 1))
    slot = np.zeros(max(nt, 1), np.int64)
    nnz = lib().oracle_compress(nt, n_nodes, _ptr(rows), _ptr(cols), _ptr(vals), _ptr(cs),
                                _ptr(rowptr), _ptr(col), _ptr(val), _ptr(ab), _ptr(sc), _ptr(slot))
    return dict(rowptr=rowptr, col=col[:nnz].copy(), vals=val[:nnz].copy(), abs=ab[:nnz].copy(),
                cs=sc[:nnz].copy(), slot=slot[:nt].copy(), nnz=int(nnz))


def build_K(npe: int, X, E, c, op: str = "stiffness"):
    """Algorithm 1 end to end: global lower-triangular CSR K (or M, op="mass"; or
    the 3N x 3N elasticity matrix, op="elasticity") in FP64.

    Returns a dict with rowptr, col, vals, abs (sum of |contribution|), cs (sum of
    Cauchy-Schwarz scales), slot (CSR position of each packed (e, p)), nnz, and
    n_bad (elements with a non-positive Jacobian determinant)."""
    X, E, c = _inputs(X, E, c)
    rows, cols, vals, cs, bad = triplets(npe, X, E, c, op)
    out = compress(X.shape[0] * dofs(op), rows, cols, vals, cs)
    out["n_bad"] = bad
    return out


def vjp(npe: int, X, E, c, S, op: str = "stiffness"):
    """Gradient of L = sum_(e,p) S[e,p] k_e[p] with respect to X [n_nodes, 3] and c [n_elems]
    (op: "stiffness", "mass" or "elasticity", for which c and dc are [n_elems, 2])."""
    X, E, c = _inputs(X, E, c)
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(E.shape[0], npairs(npe, op))
    dX = np.zeros_like(X)
    dc = np.zeros((E.shape[0], 2) if op == "elasticity" else E.shape[0])
    lib().oracle_vjp_op(OPS[op], npe, E.shape[0], _ptr(E), _ptr(X), _ptr(c), _ptr(S), _ptr(dX), _ptr(dc))
    return dX, dc


def vjp_from_G(npe: int, X, E, c, G, slot, op: str = "stiffness"):
    """Gradient of L = sum over stored entries G_ij K_ij (Section 3's lower storage,
    each packed pair counted once) given the CSR slot map from ``build_K``."""
    S = np.asarray(G)[np.asarray(slot)]
    return vjp(npe, X, E, c, S, op)


def load_vector(npe: int, X, E, s):
    """Global load vector F [n_nodes] of a per-element constant source s [n_elems]
    (F_n = sum over elements of s_e * integral N_a, a the element's local index of n).
    For a body force s [n_elems, 3] (the elasticity operator) F is [3 n_nodes],
    F[3n + i] the load of component i: the scalar load of each component."""
    if np.ndim(s) == 2:
        comps = [load_vector(npe, X, E, np.asarray(s)[:, i]) for i in range(np.shape(s)[1])]
        return np.stack(comps, axis=1).ravel()
    X, E, s = _inputs(X, E, s)
    F = np.zeros(X.shape[0])
    lib().oracle_load(npe, E.shape[0], _ptr(E), _ptr(X), _ptr(s), _ptr(F))
    return F
