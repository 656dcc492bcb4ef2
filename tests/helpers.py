"""Shared test helpers: oracle references and the error metric.

Error metric (per entry of K or of a packed k_e):
    err = |value - oracle| / scale,
where scale is the sum over contributing elements of sqrt(k_aa * k_bb), the
Cauchy-Schwarz bound of |k_ab| for a positive semidefinite element matrix.
FP rounding in k_ab scales with that bound (the integrand B_a . B_b is bounded
by |B_a||B_b|), not with |k_ab|, which can cancel to ~0 (edge couplings of an
undistorted brick are exactly 0).  Tolerances: 1e-12 in FP64, 1e-5 in mixed.
"""
import numpy as np

import meshgen
import oracle

TOL_FP64 = 1e-12
TOL_MIXED = 1e-5


def mesh_for(index, **over):
    return meshgen.config_mesh(index, **over)


def rounded_inputs(m, prec):
    """Inputs as the GPU sees them: mixed-mode X and c rounded to FP32."""
    if prec == "mixed":
        return m.X.astype(np.float32), m.c.astype(np.float32)
    return m.X, m.c


def oracle_K(m, X=None, c=None, op="stiffness"):
    X = m.X if X is None else X
    c = m.c if c is None else c
    return oracle.build_K(m.npe, np.asarray(X, np.float64), m.E, np.asarray(c, np.float64), op)


def oracle_ke(m, X=None, c=None, op="stiffness"):
    X = m.X if X is None else X
    c = m.c if c is None else c
    return oracle.ke_packed(m.npe, np.asarray(X, np.float64), m.E, np.asarray(c, np.float64), op)


def rel_err(got, ref, scale):
    got = np.asarray(got, np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300))) if len(ref) else 0.0


def oracle_rows(m, rows, X=None, c=None, op="stiffness"):
    """Exact rows of K for a sample of nodes: the oracle run on the elements that
    touch any sampled node (those rows are then complete)."""
    X = m.X if X is None else X
    c = m.c if c is None else c
    rows = np.unique(np.asarray(rows))
    touch = np.isin(m.E, rows).any(axis=1)
    sub = oracle.build_K(m.npe, np.asarray(X, np.float64), m.E[touch], np.asarray(c, np.float64)[touch], op)
    out = {}
    for r in rows:
        a, b = sub["rowptr"][r], sub["rowptr"][r + 1]
        out[int(r)] = (sub["col"][a:b], sub["vals"][a:b], sub["cs"][a:b])
    return out
