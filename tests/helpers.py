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


# Backward-pass error metric (per component).  An element's contribution to
# dL/dx_a and to dL/dc_e is a sum of terms of size |S_p| * sqrt(k_aa k_bb) / h_e
# (dL/dx) and |S_p| * sqrt(k_aa k_bb) / c_e (dL/dc): k scales as c_e * h_e (h_e
# the element's size), so its derivatives scale as c_e and as h_e; h_e is the
# shortest distance between two of its nodes, the bound for a flat element.  The scale of
# a component is the sum of those bounds over the elements that contribute to it,
# the analogue for gradients of the per-entry scale above; FP rounding in the
# reverse-mode element arithmetic is relative to it, whereas the component
# itself can cancel to ~0.
TOL_VJP_FP64 = 1e-12
TOL_VJP_MIXED = 2e-6


def vjp_scales(m, X, c, S, op="stiffness"):
    """Per-component scales (dX [n_nodes, 3], dc [n_elems] or [n_elems, 2]) of the
    gradient of L = sum_(e,p) S[e, p] k_e[p]."""
    _, cs, _ = oracle.ke_packed(m.npe, np.asarray(X, np.float64), m.E, np.asarray(c, np.float64), op)
    w = np.sum(np.abs(np.asarray(S, np.float64).reshape(cs.shape)) * cs, axis=1)
    Xe = np.asarray(X, np.float64)[m.E]                              # [n_elems, npe, 3]
    edges = Xe[:, :, None, :] - Xe[:, None, :, :]
    dist = np.sqrt((edges ** 2).sum(-1))
    dist[:, np.arange(m.npe), np.arange(m.npe)] = np.inf
    h = dist.min(axis=(1, 2))                                        # shortest node-to-node distance
    sx = np.zeros((m.n_nodes, 3))
    np.add.at(sx, m.E.ravel(), np.repeat(w / h, m.npe)[:, None] * np.ones((1, 3)))
    cc = np.asarray(c, np.float64)
    if op == "elasticity":
        stiff = cc[:, 0] + 2 * cc[:, 1]
        sc = np.repeat((w / stiff)[:, None], 2, axis=1)
    else:
        sc = w / np.abs(cc)
    return sx, sc


def vjp_err(got, ref, scale):
    got = np.asarray(got, np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300))) if np.size(ref) else 0.0
