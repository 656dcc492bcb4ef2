"""Thin binding of libfem for torch tensors.

Every method is one C-ABI call: it checks tensor devices and dtypes, passes
``data_ptr()`` and the current CUDA stream, and raises ``FemError`` on a
non-OK status.  All arithmetic runs in the library's CUDA kernels.  PyTorch
provides device memory and streams only.
"""
from __future__ import annotations

import ctypes

import torch

from . import abi

_DT = {torch.float32: abi.FEM_F32, torch.float64: abi.FEM_F64}
_PREC = {"fp64": abi.FEM_FP64, "mixed": abi.FEM_MIXED}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _prec(prec: str) -> int:
    if prec not in _PREC:
        raise ValueError("prec must be 'fp64' or 'mixed'")
    return _PREC[prec]


def value_dtype(prec: str):
    return torch.float64 if prec == "fp64" else torch.float32


def default_options() -> abi.fem_options:
    o = abi.fem_options()
    abi.load().fem_options_default(ctypes.byref(o))
    return o


def launch_count(reset: bool = False) -> int:
    return int(abi.load().fem_launch_count(1 if reset else 0))


class Mesh:
    """A mesh handle: E (int32 [n_elems, npe] on the GPU) plus the cached pattern.

    With ``operator_kind=2`` (elasticity) the matrix has three DOFs per node (DOF
    3g + i), c is [n_elems, 2] = (lambda, mu), and the pattern, the values and the
    packed element matrices are those of the DOF matrix."""

    def __init__(self, E: torch.Tensor, n_nodes: int, X: torch.Tensor | None = None, options=None, stream=None,
                 **opts):
        L = abi.load()
        if E.dim() != 2 or E.shape[1] not in (4, 8):
            raise ValueError("E must be [n_elems, 8] or [n_elems, 4]")
        self.E = E
        self.npe = int(E.shape[1])
        self.n_nodes = int(n_nodes)
        self.n_elems = int(E.shape[0])
        o = options if options is not None else default_options()
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        self.dofs = 3 if o.operator_kind == 2 else 1      # DOFs per node
        nk = self.dofs * self.npe
        self.np = nk * (nk + 1) // 2                        # packed entries of one k_e
        h = ctypes.c_void_p()
        xp = _dev(X, "X") if X is not None else None
        xd = _DT.get(X.dtype, abi.FEM_F64) if X is not None else abi.FEM_F64
        abi.check(L.fem_mesh_create(ctypes.byref(h), self.npe, self.n_nodes, self.n_elems, _dev(E, "E", torch.int32),
                                    xp, xd, ctypes.byref(o), _stream(stream)))
        self._h = h
        self.nnz = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            abi.load().fem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- symbolic
    def pattern(self, stream=None) -> int:
        n = ctypes.c_int64()
        abi.check(abi.load().fem_pattern(self._h, ctypes.byref(n), _stream(stream)))
        self.nnz = int(n.value)
        return self.nnz

    def get_pattern(self, stream=None):
        if self.nnz is None:
            self.pattern(stream)
        rowptr = torch.empty(self.dofs * self.n_nodes + 1, dtype=torch.int64, device=self.E.device)
        col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=self.E.device)
        abi.check(abi.load().fem_get_pattern(self._h, _dev(rowptr, "rowptr"), _dev(col, "col"), _stream(stream)))
        return rowptr, col[: self.nnz]

    # ---- numeric
    def integrate_local(self, X, c, prec="fp64", out=None, stream=None):
        p = _prec(prec)
        if out is None:
            out = torch.empty(self.n_elems, self.np, dtype=value_dtype(prec), device=X.device)
        abi.check(abi.load().fem_integrate_local(self._h, p, _dev(X, "X"), _DT[X.dtype], _dev(c, "c"), _DT[c.dtype],
                                                 _dev(out, "ke", value_dtype(prec)), _stream(stream)))
        return out

    def assemble_csr(self, ke, prec="fp64", out=None, stream=None):
        p = _prec(prec)
        if self.nnz is None:
            self.pattern(stream)
        if out is None:
            out = torch.empty(max(self.nnz, 1), dtype=value_dtype(prec), device=ke.device)
        abi.check(abi.load().fem_assemble_csr(self._h, p, _dev(ke, "ke", value_dtype(prec)),
                                              _dev(out, "vals", value_dtype(prec)), _stream(stream)))
        return out[: self.nnz]

    def build_K(self, X, c, prec="fp64", out=None, stream=None):
        p = _prec(prec)
        if self.nnz is None:
            self.pattern(stream)
        if out is None:
            out = torch.empty(max(self.nnz, 1), dtype=value_dtype(prec), device=X.device)
        abi.check(abi.load().fem_build_K(self._h, p, _dev(X, "X"), _DT[X.dtype], _dev(c, "c"), _DT[c.dtype],
                                         _dev(out, "vals", value_dtype(prec)), _stream(stream)))
        return out[: self.nnz]

    def build_K_host(self, X, c, prec="fp64", out=None, stream=None):
        """Host tensors in and out (pin them for full copy bandwidth)."""
        p = _prec(prec)
        if self.nnz is None:
            self.pattern(stream)
        for t, n in ((X, "X"), (c, "c")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous host tensor")
        if out is None:
            out = torch.empty(max(self.nnz, 1), dtype=value_dtype(prec), pin_memory=True)
        abi.check(abi.load().fem_build_K_host(self._h, p, ctypes.c_void_p(X.data_ptr()), _DT[X.dtype],
                                              ctypes.c_void_p(c.data_ptr()), _DT[c.dtype],
                                              ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out[: self.nnz]

    def build_K_host_async(self, X, c, prec="fp64", out=None, stream=None):
        """Page-locked host tensors in and out, ordered on `stream`; out is complete once
        the stream is synchronised."""
        p = _prec(prec)
        if self.nnz is None:
            self.pattern(stream)
        for t, n in ((X, "X"), (c, "c")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous host tensor")
        if out is None:
            out = torch.empty(max(self.nnz, 1), dtype=value_dtype(prec), pin_memory=True)
        abi.check(abi.load().fem_build_K_host_async(self._h, p, ctypes.c_void_p(X.data_ptr()), _DT[X.dtype],
                                                    ctypes.c_void_p(c.data_ptr()), _DT[c.dtype],
                                                    ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out[: self.nnz]

    def vjp(self, X, c, G, prec="fp64", stream=None):
        """dL/dX [n_nodes, 3] and dL/dc of L = sum over stored entries G_ij K_ij:
        dc is [n_elems], or [n_elems, 2] (dL/dlambda, dL/dmu) for elasticity."""
        p = _prec(prec)
        vd = value_dtype(prec)
        dX = torch.empty(self.n_nodes, 3, dtype=vd, device=X.device)
        dc = torch.empty((self.n_elems, 2) if self.dofs == 3 else (self.n_elems,), dtype=vd, device=X.device)
        abi.check(abi.load().fem_vjp(self._h, p, _dev(X, "X"), _DT[X.dtype], _dev(c, "c"), _DT[c.dtype],
                                     _dev(G, "G", vd), _dev(dX, "dX"), _dev(dc, "dc"), _stream(stream)))
        return dX, dc

    def load_vector(self, X, src, prec="fp64", out=None, stream=None):
        """Global load vector F [n_nodes] of the per-element constant source src [n_elems]
        (elasticity: F [3 n_nodes] of the per-element body force src [n_elems, 3])."""
        p = _prec(prec)
        if self.nnz is None:
            self.pattern(stream)
        vd = value_dtype(prec)
        if out is None:
            out = torch.empty(self.dofs * self.n_nodes, dtype=vd, device=X.device)
        abi.check(abi.load().fem_load_vector(self._h, p, _dev(X, "X"), _DT[X.dtype], _dev(src, "src"), _DT[src.dtype],
                                             _dev(out, "F", vd), _stream(stream)))
        return out

    def autotune(self, X, c, prec="mixed", stream=None, cache: str | None = None) -> dict:
        """Pick the work unit (elements per tile, or entries per patch) and block size by
        timing fem_build_K (overwrites a scratch vals).

        With ``cache`` (a JSON file path), a tuning stored for the same GPU model,
        element type, precision, operator and mesh size class (elements to the
        nearest power of two) is applied without timing (``tried`` = 0); a new one
        is timed and stored."""
        if self.nnz is None:
            self.pattern(stream)
        key = None
        if cache is not None:
            import json
            import math
            import os
            key = "|".join([torch.cuda.get_device_name(X.device), f"npe={self.npe}", prec,
                            f"op={self.options.operator_kind}", f"asm={self.options.assembly}",
                            f"log2n={round(math.log2(max(self.n_elems, 1)))}"])
            table = json.load(open(cache)) if os.path.exists(cache) else {}
            if key in table:
                hit = table[key]
                abi.check(abi.load().fem_set_tuning(self._h, int(hit["patch_entries"]), int(hit["block_threads"]),
                                                    _stream(stream)))
                return dict(patch_entries=hit["patch_entries"], block_threads=hit["block_threads"],
                            ms=hit["ms"], tried=0)
        vals = torch.empty(max(self.nnz, 1), dtype=value_dtype(prec), device=X.device)
        t = abi.fem_tuning()
        abi.check(abi.load().fem_autotune(self._h, _prec(prec), _dev(X, "X"), _DT[X.dtype], _dev(c, "c"),
                                          _DT[c.dtype], _dev(vals, "vals"), _stream(stream), ctypes.byref(t)))
        out = dict(patch_entries=t.patch_entries, block_threads=t.block_threads, ms=t.ms, tried=t.tried,
                   assembly=t.assembly)
        if key is not None:
            table = json.load(open(cache)) if os.path.exists(cache) else {}
            table[key] = dict(patch_entries=out["patch_entries"], block_threads=out["block_threads"], ms=out["ms"])
            tmp = f"{cache}.{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return out

    def set_tuning(self, patch_entries: int, block_threads: int, stream=None):
        """Apply a known tuning (rebuilds the plan if the pattern exists)."""
        abi.check(abi.load().fem_set_tuning(self._h, int(patch_entries), int(block_threads), _stream(stream)))

    def sync(self, stream=None):
        abi.check(abi.load().fem_sync(self._h, _stream(stream)))

    def info(self) -> dict:
        i = abi.fem_info()
        abi.check(abi.load().fem_mesh_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in abi.fem_info._fields_ if not f.startswith("reserved")}


def batched_config(meshes, prec="mixed") -> dict:
    """Launch shape the batched build of these meshes was tuned to."""
    n = len(meshes)
    H = (ctypes.c_void_p * n)(*[m.handle.value for m in meshes])
    t, b, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    abi.check(abi.load().fem_batched_config(H, n, _prec(prec), ctypes.byref(t), ctypes.byref(b), ctypes.byref(g)))
    return dict(block_threads=t.value, blocks_per_sm=b.value, grid=g.value)


def build_K_batched(meshes, X, c, prec="mixed", out=None, stream=None):
    """One persistent launch over many meshes (each with its pattern cached)."""
    p = _prec(prec)
    n = len(meshes)
    for m in meshes:
        if m.nnz is None:
            m.pattern(stream)
    if out is None:
        out = [torch.empty(max(m.nnz, 1), dtype=value_dtype(prec), device=X[i].device) for i, m in enumerate(meshes)]
    H = (ctypes.c_void_p * n)(*[m.handle.value for m in meshes])
    XP = (ctypes.c_void_p * n)(*[x.data_ptr() for x in X])
    CP = (ctypes.c_void_p * n)(*[t.data_ptr() for t in c])
    VP = (ctypes.c_void_p * n)(*[v.data_ptr() for v in out])
    abi.check(abi.load().fem_build_K_batched(H, n, p, XP, _DT[X[0].dtype], CP, _DT[c[0].dtype], VP, _stream(stream)))
    return [v[: m.nnz] for v, m in zip(out, meshes)]
