"""ctypes declarations of the C ABI in ``include/fem.h`` (same names).

This module only loads ``_build/libfem.so`` and declares argument types.  It
raises ``RuntimeError`` when the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

FEM_OK = 0
STATUS = {0: "FEM_OK", 1: "FEM_ERR_ARG", 2: "FEM_ERR_INDEX", 3: "FEM_ERR_DEGENERATE", 4: "FEM_ERR_OOM",
          5: "FEM_ERR_BUDGET", 6: "FEM_ERR_CUDA", 7: "FEM_ERR_TIMEOUT", 8: "FEM_ERR_STATE",
          9: "FEM_ERR_UNSUPPORTED"}
FEM_TET4, FEM_HEX8 = 4, 8
FEM_FP64, FEM_MIXED = 0, 1
FEM_F32, FEM_F64 = 0, 1


class fem_options(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("distortion_threshold", ctypes.c_double),
                ("valence_threshold", ctypes.c_int), ("patch_entries", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("locality_order", ctypes.c_int), ("fp64_sums", ctypes.c_int),
                ("fp64_fused", ctypes.c_int), ("fp64_dets", ctypes.c_int),
                ("wait_spins", ctypes.c_int), ("debug_stall", ctypes.c_int),
                ("operator_kind", ctypes.c_int), ("host_direct", ctypes.c_int), ("vjp_fused", ctypes.c_int),
                ("assembly", ctypes.c_int), ("tile_elems", ctypes.c_int),
                ("host_chunks", ctypes.c_int), ("group_cache", ctypes.c_int)]


class fem_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_patches", ctypes.c_int64), ("closure_elems", ctypes.c_int64),
                ("max_patch_entries", ctypes.c_int64), ("max_patch_cnodes", ctypes.c_int64),
                ("max_patch_elems", ctypes.c_int64), ("n_colors", ctypes.c_int32),
                ("max_row_len", ctypes.c_int32), ("plan_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("n_groups", ctypes.c_int32),
                ("assembly", ctypes.c_int32), ("live_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("n_chunks", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("tile_rows", ctypes.c_int64),
                ("border_rows", ctypes.c_int64),
                ("partial_values", ctypes.c_int64)]


class fem_tuning(ctypes.Structure):
    _fields_ = [("patch_entries", ctypes.c_int), ("block_threads", ctypes.c_int), ("ms", ctypes.c_float),
                ("tried", ctypes.c_int), ("assembly", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


EXPORTS = ["fem_options_default", "fem_status_str", "fem_last_error", "fem_mesh_create", "fem_mesh_destroy",
           "fem_pattern", "fem_get_pattern", "fem_pattern_ptrs", "fem_integrate_local", "fem_assemble_csr",
           "fem_build_K", "fem_build_K_host", "fem_build_K_host_async", "fem_vjp", "fem_load_vector", "fem_build_K_batched", "fem_sync", "fem_mesh_info",
           "fem_launch_count", "fem_pattern_noalloc", "fem_batched_config", "fem_autotune", "fem_set_tuning"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfem.so and declare its functions.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libfem is not built ({_build.LIB} missing): run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P, I64, I32, INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    S = ctypes.c_int  # fem_status
    L.fem_options_default.argtypes = [ctypes.POINTER(fem_options)]
    L.fem_options_default.restype = None
    L.fem_status_str.argtypes = [S]
    L.fem_status_str.restype = ctypes.c_char_p
    L.fem_last_error.argtypes = []
    L.fem_last_error.restype = ctypes.c_char_p
    L.fem_mesh_create.argtypes = [ctypes.POINTER(P), INT, I64, I64, P, P, INT, ctypes.POINTER(fem_options), P]
    L.fem_mesh_create.restype = S
    L.fem_mesh_destroy.argtypes = [P]
    L.fem_mesh_destroy.restype = None
    L.fem_pattern.argtypes = [P, ctypes.POINTER(I64), P]
    L.fem_pattern.restype = S
    L.fem_get_pattern.argtypes = [P, P, P, P]
    L.fem_get_pattern.restype = S
    L.fem_pattern_ptrs.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P)]
    L.fem_pattern_ptrs.restype = S
    L.fem_integrate_local.argtypes = [P, INT, P, INT, P, INT, P, P]
    L.fem_integrate_local.restype = S
    L.fem_assemble_csr.argtypes = [P, INT, P, P, P]
    L.fem_assemble_csr.restype = S
    L.fem_build_K.argtypes = [P, INT, P, INT, P, INT, P, P]
    L.fem_build_K.restype = S
    L.fem_build_K_host.argtypes = [P, INT, P, INT, P, INT, P, P]
    L.fem_build_K_host.restype = S
    L.fem_build_K_host_async.argtypes = L.fem_build_K_host.argtypes
    L.fem_build_K_host_async.restype = S
    L.fem_vjp.argtypes = [P, INT, P, INT, P, INT, P, P, P, P]
    L.fem_vjp.restype = S
    L.fem_load_vector.argtypes = [P, INT, P, INT, P, INT, P, P]
    L.fem_load_vector.restype = S
    L.fem_build_K_batched.argtypes = [ctypes.POINTER(P), INT, INT, ctypes.POINTER(P), INT, ctypes.POINTER(P), INT,
                                      ctypes.POINTER(P), P]
    L.fem_build_K_batched.restype = S
    L.fem_sync.argtypes = [P, P]
    L.fem_sync.restype = S
    L.fem_mesh_info.argtypes = [P, ctypes.POINTER(fem_info)]
    L.fem_mesh_info.restype = S
    L.fem_launch_count.argtypes = [INT]
    L.fem_launch_count.restype = I64
    L.fem_pattern_noalloc.argtypes = [INT, I64, I64, P, P, P, I64, ctypes.POINTER(I64), P]
    L.fem_pattern_noalloc.restype = S
    L.fem_batched_config.argtypes = [ctypes.POINTER(P), INT, INT, ctypes.POINTER(INT), ctypes.POINTER(INT),
                                     ctypes.POINTER(INT)]
    L.fem_batched_config.restype = S
    L.fem_autotune.argtypes = [P, INT, P, INT, P, INT, P, P, ctypes.POINTER(fem_tuning)]
    L.fem_autotune.restype = S
    L.fem_set_tuning.argtypes = [P, INT, INT, P]
    L.fem_set_tuning.restype = S
    _lib = L
    return L


class FemError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS.get(status, status)}: {detail}")
        self.status = status
        self.name = STATUS.get(status, str(status))


def check(status: int):
    if status != FEM_OK:
        raise FemError(status, load().fem_last_error().decode(errors="replace"))
