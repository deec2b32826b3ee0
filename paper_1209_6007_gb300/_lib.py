"""ctypes declarations of the C ABI in include/bcshatter.h."""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbcshatter.so")

BCS_OK = 0
BCS_EINVAL = -1
BCS_ENOMEM = -2
BCS_ECUDA = -3
BCS_ETIMEOUT = -4
BCS_EOVERFLOW = -5
BCS_ENODEV = -6

STEP_D, STEP_A, STEP_I = 1, 2, 4
STEPS_ALL = 7
STEP_O = 8  # BFS ordering, opt-in
STEP_S = 16  # side vertices, opt-in
STEP_U = 32  # identical vertices of unequal reach, opt-in
STEP_L = 64  # one more articulation split after merging, opt-in
NOALLOC_MAX_N = 16384

c_i64, c_i32, c_u32, c_dbl, c_vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p


class Csr(ctypes.Structure):
    _fields_ = [("n", c_i64), ("nnz", c_i64), ("row_ptr", c_vp), ("col", c_vp), ("on_device", c_i32)]


class Opts(ctypes.Structure):
    _fields_ = [("steps", c_u32), ("delta_fp32", c_i32), ("autotune", c_i32), ("device", c_i32),
                ("stream", c_vp), ("max_wait", c_i64)]


class Stats(ctypes.Structure):
    _fields_ = [(name, c_i64) for name in (
        "n_pieces", "n_slots", "n_merged", "n_entries", "peel_rounds", "n_small_items",
        "n_large_sources", "kernel_launches", "bfs_levels", "dag_edges", "n_ms_batches", "batch_ctas", "small_ng_cap", "small_smem_budget", "n_side",
        "n_wide_batches", "n_rounds", "small_limit", "tuned")] + [(name, c_dbl) for name in (
        "work_nm", "work_sources_entries", "work_sources_vertices", "ms_total", "ms_upload", "ms_validate", "ms_cc", "ms_peel",
        "ms_blocks", "ms_ident", "ms_plan", "ms_bcreach_small", "ms_bcreach_large", "ms_mapback",
        "ms_download", "ms_side")]


class ComponentsView(ctypes.Structure):
    _fields_ = [("n", c_i64), ("n_pieces", c_i64), ("n_merged", c_i64), ("n_entries", c_i64),
                ("n_members", c_i64), ("piece_vtx_off", c_vp), ("piece_N", c_vp), ("row_ptr", c_vp),
                ("col", c_vp), ("org", c_vp), ("reach", c_vp), ("ident", c_vp), ("member_off", c_vp),
                ("member", c_vp), ("bc_pre", c_vp), ("bc_corr", c_vp)]


# name -> (restype, argtypes); every entry point of include/bcshatter.h
SIGNATURES = {
    "bcs_bc_plain": (ctypes.c_int, [c_vp, c_vp, c_vp]),
    "bcs_bc_shattered": (ctypes.c_int, [c_vp, c_vp, c_vp]),
    "bcs_bc_sources": (ctypes.c_int, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "bcs_bc_plain_noalloc": (ctypes.c_int, [c_vp, c_vp, c_vp]),
    "bcs_bc_shattered_batch": (ctypes.c_int, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    "bcs_debug_sssp": (ctypes.c_int, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "bcs_shatter": (ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "bcs_components_get": (ctypes.c_int, [c_vp, ctypes.POINTER(ComponentsView)]),
    "bcs_components_free": (None, [c_vp]),
    "bcs_last_stats": (ctypes.c_int, [ctypes.POINTER(Stats)]),
    "bcs_last_error": (ctypes.c_char_p, []),
    "bcs_version": (ctypes.c_int, []),
}

_lib = None


def load():
    """Load libbcshatter.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` (there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib
