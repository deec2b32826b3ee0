"""GB300 shattered betweenness centrality: Python binding of libbcshatter.so.

The binding only marshals arguments: every step of the computation runs in
the library's CUDA kernels, driven by its host C++ code (planning, launches,
copies).  There is no CPU fallback; a missing library raises.

Graphs are given as CSR arrays (``row_ptr`` int64[n+1], ``col`` int32[nnz]),
symmetric, rows strictly ascending, no self-loops.  Pass numpy arrays for
host input (results come back as numpy) or CUDA torch tensors for
device-resident input (results come back as CUDA tensors, computed on the
tensor's device and torch's current stream).

Betweenness is Eq. 1 of Sariyuce et al., "Shattering and Compressing
Networks for Centrality Analysis": ordered pairs, no normalisation.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from ._lib import (NOALLOC_MAX_N, BCS_EINVAL, BCS_ENODEV, BCS_ENOMEM, BCS_EOVERFLOW, BCS_ECUDA, BCS_ETIMEOUT, STEP_A, STEP_D,
                   STEP_I, STEP_L, STEP_O, STEP_S, STEP_U, STEPS_ALL, ComponentsView, Csr, Opts, Stats, load)

__all__ = ["bc_plain", "bc_plain_noalloc", "bc_shattered_batch", "NOALLOC_MAX_N", "bc_shattered", "bc_sources", "debug_sssp", "shatter", "last_stats", "BcsError", "load",
           "STEP_D", "STEP_A", "STEP_I", "STEP_O", "STEP_S", "STEP_U", "STEP_L", "STEPS_ALL", "version"]

_NAMES = {BCS_EINVAL: "EINVAL", BCS_ENOMEM: "ENOMEM", BCS_ECUDA: "ECUDA", BCS_ETIMEOUT: "ETIMEOUT",
          BCS_EOVERFLOW: "EOVERFLOW", BCS_ENODEV: "ENODEV"}


class BcsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc: int):
    if rc != 0:
        raise BcsError(rc, load().bcs_last_error().decode(errors="replace"))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class _Args:
    """Keeps the marshalled buffers alive for the duration of one call."""

    def __init__(self, row_ptr, col, steps=STEPS_ALL, delta_fp32=False, stream=None, max_wait=0, autotune=False):
        self.keep = []
        self.torch = _is_torch(row_ptr)
        self.opts = Opts()
        self.opts.steps = steps
        self.opts.delta_fp32 = 1 if delta_fp32 else 0
        self.opts.device = -1
        self.opts.max_wait = max_wait
        self.opts.autotune = 1 if autotune else 0
        if self.torch:
            import torch
            if row_ptr.device.type != "cuda" or col.device.type != "cuda":
                row_ptr, col = row_ptr.cpu().numpy(), col.cpu().numpy()
                self.torch = False
            else:
                if row_ptr.dtype != torch.int64 or col.dtype != torch.int32:
                    raise TypeError("row_ptr must be int64 and col int32")
                row_ptr, col = row_ptr.contiguous(), col.contiguous()
                self.device = row_ptr.device
                self.opts.device = row_ptr.device.index if row_ptr.device.index is not None else \
                    torch.cuda.current_device()
                s = stream if stream is not None else torch.cuda.current_stream(row_ptr.device)
                self.opts.stream = ctypes.c_void_p(s.cuda_stream)
                self.keep += [row_ptr, col]
                self.csr = Csr(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr(), 1)
                return
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        self.keep += [rp, cl]
        self.csr = Csr(rp.size - 1, cl.size, rp.ctypes.data, cl.ctypes.data if cl.size else None, 0)

    @property
    def n(self) -> int:
        return int(self.csr.n)

    def out(self, n: int):
        if self.torch:
            import torch
            t = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)[:n]
            return t, t.data_ptr()
        a = np.zeros(n, dtype=np.float64)
        return a, a.ctypes.data


def _csr_of(graph_or_rp, col=None):
    if col is None:  # an object with row_ptr / col attributes
        return graph_or_rp.row_ptr, graph_or_rp.col
    return graph_or_rp, col


def bc_plain(row_ptr, col=None, *, delta_fp32: bool = False, stream=None, order: bool = False,
             autotune: bool = False):
    """Plain Brandes (Algorithm 1) on the whole graph: bc[v] for every v.
    order=True renumbers the graph in BFS order first (Section 4.1);
    autotune=True times the large-piece kernels once per shape bucket."""
    rp, cl = _csr_of(row_ptr, col)
    a = _Args(rp, cl, steps=STEPS_ALL | (STEP_O if order else 0), delta_fp32=delta_fp32, stream=stream,
              autotune=autotune)
    out, ptr = a.out(a.n)
    _check(load().bcs_bc_plain(ctypes.byref(a.csr), ctypes.byref(a.opts), ptr))
    return out


def bc_shattered(row_ptr, col=None, *, steps: int = STEPS_ALL, delta_fp32: bool = False, stream=None,
                 max_wait: int = 0, autotune: bool = False, order: bool = False, side: bool = False,
                 unequal: bool = False, resplit: bool = False):
    """Shattered + compressed BC (Section 3), equal to Eq. 1 on the input.

    max_wait bounds the polls of device-side waits (0: default, < 0: give up
    at once, which makes the call fail with ETIMEOUT; for tests).  autotune
    times the small-piece work splits once per shape bucket and reuses the
    fastest.  order=True renumbers the graph in BFS order first (Section 4.1).
    side=True also takes side vertices out of the pieces (Section 3.3.2).
    unequal=True merges identical vertices whatever their reach.
    resplit=True repeats the preprocessing to a fixpoint: split the merged
    pieces at their cut vertices, merge again, until a round merges nothing."""
    rp, cl = _csr_of(row_ptr, col)
    extra = (STEP_O if order else 0) | (STEP_S if side else 0) | (STEP_U if unequal else 0) | \
        (STEP_L if resplit else 0)
    a = _Args(rp, cl, steps=steps | extra, delta_fp32=delta_fp32, stream=stream, max_wait=max_wait,
              autotune=autotune)
    out, ptr = a.out(a.n)
    _check(load().bcs_bc_shattered(ctypes.byref(a.csr), ctypes.byref(a.opts), ptr))
    return out


def bc_shattered_batch(vtx_off, row_ptr, col=None, *, steps: int = STEPS_ALL, delta_fp32: bool = False,
                       stream=None, side: bool = False, unequal: bool = False, resplit: bool = False,
                       autotune: bool = False):
    """BC of many independent graphs packed in one CSR (graph g owns the
    vertices [vtx_off[g], vtx_off[g+1]); no edge may join two graphs).
    side=True also takes side vertices out of the pieces (Section 3.3.2);
    unequal=True merges identical vertices whatever their reach; resplit=True
    repeats splitting and merging until a round merges nothing; autotune as
    for bc_shattered."""
    rp, cl = _csr_of(row_ptr, col)
    extra = (STEP_S if side else 0) | (STEP_U if unequal else 0) | (STEP_L if resplit else 0)
    a = _Args(rp, cl, steps=steps | extra, delta_fp32=delta_fp32, stream=stream, autotune=autotune)
    off = np.ascontiguousarray(np.asarray(vtx_off, dtype=np.int64).reshape(-1))
    out, ptr = a.out(a.n)
    _check(load().bcs_bc_shattered_batch(off.ctypes.data, off.size - 1, ctypes.byref(a.csr), ctypes.byref(a.opts),
                                         ptr))
    return out


def bc_plain_noalloc(row_ptr, col=None, *, delta_fp32: bool = False, stream=None):
    """Plain Brandes without any device allocation by the library.

    For callers that cannot let a library allocate GPU memory (all device
    memory handed to their own pool, or a loop that must not enter the
    allocator).  Needs CUDA torch tensors and at most NOALLOC_MAX_N vertices;
    the result tensor is allocated here, by torch, not by the library.  The
    library's state lives in a static device array shared by all calls, so
    calls must not overlap on the GPU.
    """
    rp, cl = _csr_of(row_ptr, col)
    a = _Args(rp, cl, delta_fp32=delta_fp32, stream=stream)
    if not a.torch:
        raise TypeError("bc_plain_noalloc needs CUDA tensors (device-resident graph and output)")
    out, ptr = a.out(a.n)
    _check(load().bcs_bc_plain_noalloc(ctypes.byref(a.csr), ctypes.byref(a.opts), ptr))
    return out


def bc_sources(row_ptr, col=None, sources=None, *, delta_fp32: bool = False, stream=None, order: bool = False):
    """sum over the given sources s of delta_s(v) (Eq. 2), delta_s(s) = 0.
    order=True renumbers the graph in BFS order first (Section 4.1)."""
    rp, cl = _csr_of(row_ptr, col)
    a = _Args(rp, cl, steps=STEPS_ALL | (STEP_O if order else 0), delta_fp32=delta_fp32, stream=stream)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1))
    out, ptr = a.out(a.n)
    _check(load().bcs_bc_sources(ctypes.byref(a.csr), src.ctypes.data if src.size else None, src.size,
                                 ctypes.byref(a.opts), ptr))
    return out


@dataclass
class SSSP:
    d: np.ndarray        # int32, -1 unreachable
    sig_m: np.ndarray    # float64: sigma = sig_m * 2**sig_e
    sig_e: np.ndarray    # int32
    delta: np.ndarray    # float64


def debug_sssp(row_ptr, col=None, s: int = 0, *, delta_fp32: bool = False) -> SSSP:
    """One source of Algorithm 1 on the GPU (test hook)."""
    rp, cl = _csr_of(row_ptr, col)
    a = _Args(rp, cl, delta_fp32=delta_fp32)
    n = a.n
    d = np.zeros(n, np.int32)
    sm = np.zeros(n, np.float64)
    se = np.zeros(n, np.int32)
    de = np.zeros(n, np.float64)
    _check(load().bcs_debug_sssp(ctypes.byref(a.csr), s, ctypes.byref(a.opts), d.ctypes.data, sm.ctypes.data,
                                 se.ctypes.data, de.ctypes.data))
    return SSSP(d, sm, se, de)


@dataclass
class Components:
    """Pieces of the shattered graph (host copies of bcs_components_view)."""
    n: int
    piece_vtx_off: np.ndarray
    piece_N: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    org: np.ndarray
    reach: np.ndarray
    ident: np.ndarray
    member_off: np.ndarray
    member: np.ndarray
    bc_pre: np.ndarray
    bc_corr: np.ndarray

    @property
    def n_pieces(self) -> int:
        return int(self.piece_vtx_off.size - 1)

    def members_of(self, m: int) -> np.ndarray:
        return self.member[self.member_off[m]:self.member_off[m + 1]]


def _np(ptr, count, dtype):
    if count == 0:
        return np.zeros(0, dtype=dtype)
    ct = np.ctypeslib.as_ctypes_type(np.dtype(dtype))
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ct)), shape=(count,)).copy()


def shatter(row_ptr, col=None, *, steps: int = STEPS_ALL) -> Components:
    """Apply the steps once (D, A, I in that order) and return the pieces."""
    rp, cl = _csr_of(row_ptr, col)
    a = _Args(rp, cl, steps=steps)
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.bcs_shatter(ctypes.byref(a.csr), ctypes.byref(a.opts), ctypes.byref(h)))
    try:
        v = ComponentsView()
        _check(lib.bcs_components_get(h, ctypes.byref(v)))
        P, M, E, S, n = v.n_pieces, v.n_merged, v.n_entries, v.n_members, v.n
        return Components(
            n=n,
            piece_vtx_off=_np(v.piece_vtx_off, P + 1, np.int64),
            piece_N=_np(v.piece_N, P, np.int64),
            row_ptr=_np(v.row_ptr, M + 1, np.int64),
            col=_np(v.col, E, np.int32),
            org=_np(v.org, M, np.int32),
            reach=_np(v.reach, M, np.int32),
            ident=_np(v.ident, M, np.int32),
            member_off=_np(v.member_off, M + 1, np.int64),
            member=_np(v.member, S, np.int32),
            bc_pre=_np(v.bc_pre, n, np.int64),
            bc_corr=_np(v.bc_corr, M, np.float64),
        )
    finally:
        lib.bcs_components_free(h)


def last_stats() -> dict:
    """Statistics of this thread's last successful call."""
    s = Stats()
    _check(load().bcs_last_stats(ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in Stats._fields_}


def version() -> int:
    return int(load().bcs_version())
