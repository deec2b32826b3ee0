"""Oracle: plain, slow, obviously correct CPU reference for the hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_1209_6007_gb300``) never imports it, and this package never
imports the product.  The two share no code; they share only the seeded
input generators in ``graphgen``.

Functions and the passages they follow:

* :func:`bc` - Eq. 1 over ordered pairs, computed with Algorithm 1 (Bc-Org)
  in FP64 with an extended exponent for the path counts (``brandes.c``).
* :func:`bc_sources` - the partial sum over a list of sources (Eq. 2).
* :func:`sssp` - one source of Algorithm 1: d, sigma (mantissa, exponent),
  delta (Eq. 3).
* :func:`pair_stats` - sum over reachable ordered pairs of d(s,t) - 1.
* :func:`shatter` - the pieces of Section 3 by their definitions
  (``shatter.c`` + set grouping here): the 2-core left by degree-1 removal
  (Section 3.3.1), the biconnected components of Section 2 / 3.2.1, the reach
  of every (piece, vertex) slot (Section 3.2, Eq. 4), and the type-I /
  type-II identical-vertex classes of Section 3.3.3 restricted to equal reach
  (the paper leaves reach and ident together unspecified; equal-reach-only
  merging is the default reading, and ``STEP_U`` gives the classes of the
  other reading, keyed on the neighbourhood alone).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from collections import defaultdict
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("brandes.c", "shatter.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STEP_D, STEP_A, STEP_I = 1, 2, 4
STEP_U = 32  # with STEP_I: classes keyed on the neighbourhood alone (any reach)

_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2 -fopenmp) next to its sources."""
    with _lock:
        newest = max(os.path.getmtime(s) for s in _SRCS)
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", *_SRCS, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_bc.argtypes = [i64, vp, vp, c_int, vp]
        lib.oracle_bc_sources.argtypes = [i64, vp, vp, vp, i64, c_int, vp]
        lib.oracle_sssp.argtypes = [i64, vp, vp, i64, vp, vp, vp, vp]
        lib.oracle_pair_stats.argtypes = [i64, vp, vp, c_int, ctypes.POINTER(ctypes.c_double), _i64p]
        lib.oracle_two_core.argtypes = [i64, vp, vp, vp, vp]
        lib.oracle_components.argtypes = [i64, vp, vp, vp, vp]
        lib.oracle_components.restype = i64
        lib.oracle_blocks.argtypes = [i64, vp, vp, vp, vp]
        lib.oracle_blocks.restype = i64
        lib.oracle_reach.argtypes = [i64, vp, vp, i64, vp, vp, vp]
        _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col


def bc(g, threads: int | None = None) -> np.ndarray:
    """Betweenness of every vertex, ordered pairs, no normalisation (Eq. 1)."""
    rp, col = _csr(g)
    out = np.zeros(max(g.n, 1), dtype=np.float64)
    rc = _load().oracle_bc(g.n, rp.ctypes.data, col.ctypes.data, threads or default_threads(), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_bc failed: {rc}")
    return out[:g.n]


def bc_sources(g, sources, threads: int | None = None) -> np.ndarray:
    """sum over s in `sources` of delta_s(v), for every v (Eq. 2)."""
    rp, col = _csr(g)
    src = np.ascontiguousarray(sources, dtype=np.int64)
    out = np.zeros(max(g.n, 1), dtype=np.float64)
    rc = _load().oracle_bc_sources(g.n, rp.ctypes.data, col.ctypes.data, src.ctypes.data, src.size,
                                   threads or default_threads(), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_bc_sources failed: {rc}")
    return out[:g.n]


@dataclass
class SSSP:
    d: np.ndarray       # int32, -1 = unreachable
    sig_m: np.ndarray   # float64 mantissa in [0.5, 1), 0 when unreachable
    sig_e: np.ndarray   # int64 exponent: sigma = sig_m * 2**sig_e
    delta: np.ndarray   # float64 delta_s(v)

    def sigma_float(self) -> np.ndarray:
        """sigma as float64 (inf where it does not fit)."""
        with np.errstate(over="ignore"):
            return np.ldexp(self.sig_m, np.clip(self.sig_e, -2000, 2000).astype(np.int32))


def sssp(g, s: int) -> SSSP:
    rp, col = _csr(g)
    n = g.n
    d = np.zeros(n, dtype=np.int32)
    sm = np.zeros(n, dtype=np.float64)
    se = np.zeros(n, dtype=np.int64)
    de = np.zeros(n, dtype=np.float64)
    rc = _load().oracle_sssp(n, rp.ctypes.data, col.ctypes.data, s, d.ctypes.data, sm.ctypes.data,
                             se.ctypes.data, de.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_sssp failed: {rc}")
    return SSSP(d, sm, se, de)


def pair_stats(g, threads: int | None = None) -> tuple[float, int]:
    """(sum over reachable ordered pairs s != t of d(s,t) - 1, number of such pairs)."""
    rp, col = _csr(g)
    tot = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    rc = _load().oracle_pair_stats(g.n, rp.ctypes.data, col.ctypes.data, threads or default_threads(),
                                   ctypes.byref(tot), ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError(f"oracle_pair_stats failed: {rc}")
    return float(tot.value), int(cnt.value)


def two_core(g, mask=None) -> np.ndarray:
    rp, col = _csr(g)
    out = np.zeros(max(g.n, 1), dtype=np.uint8)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rc = _load().oracle_two_core(g.n, rp.ctypes.data, col.ctypes.data, None if m is None else m.ctypes.data,
                                 out.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_two_core failed")
    return out[:g.n].astype(bool)


def components(g, mask=None) -> tuple[int, np.ndarray]:
    rp, col = _csr(g)
    lab = np.zeros(max(g.n, 1), dtype=np.int32)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cnt = _load().oracle_components(g.n, rp.ctypes.data, col.ctypes.data,
                                    None if m is None else m.ctypes.data, lab.ctypes.data)
    if cnt < 0:
        raise RuntimeError("oracle_components failed")
    return int(cnt), lab[:g.n]


def blocks(g, mask=None) -> tuple[int, np.ndarray]:
    """(number of biconnected components, block id per CSR entry or -1)."""
    rp, col = _csr(g)
    eb = np.zeros(max(g.nnz, 1), dtype=np.int64)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cnt = _load().oracle_blocks(g.n, rp.ctypes.data, col.ctypes.data, None if m is None else m.ctypes.data,
                                eb.ctypes.data)
    if cnt < 0:
        raise RuntimeError(f"oracle_blocks failed: {cnt}")
    return int(cnt), eb[:g.nnz]


def reach(g, pieces: list[list[int]]) -> list[np.ndarray]:
    """reach of each (piece, vertex) slot, in the order the pieces list them."""
    rp, col = _csr(g)
    off = np.zeros(len(pieces) + 1, dtype=np.int64)
    for i, p in enumerate(pieces):
        off[i + 1] = off[i] + len(p)
    vtx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    for i, p in enumerate(pieces):
        vtx[off[i]:off[i + 1]] = p
    out = np.zeros(max(int(off[-1]), 1), dtype=np.int64)
    rc = _load().oracle_reach(g.n, rp.ctypes.data, col.ctypes.data, len(pieces), off.ctypes.data,
                              vtx.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_reach failed")
    return [out[off[i]:off[i + 1]].copy() for i in range(len(pieces))]


@dataclass
class Piece:
    """One component of the shattered graph, in original ids."""
    vertices: tuple            # sorted original ids
    reach: dict                # original id -> reach of its slot in this piece
    classes: tuple             # sorted tuples (size >= 2) of identical vertices
    N: int                     # size of the original connected component

    def key(self):
        return self.vertices


def shatter(g, steps: int = STEP_D | STEP_A | STEP_I) -> list[Piece]:
    """The pieces the shattering/compression steps leave, by definition.

    * D (degree-1 removal, Section 3.3.1, applied until nothing changes):
      keep only the 2-core.  A connected component that is a tree has an
      empty 2-core and leaves no piece.
    * A (articulation vertices and bridges, Sections 3.2.1-3.2.2): pieces are
      the biconnected components of what is kept; without A they are its
      connected components.  Pieces of one vertex carry no pair and are not
      listed.
    * reach of every slot (Section 3.2, Eq. 4), see ``oracle_reach``.
    * I (identical vertices, Section 3.3.3): inside each piece, vertices with
      the same open neighbourhood (type I) or the same closed neighbourhood
      (type II) within the piece, and the same reach, form a class; with U
      as well, the reach is left out of the key (the section does not settle
      how reach and ident combine; both readings are offered).
    """
    n = g.n
    keep = two_core(g) if steps & STEP_D else np.ones(n, dtype=bool)
    pieces: list[list[int]] = []
    if steps & STEP_A:
        nb, eb = blocks(g, keep.astype(np.uint8))
        members = [set() for _ in range(nb)]
        src = np.repeat(np.arange(n), g.degrees())
        for k in np.nonzero(eb >= 0)[0]:
            b = int(eb[k])
            members[b].add(int(src[k]))
            members[b].add(int(g.col[k]))
        pieces = [sorted(m) for m in members if len(m) >= 2]
    else:
        nc, lab = components(g, keep.astype(np.uint8))
        groups = defaultdict(list)
        for v in np.nonzero(keep)[0]:
            groups[int(lab[v])].append(int(v))
        pieces = [sorted(p) for p in groups.values() if len(p) >= 2]
    pieces.sort()
    reaches = reach(g, pieces)
    _, cc = components(g)
    ccsize = np.bincount(cc, minlength=1) if n else np.zeros(0)
    out = []
    for p, r in zip(pieces, reaches):
        pset = set(p)
        rmap = {v: int(x) for v, x in zip(p, r)}
        classes = []
        if steps & STEP_I:
            nb_open = {v: frozenset(int(w) for w in g.neighbors(v) if int(w) in pset) for v in p}
            for closed in (False, True):
                grp = defaultdict(list)
                for v in p:
                    key = (nb_open[v] | {v}) if closed else nb_open[v]
                    grp[(key, None if steps & STEP_U else rmap[v])].append(v)
                classes += [tuple(sorted(c)) for c in grp.values() if len(c) >= 2]
        out.append(Piece(tuple(p), rmap, tuple(sorted(classes)), int(ccsize[cc[p[0]]])))
    return out
