"""Seeded synthetic graphs (input tooling only, no betweenness arithmetic).

The heavy generators live in ``graphgen.c`` and are reached through ctypes;
the small families used by the unit tests are built here with numpy.  Every
graph comes back as a :class:`Graph` holding a CSR with int64 row offsets and
int32 columns, rows sorted ascending, no self-loops and no duplicates.

Stand-ins for the paper's DIMACS categories (Section 4, Table 1), one per
workload:

* ``config(1)``  small social-like graph: Chung-Lu core (2,000 vertices,
  gamma 2.5, mean degree 4) plus 600 pendant vertices;
* ``config(2)``  articulation-heavy: 5,000 Erdos-Renyi blocks glued at cut
  vertices plus 20% of the vertices in dangling chains;
* ``config(3)``  identical-vertex heavy: Chung-Lu core (500,000, gamma 2.1,
  mean degree 12), twin groups covering 150,000 vertices, 350,000 pendants;
* ``config(4)``  road-like: 1500 x 1500 grid minus 25% of its edges, largest
  component, trees of depth <= 8 on 10% of the perimeter vertices;
* ``batch()``    many independent Chung-Lu graphs (gamma 2.3, mean degree 8).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# Seeds of the five workloads (0xB0C0_0001 ... 0xB0C0_0005).
SEEDS = {i: 0xB0C00000 + i for i in range(1, 6)}


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
        ("col", ctypes.POINTER(ctypes.c_int32)),
    ]


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, -O2)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gg_config.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(_CSR)]
        lib.gg_chung_lu.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.POINTER(_CSR)]
        lib.gg_batch.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.POINTER(_CSR), ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))]
        lib.gg_from_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(_CSR)]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_splitmix64.argtypes = [ctypes.c_uint64]
        lib.gg_splitmix64.restype = ctypes.c_uint64
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected simple graph in CSR form (host numpy arrays)."""
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]

    def edges(self) -> np.ndarray:
        """Undirected edges (u < v) as an (m, 2) int64 array."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        mask = src < self.col
        return np.stack([src[mask], self.col[mask].astype(np.int64)], axis=1)


def _take(c: _CSR, name: str, meta: dict | None = None) -> Graph:
    lib = _load()
    n, nnz = int(c.n), int(c.nnz)
    rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    col = (np.ctypeslib.as_array(c.col, shape=(nnz,)).copy() if nnz > 0
           else np.zeros(0, dtype=np.int32))
    lib.gg_free(ctypes.cast(c.row_ptr, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(c.col, ctypes.c_void_p))
    return Graph(n, rp, col, name, meta or {})


def config(i: int, seed: int | None = None, scale_pct: int = 100) -> Graph:
    """Workload `i` (1..4) at `scale_pct` percent of its full size."""
    if i not in (1, 2, 3, 4):
        raise ValueError("config id must be 1..4 (config 5 is batch())")
    seed = SEEDS[i] if seed is None else seed
    c = _CSR()
    rc = _load().gg_config(i, seed, scale_pct, ctypes.byref(c))
    if rc != 0:
        raise RuntimeError(f"gg_config({i}) failed: {rc}")
    names = {1: "small", 2: "articulation", 3: "twins", 4: "road"}
    return _take(c, f"{names[i]}@{scale_pct}%", {"config": i, "seed": seed, "scale_pct": scale_pct})


def chung_lu(n: int, gamma: float, mean_deg: float, seed: int) -> Graph:
    c = _CSR()
    rc = _load().gg_chung_lu(n, gamma, mean_deg, seed, ctypes.byref(c))
    if rc != 0:
        raise RuntimeError(f"gg_chung_lu failed: {rc}")
    return _take(c, f"chung_lu({n},{gamma},{mean_deg})")


def batch(count: int, seed: int = SEEDS[5], n_min: int = 16, n_max: int = 65536) -> tuple[Graph, np.ndarray]:
    """`count` independent Chung-Lu graphs packed in one CSR; returns (graph, vtx_off)."""
    c = _CSR()
    off = ctypes.POINTER(ctypes.c_int64)()
    rc = _load().gg_batch(seed, count, n_min, n_max, ctypes.byref(c), ctypes.byref(off))
    if rc != 0:
        raise RuntimeError(f"gg_batch failed: {rc}")
    vtx_off = np.ctypeslib.as_array(off, shape=(count + 1,)).copy()
    _load().gg_free(ctypes.cast(off, ctypes.c_void_p))
    return _take(c, f"batch({count})", {"count": count, "seed": seed}), vtx_off


def splitmix64(x: int) -> int:
    return int(_load().gg_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


# ---------------------------------------------------------------- small families
def from_edges(n: int, edges, name: str = "") -> Graph:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    u = np.ascontiguousarray(e[:, 0].astype(np.int32))
    v = np.ascontiguousarray(e[:, 1].astype(np.int32))
    c = _CSR()
    rc = _load().gg_from_edges(n, e.shape[0], u.ctypes.data, v.ctypes.data, ctypes.byref(c))
    if rc != 0:
        raise ValueError(f"bad edge list (rc={rc})")
    return _take(c, name)


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"path({n})")


def star(n: int) -> Graph:
    """Centre 0 and n-1 leaves."""
    return from_edges(n, [(0, i) for i in range(1, n)], f"star({n})")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle({n})")


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    """Side A = 0..a-1, side B = a..a+b-1."""
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], f"K{a},{b}")


def grid(rows: int, cols: int) -> Graph:
    e = []
    for i in range(rows):
        for j in range(cols):
            v = i * cols + j
            if j + 1 < cols:
                e.append((v, v + 1))
            if i + 1 < rows:
                e.append((v, v + cols))
    return from_edges(rows * cols, e, f"grid({rows}x{cols})")


def random_tree(n: int, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    e = [(i, int(rng.integers(0, i))) for i in range(1, n)]
    return from_edges(n, e, f"tree({n},{seed})")


def gnp(n: int, p: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].shape[0]) < p
    return from_edges(n, np.stack([iu[0][keep], iu[1][keep]], axis=1), f"gnp({n},{p},{seed})")


def with_twins_and_pendants(base: Graph, seed: int, n_twins: int, n_pend: int,
                            closed_twins: int = 0) -> Graph:
    """Add open twins (copies of a vertex's neighbour set), closed twins
    (copies adjacent to the vertex and to its neighbours) and pendants."""
    rng = np.random.default_rng(seed)
    adj = [set(map(int, base.neighbors(v))) for v in range(base.n)]
    n = base.n
    edges = {(min(u, v), max(u, v)) for u in range(base.n) for v in adj[u]}
    for _ in range(n_twins):
        x = int(rng.integers(0, base.n))
        if not adj[x]:
            continue
        for y in adj[x]:
            edges.add((min(n, y), max(n, y)))
        n += 1
    for _ in range(closed_twins):
        x = int(rng.integers(0, base.n))
        for y in adj[x] | {x}:
            edges.add((min(n, y), max(n, y)))
        n += 1
    for _ in range(n_pend):
        x = int(rng.integers(0, n))
        edges.add((x, n))
        n += 1
    return from_edges(n, sorted(edges), f"{base.name}+tw{n_twins}+ctw{closed_twins}+p{n_pend}")


def with_side_vertices(base: Graph, seed: int, n_tri: int, n_grow: int = 0) -> Graph:
    """Add vertices whose neighbourhoods are cliques: n_tri new vertices, each
    joined to both ends of a uniform edge of `base`, then n_grow more, each
    joined to a uniform earlier-added vertex x and to all of x's neighbours
    (the new vertex's neighbourhood is x's closed one, a clique, and x's
    stays a clique)."""
    rng = np.random.default_rng(seed)
    ed = base.edges()
    n = base.n
    nbrs: list[list[int]] = []  # neighbourhoods of the added vertices
    out = [ed] if ed.size else []
    if n_tri and ed.shape[0]:
        pick = ed[rng.integers(0, ed.shape[0], n_tri)]
        new = np.arange(n, n + n_tri, dtype=np.int64)
        out += [np.stack([new, pick[:, 0]], 1), np.stack([new, pick[:, 1]], 1)]
        nbrs = [[int(a), int(b)] for a, b in pick]
        n += n_tri
    first = base.n
    grow = []
    for _ in range(n_grow if nbrs else 0):
        k = int(rng.integers(0, len(nbrs)))
        x = first + k
        nb = nbrs[k] + [x]
        grow += [(n, y) for y in nb]
        for y in nb:
            if y >= first:
                nbrs[y - first].append(n)
        nbrs.append(list(nb))
        n += 1
    if grow:
        out.append(np.asarray(grow, dtype=np.int64))
    edges = np.concatenate(out) if out else np.zeros((0, 2), dtype=np.int64)
    return from_edges(n, edges, f"{base.name}+side{n_tri}+grow{n_grow}")


def blow_up(base: Graph, seed: int, max_k: int = 3, p_closed: float = 0.3, n_pend: int = 0) -> Graph:
    """Replace every vertex x of `base` by a group of 1..max_k copies (open
    twins, or with probability p_closed a clique of closed twins); copies of
    adjacent vertices are all joined.  Groups of groups collapse in turn once
    merged, so the result needs several rounds of splitting and merging.
    n_pend pendants are then attached to uniform vertices."""
    rng = np.random.default_rng(seed)
    groups, n = [], 0
    edges = set()
    for _ in range(base.n):
        k = int(rng.integers(1, max_k + 1))
        grp = list(range(n, n + k))
        n += k
        if k > 1 and rng.random() < p_closed:
            edges.update((a, b) for i, a in enumerate(grp) for b in grp[i + 1:])
        groups.append(grp)
    for u, v in base.edges():
        edges.update((min(a, b), max(a, b)) for a in groups[int(u)] for b in groups[int(v)])
    for _ in range(n_pend):
        edges.add((int(rng.integers(0, n)), n))
        n += 1
    return from_edges(n, sorted(edges), f"blowup({base.name},{seed},{max_k})+p{n_pend}")


def disjoint_union(*graphs: Graph) -> Graph:
    e, off = [], 0
    for g in graphs:
        ed = g.edges()
        if ed.size:
            e.append(ed + off)
        off += g.n
    edges = np.concatenate(e) if e else np.zeros((0, 2), dtype=np.int64)
    return from_edges(off, edges, "+".join(g.name for g in graphs))


def relabel(g: Graph, seed: int) -> Graph:
    """Same graph under a seeded random permutation of the ids."""
    perm = np.random.default_rng(seed).permutation(g.n)
    ed = g.edges()
    return from_edges(g.n, perm[ed] if ed.size else ed, f"{g.name}~{seed}")
