"""The whole-GPU Bc-Reach kernel (large pieces of small BFS depth) and the
one-batch-per-CTA kernel of mid-size pieces (the same batch, its waits
CTA-wide) against the oracle, through the C ABI (needs a CUDA device).

BCS_LARGE_PATH=wide_all|mid_all sends every piece, however small, through
one of them, so graphs the oracle finishes in seconds cover them: source batches
with a ragged end and repeated sources, reach and ident from shattering,
rows long enough to be split over several warps, and path counts past the
64-bit integers and past the double range.  Bars as in test_gpu_parity.py.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
ALL = oracle.STEP_D | oracle.STEP_A | oracle.STEP_I


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b))) / max(1.0, float(np.max(np.abs(b))))


def largest_component(g):
    """The largest connected component, renumbered (input tooling only)."""
    A = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    _, lab = connected_components(A, directed=False)
    keep = np.flatnonzero(lab == np.argmax(np.bincount(lab)))
    e = g.edges()
    m = np.isin(e[:, 0], keep) & np.isin(e[:, 1], keep)
    remap = -np.ones(g.n, np.int64)
    remap[keep] = np.arange(keep.size)
    return gg.from_edges(keep.size, remap[e[m]])


def layered(k, layers):
    """Complete bipartite links between consecutive layers of k vertices:
    the path count from a first-layer vertex to layer l is k^(l-1)."""
    e = []
    for l in range(layers - 1):
        a = np.arange(k) + l * k
        b = np.arange(k) + (l + 1) * k
        e.append(np.stack(np.meshgrid(a, b), -1).reshape(-1, 2))
    return gg.from_edges(k * layers, np.concatenate(e))


@pytest.fixture(params=["wide_all", "mid_all"])
def wide_all(monkeypatch, request):
    """Every piece on the whole-GPU kernel, or on the one-batch-per-CTA
    kernel of mid-size pieces (the same batch, its waits CTA-wide)."""
    monkeypatch.setenv("BCS_LARGE_PATH", request.param)
    return request.param


@pytest.mark.parametrize("per_batch", [32, 64])
def test_wide_plain_and_repeated_sources(gpu, wide_all, monkeypatch, per_batch):
    """Plain Brandes on a connected Chung-Lu graph (batches of 32 or 64
    sources), then a source list of 45 entries with repeats (a ragged last
    batch; equal sources in one batch are two slots of one vertex)."""
    monkeypatch.setenv("BCS_WIDE_SOURCES", str(per_batch))
    g = largest_component(gg.chung_lu(3000, 2.2, 8.0, 7))
    ref = oracle.bc(g)
    for fp32, tol in ((False, TOL64), (True, TOL32)):
        assert rel(gpu.bc_plain(g.row_ptr, g.col, delta_fp32=fp32), ref) <= tol
        per = per_batch if wide_all == "wide_all" else 64  # the mid-size kernel's batches are 64 sources
        assert gpu.last_stats()["n_wide_batches"] == (g.n + per - 1) // per
    src = np.concatenate([np.random.default_rng(1).choice(g.n, 40, replace=False), [5, 5, 9, 9, 0]])
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), oracle.bc_sources(g, src)) <= TOL64


@pytest.mark.parametrize("seed", range(3))
def test_wide_shattered_reach_and_ident(gpu, wide_all, seed):
    """Shattered pieces (reach from degree-1 and articulation steps, ident
    from twins) all on the whole-GPU kernel."""
    g = gg.with_twins_and_pendants(gg.gnp(60 + 7 * seed, 0.06, seed), seed, 6, 12, 2)
    ref = oracle.bc(g)
    for fp32, tol in ((False, TOL64), (True, TOL32)):
        assert rel(gpu.bc_shattered(g.row_ptr, g.col, delta_fp32=fp32), ref) <= tol
        assert gpu.last_stats()["n_wide_batches"] > 0


def test_wide_split_rows(gpu, wide_all):
    """Hubs of degree far above the long-row item (64 entries): their rows
    are cut into items spread over many warps (the five largest hubs among
    the sources)."""
    g = largest_component(gg.chung_lu(20000, 2.0, 12.0, 3))
    deg = np.diff(g.row_ptr)
    assert deg.max() > 512
    src = np.random.default_rng(2).choice(g.n, 100, replace=False)
    src[:5] = np.argsort(deg)[-5:]
    ref = oracle.bc_sources(g, src)
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), ref) <= TOL64
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src, delta_fp32=True), ref) <= TOL32


def test_mid_path_counts_past_int64(gpu, monkeypatch):
    """The one-batch-per-CTA kernel on layers of 400 vertices, 28 deep (path
    counts leave the 64-bit integers after 7 levels), with a graph too deep
    for its levels (a path of 100) in the same call: that piece falls back to
    one source per CTA."""
    monkeypatch.setenv("BCS_LARGE_PATH", "mid_all")
    k, layers = 400, 28
    g = layered(k, layers)
    src = np.array([0, 1, 199, 10 * k + 3, k * layers - 1])
    ref = oracle.bc_sources(g, src)
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), ref) <= TOL64
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src, delta_fp32=True), ref) <= TOL32
    assert gpu.last_stats()["n_wide_batches"] == 1
    h = gg.disjoint_union(layered(30, 12), gg.path(100), gg.cycle(300))
    assert rel(gpu.bc_shattered(h.row_ptr, h.col, steps=oracle.STEP_I), oracle.bc(h)) <= TOL64


def test_wide_path_counts_past_int64_and_double(gpu, wide_all):
    """Layers of 400 vertices (rows of 800 entries, cut into 13 items):
    path counts grow by 400 per level, leave the 64-bit integers after 7
    levels and the double range (400^119 ~ 2^1029) before the last layer.
    (Whole-GPU kernel only: 120 layers are deeper than the mid-size kernel's
    levels; test_mid_path_counts_past_int64 covers that kernel.)"""
    if wide_all == "mid_all":
        pytest.skip("deeper than the mid-size kernel's level cap")
    k, layers = 400, 120
    g = layered(k, layers)
    src = np.array([0, 1, 199, 70 * k + 3, k * layers - 1])
    ref = oracle.bc_sources(g, src)
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), ref) <= TOL64
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src, delta_fp32=True), ref) <= TOL32


def test_wide_device_input_and_several_components(gpu, wide_all):
    """Device-resident input gives the same result; a whole graph of several
    components (plain Brandes) is ordered component by component, each from
    its smallest vertex, so batches may span components."""
    import torch
    g = largest_component(gg.chung_lu(2000, 2.3, 6.0, 11))
    ref = oracle.bc(g)
    rp, col = torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()
    assert rel(gpu.bc_plain(rp, col).cpu().numpy(), ref) <= TOL64
    h = gg.disjoint_union(gg.cycle(40), g, gg.path(7), gg.star(5), gg.gnp(1, 0.5, 0))
    assert rel(gpu.bc_plain(h.row_ptr, h.col), oracle.bc(h)) <= TOL64
    if wide_all == "wide_all":
        assert gpu.last_stats()["n_wide_batches"] > 0
    else:  # one piece that is not connected: left to one source per CTA
        assert gpu.last_stats()["n_wide_batches"] == 0
    src = np.array([0, 39, 40, 41, h.n - 1, h.n - 2, 45])
    assert rel(gpu.bc_sources(h.row_ptr, h.col, src, delta_fp32=True), oracle.bc_sources(h, src)) <= TOL32
