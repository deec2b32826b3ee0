"""GPU path against the oracle, through the C ABI (needs a CUDA device).

Bars (from the arithmetic of each side):
* distances, path counts below 2^53, the partition, reach and ident:
  bit-exact;
* bc in FP64: max|gpu - oracle| <= 1e-12 * max|oracle|;
* bc with the FP32 dependency recurrence: <= 1e-5 * max|oracle|.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
ALL = oracle.STEP_D | oracle.STEP_A | oracle.STEP_I


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b))) / max(1.0, float(np.max(np.abs(b))))


def on_device(g):
    import torch
    return torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()


def families():
    out = [gg.path(2), gg.path(3), gg.path(40), gg.star(6), gg.cycle(9), gg.cycle(10), gg.complete(7),
           gg.complete_bipartite(3, 5), gg.grid(12, 9), gg.random_tree(60, 3)]
    for seed in range(6):
        base = gg.gnp(30 + 7 * seed, 0.08 + 0.02 * seed, seed)
        out.append(gg.with_twins_and_pendants(base, seed, 4, 10, 2))
    out.append(gg.disjoint_union(gg.cycle(5), gg.path(4), gg.complete(4), gg.star(5), gg.gnp(1, 0.5, 0)))
    out.append(gg.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4)]))  # C4 + pendant
    out.append(gg.config(1, scale_pct=10))
    return out


FAMILIES = families()


# ----------------------------------------------------------- single source
@pytest.mark.parametrize("s", [0, 7, 1234, 2599])
def test_sssp_bit_exact_config1(gpu, s):
    g = gg.config(1)
    ref = oracle.sssp(g, s)
    got = gpu.debug_sssp(g.row_ptr, g.col, s)
    assert np.array_equal(got.d, ref.d)
    reach = ref.d >= 0
    sig_ref = ref.sigma_float()
    sig_got = np.ldexp(got.sig_m, got.sig_e)
    assert np.all(sig_ref[reach] < 2.0 ** 53)
    assert np.array_equal(sig_got[reach], sig_ref[reach])
    assert np.all(got.sig_m[~reach] == 0)
    assert rel(got.delta, ref.delta) <= TOL64


def test_sssp_grid_beyond_double_range(gpu):
    """Path counts up to C(1398, 699) ~ 2^1392: the per-level exponent keeps them."""
    side = 700
    g = gg.grid(side, side)
    ref = oracle.sssp(g, 0)
    got = gpu.debug_sssp(g.row_ptr, g.col, 0)
    assert np.array_equal(got.d, ref.d)
    # compare sigma as (log2) magnitudes: m * 2^e on both sides
    lr = np.log2(ref.sig_m) + ref.sig_e
    lg = np.log2(got.sig_m) + got.sig_e
    assert np.max(np.abs(lr - lg)) < 1e-9
    small = ref.sig_e < 53
    assert np.array_equal(np.ldexp(got.sig_m[small], got.sig_e[small]), np.ldexp(ref.sig_m[small], ref.sig_e[small].astype(np.int32)))
    assert lg[-1] > 1024  # the far corner's count is beyond the double range
    assert rel(got.delta, ref.delta) <= TOL64
    got32 = gpu.debug_sssp(g.row_ptr, g.col, 0, delta_fp32=True)
    assert rel(got32.delta, ref.delta) <= TOL32


# ------------------------------------------------------------- plain
@pytest.mark.parametrize("g", FAMILIES, ids=lambda g: g.name)
def test_plain_families(gpu, g):
    ref = oracle.bc(g)
    assert rel(gpu.bc_plain(g.row_ptr, g.col), ref) <= TOL64
    assert rel(gpu.bc_plain(g.row_ptr, g.col, delta_fp32=True), ref) <= TOL32


def test_plain_config1_host_and_device(gpu):
    g = gg.config(1)
    ref = oracle.bc(g)
    assert rel(gpu.bc_plain(g.row_ptr, g.col), ref) <= TOL64
    rp, col = on_device(g)
    got = gpu.bc_plain(rp, col)
    assert got.is_cuda
    assert rel(got.cpu().numpy(), ref) <= TOL64
    assert rel(gpu.bc_plain(rp, col, delta_fp32=True).cpu().numpy(), ref) <= TOL32


# ------------------------------------------------------------- shattered
@pytest.mark.parametrize("steps", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("g", FAMILIES, ids=lambda g: g.name)
def test_shattered_families(gpu, g, steps):
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, steps=steps), ref) <= TOL64


@pytest.mark.parametrize("steps", [1, 3, 7])
def test_shattered_config1(gpu, steps):
    g = gg.config(1)
    ref = oracle.bc(g)
    rp, col = on_device(g)
    assert rel(gpu.bc_shattered(rp, col, steps=steps).cpu().numpy(), ref) <= TOL64
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, steps=steps, delta_fp32=True), ref) <= TOL32


def test_autotuned_split_gives_the_same_result(gpu):
    """The autotuner times a few small-path work splits into a scratch
    accumulator on the first call of a shape bucket, then reuses the pick."""
    g = gg.config(2, scale_pct=3)
    ref = oracle.bc(g)
    for _ in range(2):
        assert rel(gpu.bc_shattered(g.row_ptr, g.col, autotune=True), ref) <= TOL64
        st = gpu.last_stats()
        assert st["small_ng_cap"] in (4, 8)
        assert st["small_smem_budget"] in (100 * 1024, 72 * 1024, 54 * 1024)


def test_autotuned_threshold_gives_the_same_result(gpu):
    """Pieces of about a thousand vertices need between 40 and 100 KB of
    shared memory for one source, between the threshold candidates: the
    autotuner times the candidates over the pieces (into a scratch
    accumulator), keeps one, and the result, with FP64 and FP32 dependencies,
    is the oracle's; later calls reuse the choice."""
    g = gg.disjoint_union(*[gg.chung_lu(n, 2.5, 8.0, n) for n in (700, 1000, 1300, 1600)],
                          gg.config(2, scale_pct=1))
    ref = oracle.bc(g)
    limits = set()
    for fp32, tol in ((False, TOL64), (True, TOL32), (False, TOL64)):
        assert rel(gpu.bc_shattered(g.row_ptr, g.col, autotune=True, delta_fp32=fp32), ref) <= tol
        st = gpu.last_stats()
        assert st["tuned"] & 1
        assert st["small_limit"] in (100 * 1024, 64 * 1024, 40 * 1024)
        limits.add(st["small_limit"])
    assert len(limits) == 1
    gpu.bc_shattered(g.row_ptr, g.col)
    assert gpu.last_stats()["small_limit"] == 100 * 1024  # without the autotuner: the fixed limit


def test_autotuned_large_kernel_gives_the_same_result(gpu):
    """A piece with thousands of sources: the autotuner times the whole-GPU
    kernel, 32-source batches and one source per CTA on samples of its
    sources, runs the piece on the fastest, and the result is the oracle's."""
    g = gg.chung_lu(8000, 2.3, 6.0, 21)
    ref = oracle.bc(g)
    for fp32, tol in ((False, TOL64), (True, TOL32)):
        assert rel(gpu.bc_shattered(g.row_ptr, g.col, autotune=True, delta_fp32=fp32), ref) <= tol
        st = gpu.last_stats()
        assert st["tuned"] in (1 << 1, 1 << 2, 1 << 3)
        assert st["n_large_sources"] > 0
    assert rel(gpu.bc_plain(g.row_ptr, g.col, autotune=True), ref) <= TOL64


def test_shattered_articulation_scaled(gpu):
    """Config 2 at 5% of its blocks: full oracle in seconds, many pieces."""
    g = gg.config(2, scale_pct=5)
    ref = oracle.bc(g)
    got = gpu.bc_shattered(g.row_ptr, g.col)
    assert rel(got, ref) <= TOL64
    st = gpu.last_stats()
    assert st["n_pieces"] > 100
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, delta_fp32=True), ref) <= TOL32


# ------------------------------------------------------------ partition
def canon_gpu(c):
    out = {}
    for p in range(c.n_pieces):
        reach, classes = {}, []
        for m in range(int(c.piece_vtx_off[p]), int(c.piece_vtx_off[p + 1])):
            mem = [int(x) for x in c.members_of(m)]
            assert int(c.ident[m]) == len(mem)
            assert int(c.org[m]) == min(mem)
            for x in mem:
                reach[x] = int(c.reach[m])
            if len(mem) >= 2:
                classes.append(tuple(sorted(mem)))
        out[tuple(sorted(reach))] = (reach, sorted(classes), int(c.piece_N[p]))
    return out


def canon_oracle(pieces):
    return {p.vertices: (dict(p.reach), sorted(p.classes), p.N) for p in pieces}


@pytest.mark.parametrize("steps", [0, 1, 2, 3, 4, 5, 6, 7])
def test_partition_bit_exact(gpu, steps):
    for g in [gg.config(1), gg.config(2, scale_pct=2), gg.complete_bipartite(3, 4), gg.complete(5),
              gg.with_twins_and_pendants(gg.gnp(40, 0.1, 9), 9, 6, 8, 3)]:
        got = canon_gpu(gpu.shatter(g.row_ptr, g.col, steps=steps))
        ref = canon_oracle(oracle.shatter(g, steps))
        assert got == ref, g.name


def holey_grid(side, frac, seed):
    """side x side grid with a seeded fraction of its edges removed."""
    g = gg.grid(side, side)
    e = g.edges()
    keep = np.random.default_rng(seed).random(e.shape[0]) >= frac
    return gg.from_edges(g.n, e[keep], f"holey_grid({side},{frac})")


@pytest.mark.parametrize("g", [holey_grid(40, 0.25, 1), holey_grid(30, 0.4, 2), gg.config(3, scale_pct=1),
                               gg.config(4, scale_pct=1)], ids=lambda g: g.name)
def test_partition_and_bc_structured(gpu, g):
    """Biconnected split on high-diameter, holey and twin-heavy graphs."""
    got = canon_gpu(gpu.shatter(g.row_ptr, g.col, steps=ALL))
    assert got == canon_oracle(oracle.shatter(g, ALL))
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col), ref) <= TOL64
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, delta_fp32=True), ref) <= TOL32


# --------------------------------------------- full size, sampled sources
def test_articulation_full_size_sources_vs_oracle(gpu):
    """Config 2 at full size: plain Brandes on 256 seeded sources against the
    oracle's partial sums (Eq. 2)."""
    g = gg.config(2)
    rng = np.random.default_rng(0xB0C00002)
    src = rng.choice(g.n, size=256, replace=False)
    ref = oracle.bc_sources(g, src)
    got = gpu.bc_sources(g.row_ptr, g.col, src)
    assert rel(got, ref) <= TOL64


def test_mid_size_piece(gpu):
    """A piece of ~2,500 vertices: more shared memory than the small path
    gives one source, so it runs on the global-memory path."""
    g = gg.chung_lu(3000, 2.3, 8.0, 5)
    ref = oracle.bc(g)
    for fn in (gpu.bc_plain, gpu.bc_shattered):
        for fp32, tol in ((False, TOL64), (True, TOL32)):
            assert rel(fn(g.row_ptr, g.col, delta_fp32=fp32), ref) <= tol
            assert gpu.last_stats()["n_large_sources"] > 0


# ----------------------------------------------------- BFS ordering (4.1)
@pytest.mark.parametrize("g", [gg.config(1), gg.disjoint_union(gg.config(1), gg.cycle(50), gg.path(2), gg.star(9)),
                               gg.config(2, scale_pct=3), gg.grid(30, 20)], ids=lambda g: g.name)
def test_bfs_order_gives_the_same_bc(gpu, g):
    """Renumbering in BFS order (components contiguous, rows re-sorted) and
    mapping back leaves every result unchanged up to rounding."""
    ref = oracle.bc(g)
    assert rel(gpu.bc_plain(g.row_ptr, g.col, order=True), ref) <= TOL64
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, order=True), ref) <= TOL64
    rp, col = on_device(g)
    assert rel(gpu.bc_shattered(rp, col, order=True, delta_fp32=True).cpu().numpy(), ref) <= TOL32
    src = np.random.default_rng(3).choice(g.n, size=min(40, g.n), replace=False)
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src, order=True), oracle.bc_sources(g, src)) <= TOL64


@pytest.mark.parametrize("cfg", [3, 4], ids=["twins", "road"])
def test_large_full_size_sources_vs_oracle(gpu, cfg):
    """The twin-heavy (n = 970k) and road-like (n = 2.26M, diameter in the
    thousands) workloads at full size: plain Brandes on 256 seeded sources
    against the oracle's partial sums."""
    g = gg.config(cfg)
    rng = np.random.default_rng(0xB0C00000 + cfg)
    src = rng.choice(g.n, size=256, replace=False)
    ref = oracle.bc_sources(g, src)
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), ref) <= TOL64


@pytest.mark.parametrize("cfg,pct", [(3, 5), (4, 3)], ids=["twins-5pct", "road-3pct"])
def test_shattered_matches_plain_above_oracle_scale(gpu, cfg, pct):
    """Above the size the oracle finishes in seconds: shattered (FP64 and
    FP32 dependencies) against plain Brandes, both on the GPU (Thm. 1)."""
    g = gg.config(cfg, scale_pct=pct)
    rp, col = on_device(g)
    plain = gpu.bc_plain(rp, col).cpu().numpy()
    assert rel(gpu.bc_shattered(rp, col).cpu().numpy(), plain) <= TOL64
    assert rel(gpu.bc_shattered(rp, col, delta_fp32=True).cpu().numpy(), plain) <= TOL32


# ------------------------------------------- 32-source batches, large pieces
LARGE_PATHS = ["batched", "per_source"]


@pytest.mark.parametrize("path", LARGE_PATHS)
def test_batched_sources_disconnected_and_ragged(gpu, path, monkeypatch):
    """Pieces too large for shared memory run 32 sources per CTA (or one per
    CTA; both kernels, forced); a source list of 45 entries (a ragged last
    batch) with repeats, on a graph with several components (most sources do
    not reach most vertices)."""
    monkeypatch.setenv("BCS_LARGE_PATH", path)
    g = gg.disjoint_union(gg.config(1), gg.chung_lu(3000, 2.5, 5.0, 3), gg.cycle(700))
    rng = np.random.default_rng(11)
    src = np.concatenate([rng.choice(g.n, size=40, replace=False), [5, 5, 9, 9, 2600]])
    ref = oracle.bc_sources(g, src)
    for fp32, tol in ((False, TOL64), (True, TOL32)):
        assert rel(gpu.bc_sources(g.row_ptr, g.col, src, delta_fp32=fp32), ref) <= tol
    assert rel(gpu.bc_plain(g.row_ptr, g.col), oracle.bc(g)) <= TOL64


@pytest.mark.parametrize("path", LARGE_PATHS)
def test_batched_sources_path_counts_beyond_double(gpu, path, monkeypatch):
    """Sources at and near the corners of a 700 x 700 grid: path counts reach
    2^1392, so each (level, source) pair of a batch gets its own exponent."""
    monkeypatch.setenv("BCS_LARGE_PATH", path)
    side = 700
    g = gg.grid(side, side)
    src = [0, 1, side, side * side - 1, side * side - 2, (side // 2) * side + side // 2]
    ref = oracle.bc_sources(g, src)
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), ref) <= TOL64
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src, delta_fp32=True), ref) <= TOL32


# ------------------------------------------------------- uneven batches
def test_uneven_batch_matches_per_graph_oracle(gpu):
    """Workload 5's generator at small scale: 60 independent Chung-Lu graphs
    of log-uniform sizes 16..2048 in one packed CSR, one call."""
    g, off = gg.batch(60, n_min=16, n_max=2048)
    got = gpu.bc_shattered_batch(off, g.row_ptr, g.col)
    ref = oracle.bc(g)  # the packed graph is the disjoint union: same per-graph values
    assert rel(got, ref) <= TOL64
    for i in (0, 7, 59):  # and each graph on its own
        a, b = int(off[i]), int(off[i + 1])
        sub_e = g.edges()
        sub_e = sub_e[(sub_e[:, 0] >= a) & (sub_e[:, 0] < b)] - a
        sub = gg.from_edges(b - a, sub_e)
        assert rel(got[a:b], oracle.bc(sub)) <= TOL64
    got32 = gpu.bc_shattered_batch(off, g.row_ptr, g.col, delta_fp32=True)
    assert rel(got32, ref) <= TOL32


def test_batch_rejects_crossing_edges(gpu):
    g = gg.path(6)
    with pytest.raises(gpu.BcsError) as e:
        gpu.bc_shattered_batch([0, 3, 6], g.row_ptr, g.col)  # edge 2-3 joins the two graphs
    assert e.value.code == gpu._lib.BCS_EINVAL


# ------------------------------------------------- side vertices (3.3.2)
def side_graphs():
    out = [gg.complete(7), gg.complete_bipartite(2, 3), gg.disjoint_union(gg.complete(4), gg.complete(5), gg.path(3)),
           gg.from_edges(4, [(0, 1), (1, 2), (2, 0), (2, 3)])]  # triangle with a pendant
    for seed in range(4):
        base = gg.with_side_vertices(gg.gnp(30 + 10 * seed, 0.1, seed), seed, 20 + 5 * seed, 10 * seed)
        out.append(base)
        # pendants give the side vertices reach > 1, copies of them ident > 1
        out.append(gg.with_twins_and_pendants(base, seed, 6, 15, 2))
    out.append(gg.with_side_vertices(gg.config(1, scale_pct=20), 9, 300, 200))
    return out


SIDE_GRAPHS = side_graphs()


def oracle_side_count(g, steps=ALL):
    """Side vertices of the merged pieces, by definition: a class
    representative (smallest id) whose merged neighbours in its piece, at
    most 64 of them, are pairwise adjacent."""
    count = 0
    for pc in oracle.shatter(g, steps):
        drop = {v for c in pc.classes for v in c[1:]}
        keep = [v for v in pc.vertices if v not in drop]
        ks = set(keep)
        adj = {v: {int(w) for w in g.neighbors(v) if int(w) in ks} for v in keep}
        for v in keep:
            nb = sorted(adj[v])
            if 1 <= len(nb) <= 64 and all(b in adj[a] for i, a in enumerate(nb) for b in nb[i + 1:]):
                count += 1
    return count


@pytest.mark.parametrize("steps", [0, 1, 3, 4, 7])
@pytest.mark.parametrize("g", SIDE_GRAPHS, ids=lambda g: g.name)
def test_side_vertices_give_the_same_bc(gpu, g, steps):
    """Side vertices out of the pieces (Algorithm 3, all of a piece's at
    once) leave bc unchanged; the count of side vertices is the definition's."""
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, steps=steps, side=True), ref) <= TOL64
    assert gpu.last_stats()["n_side"] == oracle_side_count(g, steps)


def test_side_vertices_fp32_device_and_ordered(gpu):
    g = SIDE_GRAPHS[-1]
    ref = oracle.bc(g)
    rp, col = on_device(g)
    assert rel(gpu.bc_shattered(rp, col, side=True, delta_fp32=True).cpu().numpy(), ref) <= TOL32
    assert rel(gpu.bc_shattered(rp, col, side=True, order=True).cpu().numpy(), ref) <= TOL64
    assert gpu.last_stats()["n_side"] > 100


@pytest.mark.parametrize("path", LARGE_PATHS)
def test_side_vertices_on_a_large_piece(gpu, path, monkeypatch):
    """A piece too large for shared memory: the side sources run one per
    CTA from the source map (the 32-source kernel is not used with a map)."""
    monkeypatch.setenv("BCS_LARGE_PATH", path)
    g = gg.with_side_vertices(gg.chung_lu(3000, 2.5, 6, 11), 12, 3000, 1500)
    ref = oracle.bc(g)
    got = gpu.bc_shattered(g.row_ptr, g.col, side=True)
    st = gpu.last_stats()
    assert rel(got, ref) <= TOL64
    assert st["n_side"] > 2000 and st["n_large_sources"] > 0


def test_side_vertices_in_a_batch_and_scaled_articulation(gpu):
    g, off = gg.batch(40, n_min=16, n_max=1024)
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered_batch(off, g.row_ptr, g.col, side=True), ref) <= TOL64
    g = gg.config(2, scale_pct=5)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, side=True), oracle.bc(g)) <= TOL64
    assert gpu.last_stats()["n_side"] > 0


# ------------------------------------- identical vertices of unequal reach
def unequal_graphs():
    out = [gg.from_edges(8, [(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4), (2, 5), (3, 6), (3, 7)]),  # K2,3 + pendants
           gg.with_twins_and_pendants(gg.chung_lu(400, 2.3, 5, 3), 4, 120, 200, 30)]
    for seed in range(3):
        out.append(gg.with_twins_and_pendants(gg.gnp(30 + 7 * seed, 0.08 + 0.02 * seed, seed), seed, 8, 25, 3))
    return out


UNEQUAL_GRAPHS = unequal_graphs()


def oracle_merged_count(g, steps):
    return sum(len(p.vertices) - sum(len(c) - 1 for c in p.classes) for p in oracle.shatter(g, steps))


@pytest.mark.parametrize("steps", [ALL, oracle.STEP_D | oracle.STEP_I, oracle.STEP_A | oracle.STEP_I, oracle.STEP_I])
@pytest.mark.parametrize("g", UNEQUAL_GRAPHS + FAMILIES[-8:], ids=lambda g: g.name)
def test_unequal_reach_merging_gives_the_same_bc(gpu, g, steps):
    """Classes keyed on the neighbourhood alone (members of any reach):
    fractional dependency start in Bc-Reach plus per-copy closed forms give
    bc unchanged; the merged vertex count is the definition's."""
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, steps=steps, unequal=True), ref) <= TOL64
    assert gpu.last_stats()["n_merged"] == oracle_merged_count(g, steps | oracle.STEP_U)


def test_unequal_reach_merging_merges_more_fp32_device_ordered(gpu):
    g = UNEQUAL_GRAPHS[1]
    ref = oracle.bc(g)
    rp, col = on_device(g)
    assert rel(gpu.bc_shattered(rp, col, unequal=True, delta_fp32=True).cpu().numpy(), ref) <= TOL32
    assert rel(gpu.bc_shattered(rp, col, unequal=True, order=True).cpu().numpy(), ref) <= TOL64
    merged_u = gpu.last_stats()["n_merged"]
    gpu.bc_shattered(rp, col)
    assert merged_u < gpu.last_stats()["n_merged"]


@pytest.mark.parametrize("path", LARGE_PATHS)
def test_unequal_reach_merging_on_a_large_piece(gpu, path, monkeypatch):
    """A piece too large for shared memory: both global-memory kernels take
    the fractional dependency start and source weight."""
    monkeypatch.setenv("BCS_LARGE_PATH", path)
    g = gg.with_twins_and_pendants(gg.chung_lu(3000, 2.3, 6, 5), 6, 900, 1500, 100)
    ref = oracle.bc(g)
    for fp32, tol in ((False, TOL64), (True, TOL32)):
        assert rel(gpu.bc_shattered(g.row_ptr, g.col, unequal=True, delta_fp32=fp32), ref) <= tol
        assert gpu.last_stats()["n_large_sources"] > 0


def test_unequal_reach_merging_in_a_batch(gpu):
    graphs = UNEQUAL_GRAPHS[:4]
    g = gg.disjoint_union(*graphs)
    off = np.cumsum([0] + [x.n for x in graphs])
    assert rel(gpu.bc_shattered_batch(off, g.row_ptr, g.col, unequal=True), oracle.bc(g)) <= TOL64


# --------------------------- one more articulation split after merging
def twins_joining(seed, k, pend=0):
    """Two random 2-connected parts joined only through k open twins (each
    adjacent to the same vertices of both parts): biconnected as given, and
    the twins' merged vertex is a cut vertex (the situation of Fig. 3)."""
    rng = np.random.default_rng(seed)
    na, nb = int(rng.integers(4, 12)), int(rng.integers(4, 12))
    e = []
    for off, m in ((0, na), (na, nb)):
        e += [(off + i, off + (i + 1) % m) for i in range(m)]
        e += [(off + int(a), off + int(b)) for a, b in rng.integers(0, m, (int(rng.integers(0, 4)), 2)) if a != b]
    S = list(rng.choice(na, 2, replace=False)) + list(na + rng.choice(nb, 2, replace=False))
    n = na + nb
    e += [(n + t, int(x)) for t in range(k) for x in S]
    n += k
    for _ in range(pend):
        e.append((int(rng.integers(0, n)), n))
        n += 1
    e = {(min(a, b), max(a, b)) for a, b in e}
    return gg.from_edges(n, sorted(e), f"twins_joining({seed},{k},{pend})")


RESPLIT_GRAPHS = [twins_joining(s, k, p) for s, k, p in ((1, 2, 0), (2, 3, 0), (3, 4, 6), (4, 2, 10), (5, 3, 4))]


@pytest.mark.parametrize("steps", [ALL, oracle.STEP_A | oracle.STEP_I, oracle.STEP_I, oracle.STEP_D | oracle.STEP_A])
@pytest.mark.parametrize("g", RESPLIT_GRAPHS + FAMILIES[-8:], ids=lambda g: g.name)
def test_resplit_gives_the_same_bc(gpu, g, steps):
    """The merged pieces split again at their cut vertices (a merged cut
    vertex's copies carry 1/k of the weight beyond it per member): bc
    unchanged."""
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, steps=steps, resplit=True), ref) <= TOL64


def test_resplit_splits_at_merged_twins(gpu):
    g = RESPLIT_GRAPHS[1]
    gpu.bc_shattered(g.row_ptr, g.col)
    before = gpu.last_stats()["n_pieces"]
    gpu.bc_shattered(g.row_ptr, g.col, resplit=True)
    assert gpu.last_stats()["n_pieces"] > before


def test_resplit_larger_graphs_fp32_device_ordered_and_batch(gpu):
    for g in (gg.config(1), gg.config(2, scale_pct=3),
              gg.with_twins_and_pendants(gg.chung_lu(400, 2.3, 5, 3), 4, 120, 200, 30)):
        ref = oracle.bc(g)
        rp, col = on_device(g)
        assert rel(gpu.bc_shattered(rp, col, resplit=True).cpu().numpy(), ref) <= TOL64
        assert rel(gpu.bc_shattered(rp, col, resplit=True, delta_fp32=True).cpu().numpy(), ref) <= TOL32
        assert rel(gpu.bc_shattered(rp, col, resplit=True, order=True).cpu().numpy(), ref) <= TOL64
    graphs = RESPLIT_GRAPHS
    g = gg.disjoint_union(*graphs)
    off = np.cumsum([0] + [x.n for x in graphs])
    assert rel(gpu.bc_shattered_batch(off, g.row_ptr, g.col, resplit=True), oracle.bc(g)) <= TOL64


@pytest.mark.parametrize("path", LARGE_PATHS)
def test_resplit_on_a_large_piece(gpu, path, monkeypatch):
    monkeypatch.setenv("BCS_LARGE_PATH", path)
    g = gg.with_twins_and_pendants(gg.chung_lu(3000, 2.3, 6, 5), 6, 900, 1500, 100)
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, resplit=True), ref) <= TOL64
    assert gpu.last_stats()["n_large_sources"] > 0


# ------------------------- the preprocessing loop repeated to a fixpoint
def blown_up(seed):
    """The blown-up graphs of the CPU fixpoint check (tests/test_readings.py)."""
    rng = np.random.default_rng(100 + seed)
    nb = int(rng.integers(3, 8))
    base = gg.random_tree(nb, seed) if seed % 2 else gg.gnp(nb, 0.5, seed)
    return gg.blow_up(base, seed, max_k=3, p_closed=0.3, n_pend=int(rng.integers(0, 4)))


@pytest.mark.parametrize("unequal", [False, True])
def test_fixpoint_loop_on_blown_up_graphs(gpu, unequal):
    """Split and merge repeated until a round merges nothing: bc equal to the
    oracle's, over graphs needing up to four rounds, with every step subset
    that merges (one round without identical merging)."""
    rounds = []
    for seed in range(24):
        g = blown_up(seed)
        ref = oracle.bc(g)
        for steps in (ALL, oracle.STEP_A | oracle.STEP_I, oracle.STEP_I, oracle.STEP_D | oracle.STEP_A):
            got = gpu.bc_shattered(g.row_ptr, g.col, steps=steps, resplit=True, unequal=unequal)
            assert rel(got, ref) <= TOL64, (seed, steps)
            r = gpu.last_stats()["n_rounds"]
            if steps & oracle.STEP_I:
                rounds.append(r)
            else:
                assert r <= 1  # one split, none when nothing is left after peeling
        got = gpu.bc_shattered(g.row_ptr, g.col, resplit=True, unequal=unequal, delta_fp32=True)
        assert rel(got, ref) <= TOL32
    assert max(rounds) >= 3


def test_fixpoint_loop_on_a_nested_four_cycle(gpu):
    """C4 blown up: the first merge takes each pair of opposite corner groups
    into one vertex, leaving one edge; the first split-and-merge round splits
    it off and merges its closed pair, the second finds nothing to merge."""
    g = gg.blow_up(gg.cycle(4), 3, max_k=3, p_closed=0.0)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col, resplit=True), oracle.bc(g)) <= TOL64
    assert gpu.last_stats()["n_rounds"] == 2


@pytest.mark.parametrize("path", LARGE_PATHS)
def test_fixpoint_loop_larger_graphs_and_batch(gpu, path, monkeypatch):
    """A blown-up random tree with extra edges (thousands of vertices, pieces
    on the large-piece path too) and a batch of blown-up graphs."""
    monkeypatch.setenv("BCS_LARGE_PATH", path)
    base = gg.disjoint_union(gg.random_tree(300, 4), gg.gnp(40, 0.15, 2))
    g = gg.blow_up(base, 9, max_k=4, p_closed=0.3, n_pend=200)
    ref = oracle.bc(g)
    for unequal in (False, True):
        assert rel(gpu.bc_shattered(g.row_ptr, g.col, resplit=True, unequal=unequal), ref) <= TOL64
        assert gpu.last_stats()["n_rounds"] >= 2
    rp, col = on_device(g)
    got = gpu.bc_shattered(rp, col, resplit=True, unequal=True, delta_fp32=True).cpu().numpy()
    assert rel(got, ref) <= TOL32
    graphs = [blown_up(s) for s in range(10)]
    h = gg.disjoint_union(*graphs)
    off = np.cumsum([0] + [x.n for x in graphs])
    assert rel(gpu.bc_shattered_batch(off, h.row_ptr, h.col, resplit=True, unequal=True), oracle.bc(h)) <= TOL64


# --------------------------------------------------------------- errors
def test_malformed_inputs_rejected(gpu):
    bad = {
        "asymmetric": (np.array([0, 1, 1], np.int64), np.array([1], np.int32)),
        "self-loop": (np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32)),
        "duplicate": (np.array([0, 2, 4], np.int64), np.array([1, 1, 0, 0], np.int32)),
        "unsorted": (np.array([0, 2, 3, 4], np.int64), np.array([2, 1, 0, 0], np.int32)),
        "out-of-range": (np.array([0, 1, 2], np.int64), np.array([5, 0], np.int32)),
    }
    for name, (rp, col) in bad.items():
        for fn in (gpu.bc_plain, gpu.bc_shattered):
            with pytest.raises(gpu.BcsError) as e:
                fn(rp, col)
            assert e.value.code == gpu._lib.BCS_EINVAL, name


def test_bounded_wait_times_out_and_context_survives(gpu):
    """The spanning-forest kernel's grid barrier polls a bounded number of
    times; with max_wait < 0 every wait gives up at once, the call returns
    ETIMEOUT and the next call on the same context is correct."""
    g = gg.config(2, scale_pct=2)
    with pytest.raises(gpu.BcsError) as e:
        gpu.bc_shattered(g.row_ptr, g.col, max_wait=-1)
    assert e.value.code == gpu._lib.BCS_ETIMEOUT
    ref = oracle.bc(g)
    assert rel(gpu.bc_shattered(g.row_ptr, g.col), ref) <= TOL64


def test_degenerate_graphs(gpu):
    one = (np.array([0, 0], np.int64), np.zeros(0, np.int32))
    assert np.array_equal(gpu.bc_plain(*one), [0.0])
    assert np.array_equal(gpu.bc_shattered(*one), [0.0])
    empty5 = (np.zeros(6, np.int64), np.zeros(0, np.int32))
    assert np.array_equal(gpu.bc_shattered(*empty5), np.zeros(5))
    k2 = gg.path(2)
    assert np.array_equal(gpu.bc_shattered(k2.row_ptr, k2.col), [0.0, 0.0])
    assert gpu.shatter(k2.row_ptr, k2.col).n_pieces == 0
