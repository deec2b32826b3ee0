"""Pins for the oracle's definitions of the shattered pieces (CPU only).

* blocks against brute force: two edges share a biconnected component iff a
  simple cycle passes through both (enumerated on graphs of <= 9 vertices),
  and against networkx's biconnected components (a library routine);
* the 2-core against networkx's k-core;
* reach: sum_{v in P} reach[v_P] = N_C for every piece (it follows from
  Eq. 4 and the degree-1 update of Section 3.3.1), hand-computed values on
  constructed graphs, and reach = 1 everywhere when nothing is removed;
* identical-vertex classes on graphs whose classes are known by
  construction, including a graph matching the facts printed for Fig. 3.
"""
import os
from collections import defaultdict

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DAI = oracle.STEP_D | oracle.STEP_A | oracle.STEP_I


def block_partition_from_oracle(g, mask=None):
    nb, eb = oracle.blocks(g, None if mask is None else mask.astype(np.uint8))
    src = np.repeat(np.arange(g.n), g.degrees())
    groups = defaultdict(set)
    for k in range(g.nnz):
        if eb[k] >= 0 and src[k] < g.col[k]:
            groups[int(eb[k])].add((int(src[k]), int(g.col[k])))
    return sorted(tuple(sorted(s)) for s in groups.values()), nb


def brute_force_blocks(g):
    """Union the edges of every simple cycle; leftover edges are bridges."""
    n = g.n
    edges = [tuple(e) for e in g.edges().tolist()]
    parent = {e: e for e in edges}

    def find(e):
        while parent[e] != e:
            e = parent[e]
        return e

    adj = [sorted(int(w) for w in g.neighbors(v)) for v in range(n)]
    # enumerate simple cycles by DFS from their smallest vertex
    for s in range(n):
        stack = [(s, [s])]
        while stack:
            v, pth = stack.pop()
            for w in adj[v]:
                if w == s and len(pth) >= 3:
                    cyc = pth + [s]
                    es = [tuple(sorted((cyc[i], cyc[i + 1]))) for i in range(len(cyc) - 1)]
                    r0 = find(es[0])
                    for e in es[1:]:
                        r = find(e)
                        if r != r0:
                            parent[r] = r0
                elif w > s and w not in pth:
                    stack.append((w, pth + [w]))
    groups = defaultdict(set)
    for e in edges:
        groups[find(e)].add(e)
    return sorted(tuple(sorted(s)) for s in groups.values())


def small_graphs():
    out = []
    for n in range(3, 10):
        for p in (0.3, 0.45, 0.7):
            out.append(gg.gnp(n, p, seed=77 * n + int(100 * p)))
    out.append(gg.from_edges(7, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3), (5, 6)], "bowtie-ish"))
    out.append(gg.disjoint_union(gg.cycle(4), gg.star(4)))
    return out


@pytest.mark.parametrize("g", small_graphs(), ids=lambda g: g.name)
def test_blocks_brute_force(g):
    got, nb = block_partition_from_oracle(g)
    assert got == brute_force_blocks(g)
    assert nb == len(got)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_blocks_and_core_networkx(seed):
    nx = pytest.importorskip("networkx")
    g = gg.chung_lu(300, 2.3, 3.0, seed)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(map(tuple, g.edges().tolist()))
    ref = sorted(tuple(sorted(tuple(sorted(e)) for e in b)) for b in nx.biconnected_component_edges(G))
    got, _ = block_partition_from_oracle(g)
    assert got == ref
    core = oracle.two_core(g)
    assert set(np.nonzero(core)[0].tolist()) == set(nx.k_core(G, 2).nodes())


def reach_sums_ok(g, pieces):
    for p in pieces:
        assert sum(p.reach.values()) == p.N, p.vertices


@pytest.mark.parametrize("steps", [1, 2, 3, 5, 6, 7, 0, 4])
def test_reach_sum_invariant(steps):
    g = gg.config(1, scale_pct=25)
    pieces = oracle.shatter(g, steps)
    reach_sums_ok(g, pieces)
    if not steps & oracle.STEP_A and not steps & oracle.STEP_D:
        assert all(r == 1 for p in pieces for r in p.reach.values())


def test_reach_hand_computed():
    """Two triangles {0,1,2} and {4,5,6} joined by the path 2-3-4, a pendant
    path 0-7-8 on vertex 0 and a pendant 9 on vertex 5.  N_C = 10."""
    e = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 6), (6, 4), (0, 7), (7, 8), (5, 9)]
    g = gg.from_edges(10, e)
    pieces = {p.vertices: p for p in oracle.shatter(g, oracle.STEP_D | oracle.STEP_A)}
    # degree-1 removal takes 7, 8, 9; the 2-core is the triangles plus 2-3-4,
    # whose blocks are the two triangles and the bridges {2,3}, {3,4}
    assert set(pieces) == {(0, 1, 2), (4, 5, 6), (2, 3), (3, 4)}
    assert pieces[(0, 1, 2)].reach == {0: 3, 1: 1, 2: 6}
    assert pieces[(4, 5, 6)].reach == {4: 7, 5: 2, 6: 1}
    assert pieces[(2, 3)].reach == {2: 5, 3: 5}
    assert pieces[(3, 4)].reach == {3: 6, 4: 4}
    # degree-1 removal alone: one piece, reach = 1 + size of the hanging trees
    only_d = oracle.shatter(g, oracle.STEP_D)
    assert len(only_d) == 1
    assert only_d[0].reach == {0: 3, 1: 1, 2: 1, 3: 1, 4: 1, 5: 2, 6: 1}
    reach_sums_ok(g, only_d)


def test_trees_leave_nothing_with_degree1_removal():
    g = gg.disjoint_union(gg.random_tree(20, 1), gg.path(2), gg.star(5))
    assert oracle.shatter(g, DAI) == []
    # without degree-1 removal every tree edge is its own block
    pieces = oracle.shatter(g, oracle.STEP_A)
    assert len(pieces) == g.m
    reach_sums_ok(g, pieces)


def classes_of(pieces):
    return sorted(c for p in pieces for c in p.classes)


def test_classes_complete_bipartite_and_complete():
    pieces = oracle.shatter(gg.complete_bipartite(2, 3), DAI)
    assert classes_of(pieces) == [(0, 1), (2, 3, 4)]
    pieces = oracle.shatter(gg.complete(5), DAI)
    assert classes_of(pieces) == [(0, 1, 2, 3, 4)]
    pieces = oracle.shatter(gg.cycle(4), DAI)
    assert classes_of(pieces) == [(0, 2), (1, 3)]
    assert classes_of(oracle.shatter(gg.cycle(5), DAI)) == []


def test_classes_need_equal_reach():
    """C4 with a pendant on vertex 0: 0 and 2 share a neighbourhood but not
    their reach, so only {1, 3} is a class."""
    g = gg.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4)])
    pieces = oracle.shatter(g, DAI)
    assert classes_of(pieces) == [(1, 3)]


def test_classes_of_any_reach():
    """With STEP_U the reach leaves the key: in the C4 with a pendant on 0,
    0 and 2 (same neighbours {1, 3}, reaches 2 and 1) form a class too; on
    graphs where every reach is equal, or with no removal at all, the
    classes are exactly the equal-reach ones; and an equal-reach class is
    always inside a class of any reach."""
    g = gg.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4)])
    assert classes_of(oracle.shatter(g, DAI | oracle.STEP_U)) == [(0, 2), (1, 3)]
    for g in (gg.complete_bipartite(2, 3), gg.complete(5), gg.cycle(4)):
        assert classes_of(oracle.shatter(g, DAI | oracle.STEP_U)) == classes_of(oracle.shatter(g, DAI))
    for seed in range(4):
        g = gg.with_twins_and_pendants(gg.gnp(40, 0.1, seed), seed, 8, 25, 3)
        assert classes_of(oracle.shatter(g, oracle.STEP_I | oracle.STEP_U)) == \
            classes_of(oracle.shatter(g, oracle.STEP_I))
        wide = [set(c) for c in classes_of(oracle.shatter(g, DAI | oracle.STEP_U))]
        for c in classes_of(oracle.shatter(g, DAI)):
            assert any(set(c) <= w for w in wide)


def test_added_side_vertices_have_clique_neighbourhoods():
    """The side-vertex generator's claim: every added vertex's neighbours
    are pairwise adjacent in the final graph."""
    base = gg.gnp(30, 0.15, 4)
    g = gg.with_side_vertices(base, 5, 25, 20)
    assert g.n == base.n + 45
    adj = [set(map(int, g.neighbors(v))) for v in range(g.n)]
    for v in range(base.n, g.n):
        nb = sorted(adj[v])
        assert len(nb) >= 2
        assert all(b in adj[a] for i, a in enumerate(nb) for b in nb[i + 1:])


def test_figure3_identical_vertices_golden():
    """Fig. 3 (Section 3.4): vertices 1 and 8 are identical with neighbours
    {2,4,6,7}; with one of them removed the other is an articulation vertex.
    The figure itself is missing from the text, so the fixture is a graph
    built to match those printed facts."""
    path = os.path.join(GOLDEN, "fig3_identical.txt")
    edges = []
    meta = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                if line.startswith("# expect"):
                    k, v = line[len("# expect "):].split("=")
                    meta[k.strip()] = v.strip()
                continue
            a, b = line.split()
            edges.append((int(a), int(b)))
    n = int(meta["n"])
    g = gg.from_edges(n, edges)
    assert sorted(int(w) for w in g.neighbors(1)) == [2, 4, 6, 7]
    assert sorted(int(w) for w in g.neighbors(8)) == [2, 4, 6, 7]
    pieces = oracle.shatter(g, oracle.STEP_A | oracle.STEP_I)
    assert len(pieces) == 1  # biconnected before merging
    assert (1, 8) in pieces[0].classes
    # remove vertex 8: vertex 1 becomes an articulation vertex
    keep = [v for v in range(n) if v != 8]
    idx = {v: i for i, v in enumerate(keep)}
    g2 = gg.from_edges(n - 1, [(idx[a], idx[b]) for a, b in edges if a != 8 and b != 8])
    cnt, lab = oracle.components(g2)
    mask = np.ones(g2.n, dtype=np.uint8)
    mask[idx[1]] = 0
    cnt_without, _ = oracle.components(g2, mask)
    assert cnt == 1 and cnt_without == 2


def test_shatter_config1_consistency():
    g = gg.config(1)
    pieces = oracle.shatter(g, DAI)
    reach_sums_ok(g, pieces)
    # every 2-core vertex lies in at least one piece; nothing else does
    core = set(np.nonzero(oracle.two_core(g))[0].tolist())
    covered = set(v for p in pieces for v in p.vertices)
    assert covered == core
    for p in pieces:
        for c in p.classes:
            assert len({p.reach[v] for v in c}) == 1
