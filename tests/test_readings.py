"""The readings the device path takes where the paper is silent, checked on
the CPU against the oracle's plain Brandes (Eq. 1).

* side vertices leaving a piece all at once (Section 3.3.2, Algorithm 3 in
  set form);
* identical classes whose members differ in reach (Section 3.3.3 leaves
  reach and ident together out);
* a merged vertex that is a cut vertex (Fig. 3), split with fractional
  copies;
* merging again after that split (classes whose members are themselves
  merged vertices or copies).

Each test writes the reading out with a small weighted Bc-Reach of its own
(Algorithm 2 with reach and ident: a predecessor v counts ident[v] times in
sigma, delta starts at reach - 1, the source weighs reach[s] * ident[s]),
independent of the device path; the GPU tests compare the device path with
the oracle directly.
"""
import itertools
import random
from collections import deque

import numpy as np
import pytest

import graphgen as gg
import oracle


def weighted_bcreach(adj, nodes, reach, ident, sources):
    """bc'[w] = sum over the sources s of reach[s] ident[s] delta_s(w)."""
    bc = {v: 0.0 for v in nodes}
    for s in sources:
        d = {s: 0}
        sig = {v: 0.0 for v in nodes}
        sig[s] = 1.0
        order, q = [], deque([s])
        while q:
            v = q.popleft()
            order.append(v)
            for w in adj[v]:
                if w not in d:
                    d[w] = d[v] + 1
                    q.append(w)
                if d[w] == d[v] + 1:
                    sig[w] += sig[v] * (1 if v == s else ident[v])
        delta = {v: reach[v] - 1.0 for v in order}
        for w in reversed(order):
            for v in adj[w]:
                if d.get(v, -2) == d[w] - 1:
                    delta[v] += sig[v] / sig[w] * ident[w] * (1.0 + delta[w])
            if w != s:
                bc[w] += reach[s] * ident[s] * delta[w]
    return bc


def rel(got, ref):
    ref = np.asarray(ref, float)
    return float(np.max(np.abs(np.asarray(got, float) - ref))) / max(1.0, float(np.max(np.abs(ref))))


def is_side(adj, v):
    nb = sorted(adj[v])
    return len(nb) >= 1 and all(b in adj[a] for a, b in itertools.combinations(nb, 2))


def side_set_bcreach(adj, nodes, reach, ident):
    """Every side vertex u: a search on the full piece with the targets
    outside S weighted 2 reach; the others: a search on the piece without S;
    then reach[v] * SW off every v outside S and (reach[u] - 1) * NW onto
    every u in S."""
    S = {v for v in nodes if is_side(adj, v)}
    reach2 = {v: reach[v] if v in S else 2 * reach[v] for v in nodes}
    bc = weighted_bcreach(adj, nodes, reach2, ident, sorted(S))
    rest = [v for v in nodes if v not in S]
    adj_r = {v: [w for w in adj[v] if w not in S] for v in rest}
    for v, x in weighted_bcreach(adj_r, rest, reach, ident, rest).items():
        bc[v] += x
    SW = sum(reach[u] * ident[u] for u in S)
    NW = sum(reach[v] * ident[v] for v in rest)
    for v in nodes:
        bc[v] += (reach[v] - 1) * NW if v in S else -reach[v] * SW
    return bc, len(S)


def random_side_graph(rng, n):
    adj = {v: set() for v in range(n)}
    for v in range(1, n):
        u = rng.randrange(v)
        adj[u].add(v)
        adj[v].add(u)
    for _ in range(rng.randint(0, n)):
        a, b = rng.sample(range(n), 2)
        adj[a].add(b)
        adj[b].add(a)
    for v in range(n):  # close some triangles: more side vertices
        nb = list(adj[v])
        if len(nb) >= 2 and rng.random() < 0.5:
            a, b = rng.sample(nb, 2)
            adj[a].add(b)
            adj[b].add(a)
    return adj


def test_side_vertices_as_a_set_keep_weighted_bc():
    """Any reach and ident: the set form equals Bc-Reach with every vertex a
    source on the whole piece."""
    rng = random.Random(7)
    found = 0
    for _ in range(150):
        n = rng.randint(2, 12)
        adj = random_side_graph(rng, n)
        reach = {v: float(rng.choice([1, 1, 2, 5])) for v in adj}
        ident = {v: rng.choice([1, 1, 2, 3]) for v in adj}
        full = weighted_bcreach(adj, list(adj), reach, ident, list(adj))
        got, ns = side_set_bcreach(adj, list(adj), reach, ident)
        found += ns
        assert rel([got[v] for v in adj], [full[v] for v in adj]) <= 1e-12
    assert found > 100


def test_side_vertices_as_a_set_match_the_oracle():
    for seed in range(6):
        g = gg.with_side_vertices(gg.gnp(25, 0.15, seed), seed, 15, 10)
        if not all(len(g.neighbors(v)) for v in range(g.n)):
            continue
        adj = {v: set(map(int, g.neighbors(v))) for v in range(g.n)}
        ones = {v: 1.0 for v in adj}
        got, ns = side_set_bcreach(adj, list(adj), ones, {v: 1 for v in adj})
        assert ns > 0
        assert rel([got[v] for v in range(g.n)], oracle.bc(g)) <= 1e-12


def twins_with_pendants(seed):
    """A 2-connected base (cycle plus chords), k open twins joined to the
    same base vertices, and pendant paths on some twins (so the twins'
    reaches differ)."""
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(5, 10))
    e = [(i, (i + 1) % nb) for i in range(nb)]
    e += [(int(a), int(b)) for a, b in rng.integers(0, nb, (3, 2)) if a != b]
    S = sorted(set(int(x) for x in rng.choice(nb, 3, replace=False)))
    k = int(rng.integers(2, 5))
    twins = list(range(nb, nb + k))
    e += [(t, x) for t in twins for x in S]
    n = nb + k
    tails = {}
    for t in twins:
        length = int(rng.integers(0, 4))
        prev = t
        for _ in range(length):
            e.append((prev, n))
            prev = n
            n += 1
        tails[t] = length
    e = sorted({(min(a, b), max(a, b)) for a, b in e})
    return gg.from_edges(n, e), nb, twins, tails, S


def test_unequal_reach_classes_match_the_oracle():
    """Twins of reaches 1 + (pendant path length) merged into one vertex:
    dependency start R/K - 1, source weight R, and on each copy
    (r - 1)(R - r) + (r - R/K)(N - R); each common neighbour gets
    (R^2 - sum r^2) / K_N.  Pendant paths are removed by the degree-1 terms
    of Section 3.3.1 (order does not matter)."""
    for seed in range(12):
        g, nb, twins, tails, S = twins_with_pendants(seed)
        N = g.n
        ref = oracle.bc(g)
        bc = np.zeros(g.n)
        # degree-1 removal along each pendant path, leaf first
        r = {t: 1 + tails[t] for t in twins}
        adj = {v: set(map(int, g.neighbors(v))) for v in range(g.n)}
        for t in twins:
            path = [t]
            while True:
                nxt = [w for w in adj[path[-1]] if w >= nb + len(twins) and w not in path]
                if not nxt:
                    break
                path.append(nxt[0])
            reach_here = 1
            for i in range(len(path) - 1, 0, -1):  # remove path[i] into path[i-1]
                u, v = path[i], path[i - 1]
                bc[u] += (reach_here - 1) * (N - reach_here)
                bc[v] += reach_here * (N - reach_here - 1)
                reach_here += 1
        # the 2-core: base + twins, one piece (biconnected); merge the twins
        core = list(range(nb)) + [twins[0]]
        K = len(twins)
        R = sum(r[t] for t in twins)
        Q = sum(r[t] ** 2 for t in twins)
        w = twins[0]
        cadj = {v: set(x for x in adj[v] if x < nb or x == w) for v in core}
        reach = {v: 1.0 for v in core}
        reach[w] = R / K
        ident = {v: 1 for v in core}
        ident[w] = K
        bcp = weighted_bcreach(cadj, core, reach, ident, core)
        for x in S:
            bcp[x] += (R * R - Q) / len(S)
        for v in range(nb):
            bc[v] += bcp[v]
        for t in twins:
            bc[t] += bcp[w] + (r[t] - 1) * (R - r[t]) + (r[t] - R / K) * (N - R)
        assert rel(bc, ref) <= 1e-12, seed


def test_merged_cut_vertex_split_with_fractional_copies():
    """Two parts joined only through k open twins: merged, the twins are
    one cut vertex w of ident k; split there, w's copy in each block has
    reach 1 + (weight beyond it) / k and keeps ident k."""
    import networkx as nx
    rng = np.random.default_rng(11)
    for _ in range(40):
        na, nbb = int(rng.integers(3, 8)), int(rng.integers(3, 8))
        G = nx.Graph()
        for off, m in ((0, na), (na, nbb)):
            G.add_edges_from((off + i, off + (i + 1) % m) for i in range(m))
            for a, b in rng.integers(0, m, (2, 2)):
                if a != b:
                    G.add_edge(off + int(a), off + int(b))
        S = [int(x) for x in rng.choice(na, 2, replace=False)] + [na + int(x) for x in rng.choice(nbb, 2, replace=False)]
        k = int(rng.integers(2, 5))
        T = list(range(na + nbb, na + nbb + k))
        G.add_edges_from((t, x) for t in T for x in S)
        n = G.number_of_nodes()
        g = gg.from_edges(n, sorted((min(a, b), max(a, b)) for a, b in G.edges()))
        ref = oracle.bc(g)
        w = T[0]
        H = G.copy()
        H.remove_nodes_from(T[1:])
        ident = {v: 1 for v in H}
        ident[w] = k
        W = {v: float(ident[v]) for v in H}
        extra = np.zeros(n)
        for x in S:
            extra[x] += k * (k - 1) / len(S)  # the type-I class terms, reach 1
        cuts = set(nx.articulation_points(H))
        assert w in cuts
        bcp = {v: 0.0 for v in H}
        for blk in map(set, nx.biconnected_components(H)):
            reach = {}
            for v in blk:
                if v in cuts:
                    Hv = H.copy()
                    Hv.remove_node(v)
                    other = sum(W[x] for c in nx.connected_components(Hv) if not (c & blk) for x in c)
                    reach[v] = 1.0 + other / ident[v]
                else:
                    reach[v] = 1.0
            adj = {v: [x for x in H[v] if x in blk] for v in blk}
            for v, x in weighted_bcreach(adj, blk, reach, ident, blk).items():
                bcp[v] += x
        got = np.array([(bcp[w] if v in T else bcp[v]) + extra[v] for v in range(n)])
        assert rel(got, ref) <= 1e-12


def test_merging_again_after_the_split():
    """After the split at the merged twins w, a vertex x whose neighbours are
    exactly w's in one block becomes identical to w's copy there.  Merged
    into one vertex U (K = 1 + k members; sub-units {x} and w's k members,
    weights T_x and T_w, T = T_x + T_w): dependency start T/K - 1, and on
    each member m of sub-unit i, (t_m - T/K)(N - T) + (t_m - 1)(T - T_i);
    each common neighbour gets (T^2 - T_x^2 - T_w^2) / K_N.  Pairs inside a
    sub-unit were counted when it formed, hence T - T_i."""
    import networkx as nx
    rng = np.random.default_rng(5)
    for _ in range(30):
        na, nb = int(rng.integers(3, 8)), int(rng.integers(3, 8))
        G = nx.Graph()
        for off, m in ((0, na), (na, nb)):
            G.add_edges_from((off + i, off + (i + 1) % m) for i in range(m))
            for a, b in rng.integers(0, m, (2, 2)):
                if a != b:
                    G.add_edge(off + int(a), off + int(b))
        SA = [int(v) for v in rng.choice(na, 2, replace=False)]
        SB = [na + int(v) for v in rng.choice(nb, 2, replace=False)]
        k = int(rng.integers(2, 5))
        twins = list(range(na + nb, na + nb + k))
        G.add_edges_from((t, s) for t in twins for s in SA + SB)
        x = na + nb + k
        G.add_edges_from((x, s) for s in SA)
        n = N = G.number_of_nodes()
        g = gg.from_edges(n, sorted((min(a, b), max(a, b)) for a, b in G.edges()))
        ref = oracle.bc(g)
        w = twins[0]
        bc = np.zeros(n)
        for s in SA + SB:  # the twins' type-I class terms, reach 1
            bc[s] += k * (k - 1) / (len(SA) + len(SB))
        H = G.copy()
        H.remove_nodes_from(twins[1:])
        ident = {v: 1 for v in H}
        ident[w] = k
        cuts = set(nx.articulation_points(H))
        merged = 0
        for blk in map(set, nx.biconnected_components(H)):
            t = {}
            for v in blk:
                other = 0.0
                if v in cuts:
                    Hv = H.copy()
                    Hv.remove_node(v)
                    other = sum(ident[y] for c in nx.connected_components(Hv) if not (c & blk) for y in c)
                t[v] = 1.0 + other / ident[v]
            adj = {v: set(y for y in H[v] if y in blk) for v in blk}
            if x in blk and w in blk and adj[x] == adj[w]:
                merged += 1
                K, Tx, Tw = 1 + k, t[x], k * t[w]
                T = Tx + Tw
                nodes = [v for v in blk if v != x]
                reach = {v: t[v] for v in nodes}
                reach[w] = T / K
                idn = {v: ident[v] for v in nodes}
                idn[w] = K
                part = weighted_bcreach({v: adj[v] - {x} for v in nodes}, nodes, reach, idn, nodes)
                for v in nodes:
                    if v != w:
                        bc[v] += part[v]
                bc[x] += part[w] + (t[x] - T / K) * (N - T) + (t[x] - 1) * (T - Tx)
                for tw in twins:
                    bc[tw] += part[w] + (t[w] - T / K) * (N - T) + (t[w] - 1) * (T - Tw)
                for s in adj[x]:
                    bc[s] += (T * T - Tx * Tx - Tw * Tw) / len(adj[x])
            else:
                part = weighted_bcreach(adj, blk, t, ident, blk)
                for v in blk:
                    for member in (twins if v == w else [v]):
                        bc[member] += part[v]
        assert merged == 1
        assert rel(bc, ref) <= 1e-12


def fixpoint_bc(g):
    """The preprocessing loop repeated to a fixpoint (Section 3.4, Fig. 3),
    written out on the CPU.  Every connected component starts as one piece
    whose vertices are units: k original members of weight t each (T = k t;
    at first k = t = 1).  A round splits every piece at its cut vertices (a
    copy weighs T plus all the weight beyond it away from its block, shared
    by its k members) and merges the identical units of every block.  A class
    of sub-units x (K = sum k_x, T = sum T_x) becomes one unit of K members of
    weight T / K; each member of x gets (t_x - T/K)(N - T) + (t_x - 1)(T - T_x)
    (pairs inside a sub-unit were counted when it formed); in a type-I class
    (open neighbourhoods equal) every member of a neighbour gets
    (T^2 - sum T_x^2) / K_N, K_N the members of the class's neighbours.
    Rounds repeat until one merges nothing; weighted Bc-Reach on the final
    pieces completes bc.  Returns (bc, rounds)."""
    import networkx as nx
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(map(tuple, g.edges()))
    bc = np.zeros(g.n)
    members, weight = {}, {}  # unit -> its original vertices; unit -> t

    def unit(mem, t):
        u = len(members)
        members[u], weight[u] = mem, t
        return u

    pieces = []
    for comp in nx.connected_components(G):
        ids = {v: unit([v], 1.0) for v in comp}
        pieces.append((nx.relabel_nodes(G.subgraph(comp), ids), len(comp)))
    rounds = 0
    while True:
        rounds += 1
        blocks = []
        for H, N in pieces:
            if H.number_of_nodes() < 2:
                continue
            W = {v: len(members[v]) * weight[v] for v in H}
            cuts = set(nx.articulation_points(H))
            for blk in map(set, nx.biconnected_components(H)):
                copy = {}
                for v in blk:
                    beyond = 0.0
                    if v in cuts:
                        Hv = H.copy()
                        Hv.remove_node(v)
                        beyond = sum(W[y] for c in nx.connected_components(Hv) if not (c & blk) for y in c)
                    copy[v] = unit(members[v], (W[v] + beyond) / len(members[v]))
                blocks.append((nx.relabel_nodes(H.subgraph(blk), copy), N))
        merged_any = False
        pieces = []
        for B, N in blocks:
            by_open, by_closed = {}, {}
            for v in B:
                by_open.setdefault(frozenset(B[v]), []).append(v)
            classes = [(c, True) for c in by_open.values() if len(c) > 1]
            taken = {v for c, _ in classes for v in c}
            for v in B:
                if v not in taken:
                    by_closed.setdefault(frozenset(B[v]) | {v}, []).append(v)
            classes += [(c, False) for c in by_closed.values() if len(c) > 1]
            rename = {}
            for cls, open_twins in classes:
                merged_any = True
                K = sum(len(members[x]) for x in cls)
                Tx = {x: len(members[x]) * weight[x] for x in cls}
                T = sum(Tx.values())
                for x in cls:
                    amt = (weight[x] - T / K) * (N - T) + (weight[x] - 1.0) * (T - Tx[x])
                    for m in members[x]:
                        bc[m] += amt
                if open_twins:
                    nbrs = B[cls[0]]
                    KN = sum(len(members[y]) for y in nbrs)
                    amt = (T * T - sum(t * t for t in Tx.values())) / KN
                    for y in nbrs:
                        for m in members[y]:
                            bc[m] += amt
                u = unit([m for x in cls for m in members[x]], T / K)
                for x in cls:
                    rename[x] = u
            if rename:
                Bm = nx.Graph()
                Bm.add_nodes_from({rename.get(v, v) for v in B})
                Bm.add_edges_from((rename.get(a, a), rename.get(b, b)) for a, b in B.edges()
                                  if rename.get(a, a) != rename.get(b, b))
                B = Bm
            pieces.append((B, N))
        if not merged_any:
            break
    for H, N in pieces:
        nodes = list(H)
        reach = {v: weight[v] for v in nodes}
        ident = {v: len(members[v]) for v in nodes}
        part = weighted_bcreach({v: set(H[v]) for v in nodes}, nodes, reach, ident, nodes)
        for v in nodes:
            for m in members[v]:
                bc[m] += part[v]
    return bc, rounds


def test_preprocessing_loop_to_a_fixpoint_matches_the_oracle():
    """Blown-up graphs (every vertex of a small base replaced by open or
    closed twins, pendants added): merged groups become cut vertices, their
    copies become twins of other groups, and so on, for several rounds."""
    rounds_seen = []
    for seed in range(40):
        rng = np.random.default_rng(100 + seed)
        nb = int(rng.integers(3, 8))
        base = gg.random_tree(nb, seed) if seed % 2 else gg.gnp(nb, 0.5, seed)
        g = gg.blow_up(base, seed, max_k=3, p_closed=0.3, n_pend=int(rng.integers(0, 4)))
        got, rounds = fixpoint_bc(g)
        rounds_seen.append(rounds)
        assert rel(got, oracle.bc(g)) <= 1e-12, (seed, rounds)
    assert max(rounds_seen) >= 3


def test_fixpoint_loop_on_a_nested_four_cycle():
    """C4 with every vertex blown up: the opposite corners are open twins;
    merged, the other two corners become twins of each other, then the
    last edge is a closed pair (three rounds, one vertex left)."""
    g = gg.blow_up(gg.cycle(4), 3, max_k=3, p_closed=0.0)
    got, rounds = fixpoint_bc(g)
    assert rounds >= 3
    assert rel(got, oracle.bc(g)) <= 1e-12
