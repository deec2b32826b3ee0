"""Pins for the Brandes oracle (CPU only).

The oracle (Algorithm 1, FP64 with an extended exponent for sigma) is pinned
to things other than itself:

* brute force: every shortest path of every ordered pair enumerated
  explicitly on graphs of <= 11 vertices, with exact rational arithmetic and
  distances from Floyd-Warshall (Eq. 1 written out);
* closed forms: paths, stars, cycles, complete and complete bipartite graphs,
  and any tree (the paper's binary-tree formula of Section 3.1 generalised to
  branch sizes);
* the invariant sum_v bc[v] = sum over reachable ordered pairs of (d - 1);
* path counts on a grid are binomial coefficients, also far beyond 2^1024;
* networkx's exact betweenness (a library routine, unordered pairs) on
  random graphs.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(float(np.max(np.abs(b))) if b.size else 0.0, 1.0)
    return float(np.max(np.abs(a - b))) / scale if a.size else 0.0


# --------------------------------------------------------------- brute force
def floyd_warshall(g):
    n = g.n
    INF = 10 ** 9
    d = [[INF] * n for _ in range(n)]
    for v in range(n):
        d[v][v] = 0
        for w in g.neighbors(v):
            d[v][int(w)] = 1
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik == INF:
                continue
            di = d[i]
            for j in range(n):
                if dik + dk[j] < di[j]:
                    di[j] = dik + dk[j]
    return d, INF


def brute_force_bc(g):
    """Eq. 1 by enumerating every shortest s-t path (exact fractions)."""
    n = g.n
    d, INF = floyd_warshall(g)
    adj = [[int(w) for w in g.neighbors(v)] for v in range(n)]
    bc = [Fraction(0)] * n
    for s in range(n):
        for t in range(n):
            if s == t or d[s][t] == INF:
                continue
            paths = []

            def walk(x, acc):
                if x == t:
                    paths.append(list(acc))
                    return
                for y in adj[x]:
                    if d[s][y] == d[s][x] + 1 and d[y][t] == d[x][t] - 1:
                        acc.append(y)
                        walk(y, acc)
                        acc.pop()

            walk(s, [s])
            through = [0] * n
            for p in paths:
                for v in p[1:-1]:
                    through[v] += 1
            for v in range(n):
                if through[v]:
                    bc[v] += Fraction(through[v], len(paths))
    return np.array([float(x) for x in bc]), d, INF


def tiny_graphs():
    out = []
    for n in range(1, 12):
        for p in (0.25, 0.5, 0.8):
            out.append(gg.gnp(n, p, seed=1000 * n + int(p * 100)))
    for n in (5, 8, 11):
        out.append(gg.random_tree(n, seed=n))
    out.append(gg.with_twins_and_pendants(gg.cycle(5), seed=3, n_twins=2, n_pend=2, closed_twins=1))
    out.append(gg.disjoint_union(gg.cycle(4), gg.path(3), gg.complete(3)))
    out.append(gg.complete_bipartite(3, 4))
    out.append(gg.grid(3, 3))
    return out


@pytest.mark.parametrize("g", tiny_graphs(), ids=lambda g: g.name)
def test_bc_matches_brute_force(g):
    ref, d, INF = brute_force_bc(g)
    got = oracle.bc(g, threads=2)
    assert rel_err(got, ref) <= 1e-12
    # the sum invariant against Floyd-Warshall distances
    s = sum(d[a][b] - 1 for a in range(g.n) for b in range(g.n) if a != b and d[a][b] < INF)
    assert abs(got.sum() - s) <= 1e-9 * max(1, s)
    tot, pairs = oracle.pair_stats(g, threads=2)
    assert tot == s
    assert pairs == sum(1 for a in range(g.n) for b in range(g.n) if a != b and d[a][b] < INF)


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 3, 7, 50, 201])
def test_path(n):
    got = oracle.bc(gg.path(n))
    ref = np.array([2 * i * (n - 1 - i) for i in range(n)], dtype=np.float64)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [2, 3, 10, 300])
def test_star(n):
    got = oracle.bc(gg.star(n))
    ref = np.zeros(n)
    ref[0] = (n - 1) * (n - 2)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [3, 4, 5, 10, 11, 100, 101])
def test_cycle(n):
    got = oracle.bc(gg.cycle(n))
    val = (n - 1) * (n - 3) / 4 if n % 2 else (n - 2) ** 2 / 4
    assert rel_err(got, np.full(n, val)) <= 1e-13


@pytest.mark.parametrize("n", [1, 2, 5, 30])
def test_complete(n):
    assert np.array_equal(oracle.bc(gg.complete(n)), np.zeros(n))


@pytest.mark.parametrize("a,b", [(1, 5), (2, 3), (3, 7), (10, 4)])
def test_complete_bipartite(a, b):
    got = oracle.bc(gg.complete_bipartite(a, b))
    ref = np.array([b * (b - 1) / a] * a + [a * (a - 1) / b] * b)
    assert rel_err(got, ref) <= 1e-13


def tree_closed_form(g):
    """bc[v] = (n-1)^2 - sum of squared branch sizes at v (every pair of
    vertices in different branches has exactly one path, through v)."""
    n = g.n
    out = np.zeros(n)
    for v in range(n):
        seen = {v}
        sq = 0
        for w0 in g.neighbors(v):
            w0 = int(w0)
            stack, size = [w0], 0
            seen.add(w0)
            while stack:
                x = stack.pop()
                size += 1
                for y in g.neighbors(x):
                    y = int(y)
                    if y not in seen:
                        seen.add(y)
                        stack.append(y)
            sq += size * size
        out[v] = (n - 1) ** 2 - sq
    return out


@pytest.mark.parametrize("n,seed", [(2, 0), (10, 1), (64, 2), (500, 3)])
def test_random_tree(n, seed):
    g = gg.random_tree(n, seed)
    assert np.array_equal(oracle.bc(g), tree_closed_form(g))


def test_binary_tree_formula_of_section_3_1():
    """Complete binary tree with 31 vertices: the paper's formula
    bc[v] = 2 (l_v r_v + (n - l_v - r_v - 1)(l_v + r_v))."""
    n = 31
    g = gg.from_edges(n, [(i, (i - 1) // 2) for i in range(1, n)], "bintree31")

    def size(v):
        return 0 if v >= n else 1 + size(2 * v + 1) + size(2 * v + 2)

    ref = np.array([2 * (size(2 * v + 1) * size(2 * v + 2)
                         + (n - size(2 * v + 1) - size(2 * v + 2) - 1) * (size(2 * v + 1) + size(2 * v + 2)))
                    for v in range(n)], dtype=np.float64)
    assert np.array_equal(oracle.bc(g), ref)


# ------------------------------------------------------------ sigma on grids
def exact_sigma_check(res, rows, cols, cells):
    for (i, j) in cells:
        v = i * cols + j
        exact = math.comb(i + j, i)
        assert res.d[v] == i + j
        m, e = float(res.sig_m[v]), int(res.sig_e[v])
        if exact < 2 ** 53:
            assert math.ldexp(m, e) == float(exact)  # bit-exact
        else:
            got = Fraction(m) * (Fraction(2) ** e)
            assert abs(got / exact - 1) < Fraction(1, 10 ** 12)


def test_grid_sigma_binomial_small():
    rows, cols = 40, 30
    res = oracle.sssp(gg.grid(rows, cols), 0)
    exact_sigma_check(res, rows, cols, [(i, j) for i in range(rows) for j in range(cols)])


def test_grid_sigma_beyond_double_range():
    """C(1398, 699) ~ 2^1392 overflows a double; the extended exponent keeps it."""
    side = 700
    res = oracle.sssp(gg.grid(side, side), 0)
    cells = [(side - 1, side - 1), (side - 1, 0), (350, 349), (600, 650), (699, 500), (10, 20)]
    exact_sigma_check(res, side, side, cells)
    assert int(res.sig_e[side * side - 1]) > 1024


# ------------------------------------------------------------ sources, sssp
def test_sources_partial_sums():
    g = gg.config(1, scale_pct=10)
    full = oracle.bc(g)
    allsrc = oracle.bc_sources(g, np.arange(g.n))
    assert np.array_equal(full, allsrc)
    rng = np.random.default_rng(5)
    a = rng.choice(g.n, size=g.n // 2, replace=False)
    b = np.setdiff1d(np.arange(g.n), a)
    assert rel_err(oracle.bc_sources(g, a) + oracle.bc_sources(g, b), full) <= 1e-13
    # one source = delta_s(v) off the source
    s = int(a[0])
    one = oracle.bc_sources(g, [s])
    res = oracle.sssp(g, s)
    exp = res.delta.copy()
    exp[s] = 0.0
    assert np.array_equal(one, exp)


def test_thread_count_does_not_change_much():
    g = gg.config(1, scale_pct=20)
    assert rel_err(oracle.bc(g, threads=1), oracle.bc(g, threads=5)) <= 1e-14


def test_sum_invariant_config1():
    g = gg.config(1)
    bc = oracle.bc(g)
    tot, _ = oracle.pair_stats(g)
    assert abs(bc.sum() - tot) <= 1e-10 * tot


# ------------------------------------------------------------- networkx
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_networkx_cross_check(seed):
    nx = pytest.importorskip("networkx")
    g = gg.chung_lu(150, 2.5, 4.0, seed)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(map(tuple, g.edges().tolist()))
    ref = nx.betweenness_centrality(G, normalized=False)
    ref = np.array([2.0 * ref[v] for v in range(g.n)])  # networkx counts unordered pairs
    assert rel_err(oracle.bc(g), ref) <= 1e-12


# ------------------------------------------------ a planted mistake is caught
def test_brute_force_catches_a_dropped_term():
    """Drop the '1 +' of Eq. 3 in a copy of the recursion (on the CPU) and
    check that the brute-force pin rejects it: the pins can fail."""
    g = gg.gnp(9, 0.45, seed=4)
    ref, _, _ = brute_force_bc(g)
    n = g.n
    wrong = np.zeros(n)
    for s in range(n):
        res = oracle.sssp(g, s)
        sig = res.sigma_float()
        order = np.argsort(-res.d)
        delta = np.zeros(n)
        for w in order:
            if res.d[w] <= 0:
                continue
            for v in g.neighbors(w):
                if res.d[v] == res.d[w] - 1:
                    delta[v] += sig[v] / sig[w] * delta[w]  # planted: missing "1 +"
        delta[s] = 0
        wrong += delta
    assert rel_err(wrong, ref) > 1e-3
