"""The seeded synthetic workloads are what the measurements quote: their
sizes are fixed by the generators' recipes and seeds (the same on every
machine: integer-only seeded generators), so a change to a generator shows
up here before it silently changes a measured workload."""
import pytest

import graphgen as gg


@pytest.mark.parametrize("i,n,m", [(1, 2600, 4548), (2, 647586, 1697407), (3, 970060, 5024502),
                                   (4, 2258525, 3391149)])
def test_workload_sizes(i, n, m):
    g = gg.config(i)
    assert (g.n, g.m) == (n, m)


def test_secondary_workload_sizes():
    side = gg.with_side_vertices(gg.config(2), 0xB0C00006, 150000, 50000)
    assert (side.n, side.m) == (847586, 2163991)
    uneq = gg.with_twins_and_pendants(gg.chung_lu(25000, 2.1, 12, 0xB0C00007), 0xB0C00007, 7500, 17500)
    assert (uneq.n, uneq.m) == (49787, 245132)


def test_scaled_workload_is_deterministic():
    a = gg.config(2, scale_pct=5)
    b = gg.config(2, scale_pct=5)
    assert a.n == b.n and (a.row_ptr == b.row_ptr).all() and (a.col == b.col).all()
    assert a.n < gg.config(2).n
