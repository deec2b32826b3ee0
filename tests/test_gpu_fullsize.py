"""Above the size the oracle finishes in seconds, at full size: shattered
betweenness (FP64 and FP32 dependencies) against plain Brandes on the whole
graph, both on the GPU, element by element (Theorem 1: the shattered and
compressed computation gives exactly the betweenness of Eq. 1; plain
Brandes itself is held to the oracle on seeded sources of the same graphs in
test_gpu_parity.py).  These are the graphs bench.py times.  Minutes each.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL64 = 1e-12
TOL32 = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b))) / max(1.0, float(np.max(np.abs(b))))


def on_device(g):
    import torch
    return torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()


def test_articulation_full_size_shattered_vs_plain(gpu, monkeypatch):
    """The articulation-heavy workload (n = 647,586): plain Brandes through
    the whole-GPU kernel (its components are at most 88 levels deep from
    their first vertices)."""
    g = gg.config(2)
    rp, col = on_device(g)
    monkeypatch.setenv("BCS_LARGE_PATH", "wide")
    plain = gpu.bc_plain(rp, col).cpu().numpy()
    assert gpu.last_stats()["n_wide_batches"] > 0
    monkeypatch.delenv("BCS_LARGE_PATH")
    assert rel(gpu.bc_shattered(rp, col).cpu().numpy(), plain) <= TOL64
    assert rel(gpu.bc_shattered(rp, col, delta_fp32=True).cpu().numpy(), plain) <= TOL32


def test_twins_full_size_shattered_vs_plain(gpu):
    """The twin-heavy workload (n = 970,060, m = 5,024,502; 22,588
    components), the headline of bench.py: plain Brandes over every
    component against the shattered call in both precisions."""
    g = gg.config(3)
    rp, col = on_device(g)
    plain = gpu.bc_plain(rp, col).cpu().numpy()
    assert gpu.last_stats()["n_wide_batches"] > 0
    b64 = gpu.bc_shattered(rp, col).cpu().numpy()
    assert rel(b64, plain) <= TOL64
    b32 = gpu.bc_shattered(rp, col, delta_fp32=True).cpu().numpy()
    assert rel(b32, plain) <= TOL32


def test_road_full_size_fp32_against_fp64_on_sampled_sources(gpu):
    """The road-like workload (n = 2,258,525; BFS depth in the thousands,
    where an FP32 dependency recurrence has the most levels to drift over):
    plain Brandes partial sums over 512 seeded sources with FP32
    dependencies against the same sums in FP64, within the 1e-5 bar."""
    g = gg.config(4)
    rp, col = on_device(g)
    src = np.random.default_rng(44).choice(g.n, 512, replace=False)
    b64 = gpu.bc_sources(rp, col, src).cpu().numpy()
    b32 = gpu.bc_sources(rp, col, src, delta_fp32=True).cpu().numpy()
    err = rel(b32, b64)
    assert err <= TOL32, err
