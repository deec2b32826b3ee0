"""bench.py's roofline arithmetic on CPU, from fixed call statistics: the
HBM figure of a call whose Bc-Reach time is mostly the whole-GPU kernel
(algorithmic bytes per (source, CSR entry) x pairs / kernel time, traffic
only from a profile record of the same kernel sources), and the issue-rate
figure of a call that is all shared-memory pieces (warp instructions per
launch from the profile record / kernel time against 152 x 4 x clock)."""
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def stats(**kw):
    st = {"dag_edges": 0.0, "work_sources_entries": 0.0, "work_sources_vertices": 0.0, "ms_bcreach_large": 0.0,
          "ms_bcreach_small": 0.0, "n_wide_batches": 0, "n_large_sources": 0}
    st.update(kw)
    return st


def test_hbm_figure_of_the_whole_gpu_kernel(monkeypatch):
    # 10^9 (source, entry) pairs, a quarter of them DAG edges, 10^8 (source, vertex) pairs, 64-source batches
    st = stats(dag_edges=2.5e8, work_sources_entries=1e9, work_sources_vertices=1e8, ms_bcreach_large=100.0,
               n_wide_batches=10, n_large_sources=640)
    monkeypatch.setattr(bench, "measured_traffic", lambda kind: None)
    r = bench.roofline(st, {"sm_mhz": 2070.0}, {"hbm_gbs": 6658.0}, 152)
    by = 1e9 * (8.0 / 64 + 2.0 / 8 + 0.25 * 28.0) + 1e8 * 32.0
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(by / 0.1 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6658.0)
    assert r["traffic"] is None  # no profile record of these kernel sources
    monkeypatch.setattr(bench, "measured_traffic", lambda kind: {"dram_bytes_per_batch": 3.0e9})
    assert bench.roofline(st, {"sm_mhz": 2070.0}, {"hbm_gbs": 6658.0}, 152)["traffic"] == pytest.approx(3.0e10)


def test_issue_rate_figure_of_the_shared_memory_kernel(monkeypatch):
    st = stats(dag_edges=2.0e8, work_sources_entries=1e9, work_sources_vertices=1e8, ms_bcreach_small=5.0)
    rec = {"warp_inst_per_launch": 4.0e9, "thread_inst_per_launch": 6.4e10, "dram_bytes_per_launch": 2.6e7}
    monkeypatch.setattr(bench, "measured_traffic", lambda kind: rec)
    r = bench.roofline(st, {"sm_mhz": 2000.0}, {"hbm_gbs": 6658.0}, 152)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 4 * 2000e6 / 1e9)  # G warp instructions per second
    assert r["achieved"] == pytest.approx(4.0e9 / 5e-3 / 1e9)
    assert r["lane_efficiency"] == pytest.approx(0.5)
    assert r["traffic"] == pytest.approx(2.6e7)
    assert r["fp64"]["achieved"] == pytest.approx((2 * 2.0e8 + 9 * 1e8) / 5e-3 / 1e12)
    # without the record: the FP64 figure alone
    monkeypatch.setattr(bench, "measured_traffic", lambda kind: None)
    r = bench.roofline(st, {"sm_mhz": 2000.0}, {}, 152)
    assert r["unit"] == "TFLOP/s" and r["traffic"] is None
