"""Failure reporting through the C ABI, caused on the host: nothing here
faults, traps or hangs the GPU (needs a CUDA device).

* BCS_TEST_FAIL_ALLOC=k makes every device allocation of a call after its
  first k fail as if the device were out of memory: the call returns
  BCS_ENOMEM, frees what it holds, and the next call succeeds.
* BCS_TEST_SIGMA_CAP=k makes path counts above 2^k count as out of range in
  the whole-GPU Bc-Reach kernel: the call returns BCS_EOVERFLOW, as it would
  if counts left the range the kernels can scale.
* A device-side wait that runs out is covered in test_gpu_parity.py
  (test_bounded_wait_times_out_and_context_survives).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b))) / max(1.0, float(np.max(np.abs(b))))


@pytest.mark.parametrize("budget", [0, 1, 5, 15])
def test_allocation_failure_reports_enomem(gpu, monkeypatch, budget):
    g = gg.config(1)
    monkeypatch.setenv("BCS_TEST_FAIL_ALLOC", str(budget))
    # the plain call makes at least 7 allocations, the shattered one dozens
    for call in ((gpu.bc_shattered, gpu.bc_plain) if budget <= 5 else (gpu.bc_shattered,)):
        with pytest.raises(gpu.BcsError) as e:
            call(g.row_ptr, g.col)
        assert e.value.code == gpu._lib.BCS_ENOMEM
        assert "BCS_TEST_FAIL_ALLOC" in str(e.value)
    monkeypatch.delenv("BCS_TEST_FAIL_ALLOC")
    assert rel(gpu.bc_shattered(g.row_ptr, g.col), oracle.bc(g)) <= TOL64


def layered(k, layers):
    e = []
    for l in range(layers - 1):
        a = np.arange(k) + l * k
        b = np.arange(k) + (l + 1) * k
        e.append(np.stack(np.meshgrid(a, b), -1).reshape(-1, 2))
    return gg.from_edges(k * layers, np.concatenate(e))


def test_path_count_range_reports_eoverflow(gpu, monkeypatch):
    """Layers of 20: the path count to layer l is 20^(l-1), 2^82 at the last
    of 20 layers, past a cap of 2^40."""
    monkeypatch.setenv("BCS_LARGE_PATH", "wide_all")
    g = layered(20, 20)
    src = np.array([0, 5, 199, 399])
    monkeypatch.setenv("BCS_TEST_SIGMA_CAP", "40")
    with pytest.raises(gpu.BcsError) as e:
        gpu.bc_sources(g.row_ptr, g.col, src)
    assert e.value.code == gpu._lib.BCS_EOVERFLOW
    monkeypatch.delenv("BCS_TEST_SIGMA_CAP")
    assert rel(gpu.bc_sources(g.row_ptr, g.col, src), oracle.bc_sources(g, src)) <= TOL64
