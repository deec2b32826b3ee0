"""bcs_bc_plain_noalloc: plain Brandes for callers that cannot let the
library allocate device memory (all of it handed to their own pool, or a
latency-critical loop that must not enter the CUDA allocator).

The entry point keeps its kernels' state in one static device array shared
by every call, so these checks call it twice in a row (and on two different
graphs) and compare each result with bcs_bc_plain, the allocating entry
point, within the FP64 tolerance of the other parity tests; they also hold
it to the CPU oracle directly, in both dependency precisions, and on a graph
of exactly the largest size it accepts (every CTA's slice of the array used
to its end).  This file is collected last so that a failure here stops a -x
run only after every other test has run.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b))) / max(1.0, float(np.max(np.abs(b))))


def dev(g):
    import torch
    return torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda()


def test_noalloc_matches_plain_on_two_calls_in_a_row(gpu):
    g = gg.config(1)  # 2,600 vertices
    rp, col = dev(g)
    ref = gpu.bc_plain(rp, col).cpu().numpy()
    for _ in range(2):
        got = gpu.bc_plain_noalloc(rp, col)
        assert got.is_cuda
        assert rel(got.cpu().numpy(), ref) <= TOL64
    # a different, larger graph next: nothing of the previous call may leak
    g2 = gg.config(2, scale_pct=1)
    assert g2.n <= gpu.NOALLOC_MAX_N
    rp2, col2 = dev(g2)
    ref2 = gpu.bc_plain(rp2, col2).cpu().numpy()
    for _ in range(2):
        assert rel(gpu.bc_plain_noalloc(rp2, col2).cpu().numpy(), ref2) <= TOL64
    # and back to the first graph
    assert rel(gpu.bc_plain_noalloc(rp, col).cpu().numpy(), ref) <= TOL64


def test_noalloc_rejects_what_it_cannot_hold(gpu):
    import torch
    n = gpu.NOALLOC_MAX_N + 1
    big = gg.path(n)
    rp, col = dev(big)
    with pytest.raises(gpu.BcsError) as e:
        gpu.bc_plain_noalloc(rp, col)
    assert e.value.code == gpu._lib.BCS_EINVAL
    assert "at most" in str(e.value)
    with pytest.raises(TypeError):
        gpu.bc_plain_noalloc(big.row_ptr, big.col)  # host arrays: nothing to copy into
    assert torch.cuda.is_available()


def test_noalloc_matches_the_oracle_fp64_and_fp32(gpu):
    g = gg.config(1)
    ref = oracle.bc(g)
    rp, col = dev(g)
    assert rel(gpu.bc_plain_noalloc(rp, col).cpu().numpy(), ref) <= TOL64
    assert rel(gpu.bc_plain_noalloc(rp, col, delta_fp32=True).cpu().numpy(), ref) <= TOL32
    assert rel(gpu.bc_plain_noalloc(rp, col).cpu().numpy(), ref) <= TOL64  # FP64 again after FP32


def test_noalloc_at_the_largest_size(gpu):
    """A 128 x 128 grid: exactly NOALLOC_MAX_N vertices."""
    g = gg.grid(128, 128)
    assert g.n == gpu.NOALLOC_MAX_N
    ref = oracle.bc(g)
    rp, col = dev(g)
    for _ in range(2):
        assert rel(gpu.bc_plain_noalloc(rp, col).cpu().numpy(), ref) <= TOL64
