"""The C ABI library loads, exports every declared entry point, matches the
ctypes struct layouts and rejects bad arguments on the host (no GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT, cuda_available

HEADER = os.path.join(ROOT, "include", "bcshatter.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bcs_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    import paper_1209_6007_gb300 as bcs
    lib = bcs.load()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", bcs._lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bcs_\w+)", out))
    assert set(names) <= exported
    # nothing else leaks out of the library under the bcs_ prefix
    assert exported <= set(names)


def test_binding_covers_the_header():
    from paper_1209_6007_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_struct_layouts_match_the_header(tmp_path):
    """Compile a probe against the header with gcc and compare sizeof/offsetof."""
    from paper_1209_6007_gb300 import _lib
    src = tmp_path / "probe.c"
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu\\n", sizeof(bcs_csr), sizeof(bcs_opts), sizeof(bcs_stats), sizeof(bcs_components_view));
  printf("%zu %zu %zu\\n", offsetof(bcs_opts, stream), offsetof(bcs_stats, ms_download),
         offsetof(bcs_components_view, bc_corr));
  return 0;
}}
""")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = list(map(int, lines[0].split()))
    offs = list(map(int, lines[1].split()))
    assert sizes == [ctypes.sizeof(_lib.Csr), ctypes.sizeof(_lib.Opts), ctypes.sizeof(_lib.Stats),
                     ctypes.sizeof(_lib.ComponentsView)]
    assert offs == [_lib.Opts.stream.offset, _lib.Stats.ms_download.offset, _lib.ComponentsView.bc_corr.offset]


def test_host_side_argument_checks():
    import paper_1209_6007_gb300 as bcs
    lib = bcs.load()
    assert lib.bcs_bc_plain(None, None, None) == bcs.BCS_EINVAL
    # row_ptr[n] != nnz
    with pytest.raises(bcs.BcsError) as e:
        bcs.bc_plain(np.array([0, 1, 3], np.int64), np.array([1, 0], np.int32))
    assert e.value.code == bcs.BCS_EINVAL
    with pytest.raises(bcs.BcsError) as e:
        bcs.bc_sources(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), [5])
    assert e.value.code == bcs.BCS_EINVAL
    with pytest.raises(bcs.BcsError):
        bcs.bc_shattered(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), steps=8)
    # the empty graph is valid and needs no device
    assert bcs.bc_plain(np.zeros(1, np.int64), np.zeros(0, np.int32)).size == 0
    assert bcs.bc_shattered(np.zeros(1, np.int64), np.zeros(0, np.int32)).size == 0
    c = bcs.shatter(np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert c.n_pieces == 0


def test_step_bits_checked_on_the_host():
    """BCS_STEP_S, BCS_STEP_U and BCS_STEP_L are taken by the shattered calls
    (S with neither U nor L; U and L together), BCS_STEP_O by all but the
    batch call, and unknown bits are rejected before any device work."""
    import paper_1209_6007_gb300 as bcs
    rp, col = np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32)
    pairs = (bcs.STEP_S | bcs.STEP_U, bcs.STEP_S | bcs.STEP_L, bcs.STEP_S | bcs.STEP_U | bcs.STEP_L)
    for steps in (128, 256 | bcs.STEP_S) + tuple(bcs.STEPS_ALL | p for p in pairs):
        with pytest.raises(bcs.BcsError) as e:
            bcs.bc_shattered(rp, col, steps=steps)
        assert e.value.code == bcs.BCS_EINVAL
    for steps in (bcs.STEPS_ALL | bcs.STEP_O,) + tuple(bcs.STEPS_ALL | p for p in pairs):
        with pytest.raises(bcs.BcsError) as e:
            bcs.bc_shattered_batch([0, 2], rp, col, steps=steps)
        assert e.value.code == bcs.BCS_EINVAL
    for steps in (bcs.STEP_U, bcs.STEP_L):  # the pieces API has neither
        with pytest.raises(bcs.BcsError) as e:
            bcs.shatter(rp, col, steps=bcs.STEPS_ALL | steps)
        assert e.value.code == bcs.BCS_EINVAL
    for call in (lambda: bcs.bc_shattered(rp, col, side=True),
                 lambda: bcs.bc_shattered(rp, col, side=True, order=True),
                 lambda: bcs.bc_shattered(rp, col, unequal=True, order=True),
                 lambda: bcs.bc_shattered(rp, col, resplit=True, order=True),
                 lambda: bcs.bc_shattered(rp, col, resplit=True, unequal=True),
                 lambda: bcs.bc_shattered_batch([0, 2], rp, col, resplit=True, unequal=True),
                 lambda: bcs.bc_shattered_batch([0, 2], rp, col, resplit=True),
                 lambda: bcs.bc_shattered_batch([0, 2], rp, col, side=True),
                 lambda: bcs.bc_shattered_batch([0, 2], rp, col, unequal=True)):
        try:
            call()
        except bcs.BcsError as e:  # no device here: anything but a rejected argument
            assert e.code != bcs.BCS_EINVAL


def test_batch_argument_checks():
    import paper_1209_6007_gb300 as bcs
    rp = np.array([0, 1, 2, 2], np.int64)
    col = np.array([1, 0], np.int32)
    for off in ([0, 2], [0, 1, 2], [1, 3], [0, 2, 1, 3]):  # must start at 0, end at n, ascend
        with pytest.raises(bcs.BcsError) as e:
            bcs.bc_shattered_batch(off, rp, col)
        assert e.value.code == bcs.BCS_EINVAL


@pytest.mark.skipif(cuda_available(), reason="checks the no-device error path")
def test_no_device_is_reported():
    import paper_1209_6007_gb300 as bcs
    with pytest.raises(bcs.BcsError) as e:
        bcs.bc_plain(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    assert e.value.code == bcs.BCS_ENODEV
