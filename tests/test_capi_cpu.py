"""Host-side checks of the C-ABI library (no GPU): it builds for sm_103a, loads,
exports every entry point include/ms.h declares, and rejects invalid arguments
before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2503_04914_gb300 import build as B
from paper_2503_04914_gb300 import ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ms.load()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ms.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ms_[a-z_0-9]+)\s*\(", txt)))


def test_header_matches_binding():
    assert header_functions() == sorted(ms.EXPORTED)


def test_library_exports_every_header_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in header_functions():
        assert name in syms, name
        assert hasattr(lib, name)


def test_library_is_sm103a_only():
    out = subprocess.run(["cuobjdump", "--list-elf", B.LIB], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_struct_sizes_match_header(lib):
    # ms_default_opts writes exactly sizeof(ms_opts); a guard word after it must survive
    class Guarded(C.Structure):
        _fields_ = [("o", ms.ms_opts), ("guard", C.c_uint64)]
    g = Guarded()
    g.guard = 0xDEADBEEFCAFEF00D
    lib.ms_default_opts(C.byref(g.o))
    assert g.guard == 0xDEADBEEFCAFEF00D
    assert g.o.wendland_d == 3 and g.o.wendland_k == 1 and g.o.nu == 4.0


@pytest.mark.parametrize("d,L,n,h,over,code", [
    (0, 1, [4], [0.1], {}, ms.MS_ERR_ARG),
    (4, 1, [4], [0.1], {}, ms.MS_ERR_ARG),
    (2, 0, [4], [0.1], {}, ms.MS_ERR_ARG),
    (2, 1, [0], [0.1], {}, ms.MS_ERR_ARG),
    (2, 1, [4], [-1.0], {}, ms.MS_ERR_ARG),
    (2, 1, [4], [0.1], {"nu": 0.0}, ms.MS_ERR_ARG),
    (2, 1, [4], [0.1], {"wendland_k": 7}, ms.MS_ERR_ARG),
    (3, 1, [4], [0.1], {"wendland_d": 2}, ms.MS_ERR_ARG),
    (2, 1, [4], [0.1], {"threads_per_row": 3}, ms.MS_ERR_ARG),
    (2, 1, [4], [0.1], {"autotune": 2}, ms.MS_ERR_ARG),
    (2, 1, [4], [0.1], {"lower_op": 2}, ms.MS_ERR_ARG),
    # the matrix-free lower blocks take double-float offsets that only MIXED builds keep
    (2, 1, [4], [0.1], {"lower_op": ms.MS_OP_MATRIX_FREE, "precision": ms.MS_PREC_FP64}, ms.MS_ERR_ARG),
])
def test_invalid_arguments_rejected_on_host(lib, d, L, n, h, over, code):
    opts = ms.ms_default_opts(**over)
    pts = np.zeros((max(1, sum(n)), max(1, d)))
    with pytest.raises(ms.MsError) as e:
        ms.ms_build_hierarchy(d, np.array(n[:max(L, 0)] if L > 0 else [], dtype=np.int64) if L > 0 else np.array([], dtype=np.int64),
                              pts, np.array(h), opts)
    assert e.value.status == code
    assert ms.ms_last_error() != ""


def test_nonfinite_points_rejected_on_host(lib):
    pts = np.array([[0.0, 0.0], [np.nan, 0.5]])
    with pytest.raises(ms.MsError) as e:
        ms.ms_build_hierarchy(2, np.array([2]), pts, np.array([0.5]), ms.ms_default_opts())
    assert e.value.status == ms.MS_ERR_NUMERIC


def test_fit_batch_rejects_bad_arguments_on_host(lib):
    """Argument checks of the batched fit run before any CUDA call."""
    L = ms.load()
    st = (ms.ms_fit_stats * 1)()
    assert L.ms_fit_batch(None, 1, None, 1e-10, None, st) == ms.MS_ERR_ARG
    assert L.ms_fit_batch_dev(None, 0, None, 1e-10, None, st, None) == ms.MS_ERR_ARG
    hs = (C.c_void_p * 1)(None)
    fp = (C.c_void_p * 1)(None)
    assert L.ms_fit_batch_dev(hs, 1, fp, 1e-10, fp, st, None) == ms.MS_ERR_ARG
    assert "hierarchy 0" in ms.ms_last_error()


def test_peak_probe_rejects_unknown_kinds(lib):
    for kind in (-1, 3):
        with pytest.raises(ms.MsError) as e:
            ms.ms_peak_probe(kind)
        assert e.value.status == ms.MS_ERR_ARG


def test_wait_selftest_rejects_bad_arguments_on_host(lib):
    for t in (0.0, -1.0, 10.5, float("nan")):
        with pytest.raises(ms.MsError) as e:
            ms.ms_wait_selftest(t)
        assert e.value.status == ms.MS_ERR_ARG
    rc = ms.load().ms_wait_selftest(0.1, 0, None, None)
    assert rc == ms.MS_ERR_ARG
