"""The allocation-free fit (ms_fit_static_dev) against the regular device fit (ms_fit_dev).

Some callers cannot allocate device memory when they fit: their device memory
is already reserved by another allocator, or their loop must not call the
allocator.  ms_fit_static_dev serves them from a fixed device array inside the
library.  These tests call it through the C ABI, twice in a row on one handle,
and check that it returns the same coefficients as ms_fit_dev within the
parity tolerances of the other GPU tests (1e-10 FP64, 1e-8 mixed).  They also
check that hierarchies larger than the array are rejected.  This file is
collected last so that, if it fails, a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2503_04914_gb300 import build as B
from paper_2503_04914_gb300 import inputs, ms

pytestmark = pytest.mark.gpu


def _workload(sizes=(37, 150, 601, 2500, 9001), seed=41):
    allp = inputs.scrambled_halton(max(sizes), 2, seed)
    levels = [np.ascontiguousarray(allp[:n]) for n in sizes]
    h = np.array([n ** -0.5 for n in sizes])
    g = inputs.GaussianMixture(8, 2, seed + 1, sine=True)
    return inputs.Workload("static", 2, levels, h, 4.0, 2, 1, g(np.concatenate(levels)), g)


def _static_fit(lib, H, f, out, rel_tol):
    import torch
    st = ms.ms_fit_stats()
    rc = lib.ms_fit_static_dev(C.c_void_p(H.handle), C.c_void_p(f.data_ptr()), C.c_double(rel_tol),
                               C.c_void_p(out.data_ptr()), C.byref(st),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, st


@pytest.mark.parametrize("prec,tol", [(ms.MS_PREC_FP64, 1e-10), (ms.MS_PREC_MIXED, 1e-8)])
def test_static_fit_matches_fit_dev_on_two_calls(prec, tol):
    import torch
    assert torch.cuda.is_available()
    B.build()
    lib = ms.load()
    w = _workload()
    H = ms.Hierarchy.from_workload(w, device=True, precision=prec)
    g2 = inputs.GaussianMixture(5, 2, 1234)
    rhs = [w.f, g2(w.points)]
    for call, fh in enumerate(rhs):
        f = torch.from_numpy(np.ascontiguousarray(fh)).cuda()
        ref, st_ref = H.fit(f, rel_tol=1e-12)
        out = torch.full_like(f, float("nan"))
        rc, st = _static_fit(lib, H, f, out, 1e-12)
        assert rc == ms.MS_OK, (call, ms.ms_last_error())
        assert ms.ms_last_error() == ""
        torch.cuda.synchronize()
        a, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r), call
        assert max(st.rel_residual[:w.L]) <= 1e-12
        # the statistics the kernel records come back as ms_fit_dev's do
        assert st.fp64_fallbacks == st_ref["fp64_fallbacks"]
        assert list(st.cg_iterations[:w.L]) == st_ref["cg_iterations"]
        assert sum(st.phase_ms[:7]) > 0.0
    H.close()


@pytest.mark.parametrize("prec,op,tol", [(ms.MS_PREC_FP64, ms.MS_OP_CSR, 1e-10),
                                         (ms.MS_PREC_MIXED, ms.MS_OP_CSR, 1e-8),
                                         (ms.MS_PREC_MIXED, ms.MS_OP_MATRIX_FREE, 1e-8)])
def test_static_fit_first_on_a_fresh_handle(prec, op, tol):
    """The intended use: a handle that has never had a work space fits without allocating.
    Its coefficients match ms_fit_dev on a second, separately built handle, on two calls."""
    import torch
    B.build()
    lib = ms.load()
    w = _workload(seed=77)
    Hs = ms.Hierarchy.from_workload(w, device=True, precision=prec, op=op)
    Hd = ms.Hierarchy.from_workload(w, device=True, precision=prec, op=op)
    for call, fh in enumerate([w.f, inputs.GaussianMixture(6, 2, 99)(w.points)]):
        f = torch.from_numpy(np.ascontiguousarray(fh)).cuda()
        out = torch.full_like(f, float("nan"))
        rc, st = _static_fit(lib, Hs, f, out, 1e-12)
        assert rc == ms.MS_OK, (call, ms.ms_last_error())
        ref, _ = Hd.fit(f, rel_tol=1e-12)
        torch.cuda.synchronize()
        a, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r), call
        assert max(st.rel_residual[:w.L]) <= 1e-12
    Hs.close()
    Hd.close()


def test_static_fit_reports_non_finite_f():
    import torch
    B.build()
    lib = ms.load()
    w = _workload(seed=5)
    H = ms.Hierarchy.from_workload(w, device=True)
    fh = np.array(w.f)
    fh[5] = np.nan
    f = torch.from_numpy(fh).cuda()
    out = torch.empty_like(f)
    rc, st = _static_fit(lib, H, f, out, 1e-10)
    assert rc == ms.MS_ERR_NUMERIC
    assert st.device_status == ms.MS_ERR_NUMERIC
    # the array is usable again right after the failed call
    f2 = torch.from_numpy(np.ascontiguousarray(w.f)).cuda()
    rc, st = _static_fit(lib, H, f2, out, 1e-10)
    assert rc == ms.MS_OK and ms.ms_last_error() == ""
    H.close()


def test_static_fit_rejects_hierarchies_above_its_limit():
    import torch
    B.build()
    lib = ms.load()
    w = _workload(sizes=(64, 256, 1024, 4096, 16384, 65536), seed=3)  # 87,360 points > 65,536
    H = ms.Hierarchy.from_workload(w, device=True)
    f = torch.from_numpy(w.f).cuda()
    out = torch.empty_like(f)
    rc, _ = _static_fit(lib, H, f, out, 1e-10)
    assert rc == ms.MS_ERR_ARG
    assert "65536" in ms.ms_last_error()
    H.close()
