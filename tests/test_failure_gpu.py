"""Failure detection on the GPU without a fault: the bounded waits of the solve kernel.

Every wait of the persistent solve kernel (its grid barriers) gives up after a time
limit, records MS_ERR_TIMEOUT in the device status word and returns, so that the host
reads an error and the CUDA context stays usable.  ms_wait_selftest runs that barrier
code with a partner CTA that never arrives (a flag that nothing sets).  These tests
check that the wait ends at its limit with the status recorded, that a wait leaves
early once another CTA has recorded a time-out, and that the process can still fit a
hierarchy afterwards (compared with the CPU oracle).
"""
import numpy as np
import pytest

from oracle import multiscale as om
from paper_2503_04914_gb300 import build as B
from paper_2503_04914_gb300 import inputs, ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    ms.load()


def test_barrier_wait_times_out_and_records_the_status():
    for limit in (0.02, 0.2):
        status, waited = ms.ms_wait_selftest(limit)
        assert status == ms.MS_ERR_TIMEOUT
        # the limit is checked every 256 polls of the barrier word (well under a millisecond)
        assert limit <= waited < limit + 0.5, (limit, waited)


def test_barrier_wait_leaves_when_another_cta_timed_out():
    status, waited = ms.ms_wait_selftest(5.0, peer_timed_out=True)
    assert status == ms.MS_ERR_TIMEOUT
    assert waited < 0.1, waited


def test_context_is_usable_after_a_timed_out_wait():
    ms.ms_wait_selftest(0.02)
    sizes = (40, 300, 1500)
    allp = inputs.scrambled_halton(max(sizes), 2, 5)
    levels = [np.ascontiguousarray(allp[:n]) for n in sizes]
    h = np.array([n ** -0.5 for n in sizes])
    g = inputs.GaussianMixture(6, 2, 6, sine=True)
    w = inputs.Workload("after-timeout", 2, levels, h, 4.0, 2, 1, g(np.concatenate(levels)), g)
    H = ms.Hierarchy.from_workload(w)
    a, st = H.fit(w.f, rel_tol=1e-12)
    ref, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, w.wendland_d, w.wendland_k)
    ref = np.concatenate(ref) if isinstance(ref, (list, tuple)) else ref
    assert np.linalg.norm(a - ref) <= 1e-10 * np.linalg.norm(ref)
    H.close()
