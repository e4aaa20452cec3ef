"""The opt-in autotuner (ms_opts.autotune): it picks the CSR lanes per row of each
level of at least 4096 rows (matrix-free operator: lanes per target point) by
timing the stand-alone mat-vec, caches the choice per level shape, and leaves the
fitted coefficients unchanged up to the CG tolerance.
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
    assert torch.cuda.is_available()
    B.build()
    ms.load()


def workload(sizes, seed=41):
    allp = inputs.scrambled_halton(max(sizes), 2, seed)
    levels = [np.ascontiguousarray(allp[:n]) for n in sizes]
    h = np.array([n ** -0.5 for n in sizes])
    g = inputs.GaussianMixture(6, 2, seed + 1, sine=True)
    return inputs.Workload("tune", 2, levels, h, 6.0, 2, 1, g(np.concatenate(levels)), g)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SIZES = [300, 1500, 6000, 24000]


@pytest.mark.parametrize("prec", [ms.MS_PREC_FP64, ms.MS_PREC_MIXED])
def test_autotune_keeps_the_fit_and_reports_valid_widths(prec):
    w = workload(SIZES)
    H0 = ms.Hierarchy.from_workload(w, precision=prec)
    H1 = ms.Hierarchy.from_workload(w, precision=prec, autotune=1)
    a0, _ = H0.fit(w.f, rel_tol=1e-12)
    rule = H0.info()["tpr_A"]
    before = ms.ms_launch_count()
    a1, st = H1.fit(w.f, rel_tol=1e-12)
    first = ms.ms_launch_count() - before
    tuned = H1.info()["tpr_A"]
    for l, n in enumerate(SIZES):
        assert tuned[l] in (1, 2, 4, 8, 16, 32), tuned
        if n < 4096:
            assert tuned[l] == rule[l], (l, tuned, rule)  # small levels keep the rule
    assert max(st["rel_residual"]) <= 1e-12
    tol = 1e-10 if prec == ms.MS_PREC_FP64 else 1e-8
    assert rel(a1, a0) <= tol
    ref, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, w.wendland_d, w.wendland_k)
    assert rel(a1, np.concatenate(ref)) <= tol
    # the second fit of the handle does no timing; a new handle of the same shape hits the cache
    before = ms.ms_launch_count()
    a2, _ = H1.fit(w.f, rel_tol=1e-12)
    second = ms.ms_launch_count() - before
    assert second < first
    H2 = ms.Hierarchy.from_workload(w, precision=prec, autotune=1)
    before = ms.ms_launch_count()
    H2.fit(w.f, rel_tol=1e-12)
    assert ms.ms_launch_count() - before == second
    assert H2.info()["tpr_A"] == tuned
    for H in (H0, H1, H2):
        H.close()


def test_autotune_matrix_free():
    w = workload(SIZES)
    H0 = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, op=ms.MS_OP_MATRIX_FREE)
    H1 = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, op=ms.MS_OP_MATRIX_FREE, autotune=1)
    a0, _ = H0.fit(w.f, rel_tol=1e-12)
    a1, st = H1.fit(w.f, rel_tol=1e-12)
    assert max(st["rel_residual"]) <= 1e-12
    assert rel(a1, a0) <= 1e-8
    H0.close()
    H1.close()


def test_explicit_threads_per_row_overrides_autotune():
    w = workload(SIZES)
    H = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_FP64, autotune=1, threads_per_row=4)
    a, st = H.fit(w.f, rel_tol=1e-12)
    assert H.info()["tpr_A"] == [4] * len(SIZES)
    assert max(st["rel_residual"]) <= 1e-12
    H.close()


def test_peak_probes_are_plausible():
    """The instruction-rate probes behind the ALU rooflines: FP32 FMA issue far above FP64
    (GB300: 64x) and above the special-function unit's rsqrt rate."""
    f32 = ms.ms_peak_probe(ms.MS_PROBE_FP32)
    f64 = ms.ms_peak_probe(ms.MS_PROBE_FP64)
    xu = ms.ms_peak_probe(ms.MS_PROBE_XU)
    assert f32 > 4 * xu > 0 and f32 > 16 * f64 > 0, (f32, f64, xu)


def test_autotune_cell_size_and_ctas_per_sm():
    """autotune = 1 also picks the neighbour-grid cell size at the build (delta or delta / 2: the
    build plus one application of the fit's matrix-free operators, timed) and the solve kernel's
    CTAs per SM at the first fit (which fits with 1 and with 2 and keeps the faster);
    ms_hierarchy_info reports both, a new handle of the same shape takes the cached choices, and
    the coefficients agree with an untuned fit to the CG tolerance."""
    w = workload(SIZES)
    kw = {"precision": ms.MS_PREC_MIXED, "lower_op": ms.MS_OP_MATRIX_FREE}
    H0 = ms.Hierarchy.from_workload(w, **kw)
    assert H0.info()["cell_split"] == 1 and H0.info()["solve_ctas_per_sm"] == 2
    a0, _ = H0.fit(w.f, rel_tol=1e-12)
    H1 = ms.Hierarchy.from_workload(w, autotune=1, **kw)
    split = H1.info()["cell_split"]
    assert split in (1, 2)
    a1, st = H1.fit(w.f, rel_tol=1e-12)
    ctas = H1.info()["solve_ctas_per_sm"]
    assert ctas in (1, 2)
    assert max(st["rel_residual"]) <= 1e-12
    assert rel(a1, a0) <= 1e-8
    H2 = ms.Hierarchy.from_workload(w, autotune=1, **kw)
    assert H2.info()["cell_split"] == split
    before = ms.ms_launch_count()
    a2, _ = H2.fit(w.f, rel_tol=1e-12)
    once = ms.ms_launch_count() - before
    assert H2.info()["solve_ctas_per_sm"] == ctas
    before = ms.ms_launch_count()
    H2.fit(w.f, rel_tol=1e-12)
    assert ms.ms_launch_count() - before == once  # the cached choice: one fit, no timing runs
    assert rel(a2, a0) <= 1e-8
    for H in (H0, H1, H2):
        H.close()
