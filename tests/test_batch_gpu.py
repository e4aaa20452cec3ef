"""GPU parity of the batched fit (several hierarchies in one launch, ms_fit_batch)
against single fits and the CPU FP64 oracle.

Each hierarchy of a batch runs on its own partition of the grid, so its dot
products are summed over fewer CTAs than in a single fit: results agree with the
single fit to the CG tolerance (1e-10 FP64, 1e-8 MIXED at rel_tol 1e-12), not
bitwise; a repeated batch is bitwise identical.
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


def hierarchy(sizes, seed, d=2):
    """Nested scrambled-Halton levels of the given sizes, h = N^-1/d, delta = 4h, phi_{d,1}."""
    allp = inputs.scrambled_halton(max(sizes), d, seed)
    levels = [np.ascontiguousarray(allp[:n]) for n in sizes]
    h = np.array([n ** (-1.0 / d) for n in sizes])
    g = inputs.GaussianMixture(6, d, seed + 1, sine=(d == 2))
    return inputs.Workload(f"b{seed}", d, levels, h, 4.0, d, 1, g(np.concatenate(levels)), g)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ragged sizes, 1 to 5 levels (one with a single-point level)
SIZES = [[40, 160, 640, 2560], [1, 30, 300], [500], [64, 256, 1024, 4096, 9000], [100, 400, 1600],
         [20, 80, 320, 1280, 5120]]


@pytest.mark.parametrize("prec", [ms.MS_PREC_FP64, ms.MS_PREC_MIXED])
def test_batch_matches_single_fits_and_oracle(prec):
    ws = [hierarchy(s, 300 + i) for i, s in enumerate(SIZES)]
    Hs = [ms.Hierarchy.from_workload(w, precision=prec) for w in ws]
    handles = [H.handle for H in Hs]
    A, st = ms.ms_fit_batch(handles, [w.f for w in ws], rel_tol=1e-12)
    A2, _ = ms.ms_fit_batch(handles, [w.f for w in ws], rel_tol=1e-12)
    tol = 1e-10 if prec == ms.MS_PREC_FP64 else 1e-8
    for i, (w, H) in enumerate(zip(ws, Hs)):
        assert np.array_equal(A[i], A2[i]), i
        assert max(st[i]["rel_residual"]) <= 1e-12, (i, st[i])
        assert st[i]["device_status"] == 0
        a1, _ = H.fit(w.f, rel_tol=1e-12)
        assert rel(A[i], a1) <= tol, (i, rel(A[i], a1))
        ref, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, w.wendland_d, w.wendland_k)
        assert rel(A[i], np.concatenate(ref)) <= tol, i
    for H in Hs:
        H.close()


def test_batch_device_api_mixed_options():
    """Device pointers; hierarchies with different operators and preconditioners in one batch."""
    import torch
    ws = [hierarchy(s, 400 + i) for i, s in enumerate(SIZES[:4])]
    over = [{}, {"op": ms.MS_OP_MATRIX_FREE}, {"precond": ms.MS_PRECOND_EXACT}, {"cell_split": 2}]
    Hs = [ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, **o) for w, o in zip(ws, over)]
    fs = [torch.from_numpy(w.f).cuda() for w in ws]
    A, st = ms.ms_fit_batch([H.handle for H in Hs], fs, rel_tol=1e-12)
    torch.cuda.synchronize()
    for i, (w, H) in enumerate(zip(ws, Hs)):
        ref, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, w.wendland_d, w.wendland_k)
        assert rel(A[i].cpu().numpy(), np.concatenate(ref)) <= 1e-8, (i, st[i])
        H.close()


def test_batch_rejects_mixed_precisions_and_reports_failures():
    w0, w1 = hierarchy([50, 200], 500), hierarchy([60, 240], 501)
    H0 = ms.Hierarchy.from_workload(w0, precision=ms.MS_PREC_FP64)
    H1 = ms.Hierarchy.from_workload(w1, precision=ms.MS_PREC_MIXED)
    with pytest.raises(ms.MsError) as e:
        ms.ms_fit_batch([H0.handle, H1.handle], [w0.f, w1.f])
    assert e.value.status == ms.MS_ERR_ARG
    # a non-finite right-hand side fails its own hierarchy and names it
    H2 = ms.Hierarchy.from_workload(w1, precision=ms.MS_PREC_FP64)
    bad = w1.f.copy()
    bad[3] = np.nan
    with pytest.raises(ms.MsError) as e:
        ms.ms_fit_batch([H0.handle, H2.handle], [w0.f, bad])
    assert e.value.status == ms.MS_ERR_NUMERIC
    assert "hierarchy 1" in ms.ms_last_error()
    # the handles stay usable
    a, _ = H0.fit(w0.f, rel_tol=1e-12)
    ref, _ = om.fit_sequential(w0.levels, w0.f, w0.h, w0.nu, 2, 1)
    assert rel(a, np.concatenate(ref)) <= 1e-10
    for H in (H0, H1, H2):
        H.close()


def test_batch_is_faster_than_single_fits():
    """16 small hierarchies in one launch take less device time than 16 single fits."""
    rng = np.random.default_rng(7)
    ws = []
    for i in range(16):
        L = int(rng.integers(3, 6))
        ws.append(hierarchy([int(40 * 4 ** j) for j in range(L)], 600 + i))
    Hs = [ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED) for w in ws]
    handles = [H.handle for H in Hs]
    ms.ms_fit_batch(handles, [w.f for w in ws], rel_tol=1e-10)
    _, st = ms.ms_fit_batch(handles, [w.f for w in ws], rel_tol=1e-10)
    t_single = 0.0
    for w, H in zip(ws, Hs):
        _, s = H.fit(w.f, rel_tol=1e-10)
        t_single += s["fit_ms"]
    assert st[0]["fit_ms"] < 0.5 * t_single, (st[0]["fit_ms"], t_single)
    for H in Hs:
        H.close()


def _plan_setup(seed0, prec=ms.MS_PREC_MIXED):
    import torch
    ws = [hierarchy(s, seed0 + i) for i, s in enumerate(SIZES)]
    Hs = [ms.Hierarchy.from_workload(w, precision=prec) for w in ws]
    fs = [torch.from_numpy(w.f).cuda() for w in ws]
    return ws, Hs, fs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_plan_matches_batch_fit_and_replays(use_graph):
    """A prepared plan gives the batched fit's coefficients bitwise (same partition, same
    arithmetic), launch after launch, and picks up new values in the bound buffers."""
    import torch
    ws, Hs, fs = _plan_setup(700)
    handles = [H.handle for H in Hs]
    ref, _ = ms.ms_fit_batch(handles, [w.f for w in ws], rel_tol=1e-12)
    plan = ms.BatchPlan(handles, fs, rel_tol=1e-12)
    for _ in range(3):
        plan.launch(use_graph=use_graph)
        st = plan.stats()
        for i in range(len(ws)):
            assert np.array_equal(plan.alphas[i].cpu().numpy(), ref[i]), i
            assert st[i]["device_status"] == 0 and max(st[i]["rel_residual"]) <= 1e-12
    # new right-hand sides in the same buffers
    rng = np.random.default_rng(5)
    new = [rng.standard_normal(w.N) for w in ws]
    for f, v in zip(fs, new):
        f.copy_(torch.from_numpy(v))
    plan.launch(use_graph=use_graph)
    plan.stats()
    ref2, _ = ms.ms_fit_batch(handles, new, rel_tol=1e-12)
    for i, w in enumerate(ws):
        a = plan.alphas[i].cpu().numpy()
        assert np.array_equal(a, ref2[i]), i
        o, _ = om.fit_sequential(w.levels, new[i], w.h, w.nu, w.wendland_d, w.wendland_k)
        assert rel(a, np.concatenate(o)) <= 1e-8, i
    plan.close()
    for H in Hs:
        H.close()


def test_batch_plan_captured_by_the_caller_into_a_cuda_graph():
    import torch
    ws, Hs, fs = _plan_setup(720, prec=ms.MS_PREC_FP64)
    handles = [H.handle for H in Hs]
    ref, _ = ms.ms_fit_batch(handles, [w.f for w in ws], rel_tol=1e-12)
    plan = ms.BatchPlan(handles, fs, rel_tol=1e-12)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.launch(stream=s.cuda_stream)
    for a in plan.alphas:
        a.zero_()
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    st = plan.stats()
    for i in range(len(ws)):
        assert np.array_equal(plan.alphas[i].cpu().numpy(), ref[i]), i
        assert st[i]["device_status"] == 0
    del g
    plan.close()
    for H in Hs:
        H.close()


def test_batch_plan_guards():
    import torch
    ws, Hs, fs = _plan_setup(740, prec=ms.MS_PREC_FP64)
    handles = [H.handle for H in Hs]
    with pytest.raises(ms.MsError) as e:  # a hierarchy twice would share its work space
        ms.BatchPlan([handles[0], handles[0]], [fs[0], fs[0].clone()])
    assert e.value.status == ms.MS_ERR_ARG
    plan = ms.BatchPlan(handles, fs, rel_tol=1e-12)
    # the work space of a planned hierarchy cannot grow (3 right-hand sides after 1)
    w = ws[0]
    F = np.stack([w.f, 2 * w.f, -w.f], axis=1)
    with pytest.raises(ms.MsError) as e:
        Hs[0].fit(F, rel_tol=1e-12)
    assert e.value.status == ms.MS_ERR_STATE
    a1, _ = Hs[0].fit(w.f, rel_tol=1e-12)  # one right-hand side fits in the existing space
    # destroying a hierarchy invalidates the plan
    Hs[1].close()
    with pytest.raises(ms.MsError) as e:
        plan.launch()
    assert e.value.status == ms.MS_ERR_STATE
    plan.close()
    aF, _ = Hs[0].fit(F, rel_tol=1e-12)  # the plan is gone: the space may grow again
    assert rel(aF[:, 0], a1) <= 1e-10
    for H in Hs:
        H.close()


def test_batch_with_learned_preconditioner_matches_single_fits():
    """Hierarchies with the learned preconditioner (weights imported) fitted in one batched launch:
    the same coefficients as their single fits (to the CG tolerance), and real residuals."""
    ws = [hierarchy(s, 800 + i) for i, s in enumerate([[40, 160, 640, 2560], [100, 400, 1600], [64, 256, 1024, 4096]])]
    Ht = ms.Hierarchy.from_workload(ws[2], precision=ms.MS_PREC_MIXED, precond=ms.MS_PRECOND_LEARNED)
    Ht.train_precond([0, 1], epochs=20)
    params = Ht.precond_params()
    Hs = [ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, precond=ms.MS_PRECOND_LEARNED) for w in ws]
    for H in Hs:
        H.precond_params(params)
    A, st = ms.ms_fit_batch([H.handle for H in Hs], [w.f for w in ws], rel_tol=1e-12)
    for i, (w, H) in enumerate(zip(ws, Hs)):
        res = st[i]["rel_residual"]
        assert 0 < max(res) <= 1e-12, (i, res)
        assert st[i]["precond_fallbacks"] == 0
        a1, s1 = H.fit(w.f, rel_tol=1e-12)
        assert rel(A[i], a1) <= 1e-8, (i, rel(A[i], a1))
        ref, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, w.wendland_d, w.wendland_k)
        assert rel(A[i], np.concatenate(ref)) <= 1e-8, i
    for H in Hs + [Ht]:
        H.close()
