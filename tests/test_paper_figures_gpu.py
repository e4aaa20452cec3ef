"""The paper's Section 5 figures through the library's GPU operators.

The Jacobi operator M = I - T'_L = -(T_L - D_L) D_L^{-1} (eq. M) is assembled column by column
through the C ABI on the paper's grid hierarchy (grids (2^l+1)^2 on [0,1]^2, nu = 4, phi_{3,1},
h = fill distance): D_L^{-1} e_k by multi-right-hand-side fits with jacobi_sweeps = -1 (the
block-diagonal solve of eq. split alone, FP64 CG to rel_tol 1e-13), then -(T_L - D_L) by
ms_apply_dev(MS_APPLY_B64).  From it:
  * Figure 1: ||M_L||_2 for L = 2..7, to the printed three decimals;
  * Figure 2: ||M_L - M~_L(T)||_2 / ||M_L||_2 for the thresholded operator of eq. perturbedmatrix
    (entries with |x_i - x_k| >= T q_j dropped), L = 3..7, T = 1..6, to the printed five decimals;
  * Figure 3: nnz(M~_L(T)) / nnz(M_L), counting entries above 1e-8 (the cut that reproduces the
    printed ratios; see oracle.multiscale.nonzero_count), to the printed five decimals;
  * for L <= 5, the assembled M against the oracle's dense M element by element (1e-10 of max|M|).
Norms come from the largest eigenvalue of M^T M and the distances from the points themselves
(dense torch reductions of the assembled matrix: measurement, not a step of the method).
"""
import os

import numpy as np
import pytest

from oracle import multiscale as om
from paper_2503_04914_gb300 import build as B
from paper_2503_04914_gb300 import inputs, ms

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                r = line.split()
                out[int(r[0])] = [float(x) for x in r[1:]]
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    ms.load()


def assembled_jacobi(L):
    """(workload, M [N][ncol] on the device) with ncol = the points of levels 1..L-1 (the last
    block column of M is zero)."""
    import torch
    w = inputs.franke_grid_hierarchy(L)
    H = ms.Hierarchy.from_workload(w, device=True, precision=ms.MS_PREC_FP64, jacobi_sweeps=-1)
    off = om.level_offsets(w.levels)
    N, ncol = int(off[-1]), int(off[-2])
    E = torch.zeros((N, ncol), dtype=torch.float64, device="cuda")
    idx = torch.arange(ncol, device="cuda")
    E[idx, idx] = 1.0
    # D^{-1} E (input order).  1e-13 where M is compared element-wise with the oracle (L <= 5);
    # 1e-12 above, where the figures need five digits: with unit-vector columns an FP64 residual
    # of 1e-13 is near kappa(A_l) eps on the finer grids, and whether a column reaches it
    # depends on the order of its dot products' sums (1e-13 ran into the iteration cap at L = 6, 7
    # when blocks of 32 columns shared one partitioned launch)
    Y, st = H.fit(E, rel_tol=1e-13 if L <= 5 else 1e-12)
    assert st["device_status"] == 0 and st["sweeps"] == 0
    Yt = Y.t().contiguous()
    del E, Y
    M = torch.empty((ncol, N), dtype=torch.float64, device="cuda")
    for c in range(ncol):
        H.apply(ms.MS_APPLY_B64, Yt[c], M[c])
    H.close()
    return w, -M.t().contiguous()


def norm2(M):
    import torch
    G = M.t() @ M
    return float(torch.sqrt(torch.linalg.eigvalsh(G)[-1]))


def survive_mask(w, ncol, T):
    """|x_i - x_k| < T q_j for column k of level j (q_j: separation distance of level j)."""
    import torch
    off = om.level_offsets(w.levels)
    P = torch.from_numpy(w.points).cuda()
    mask = torch.zeros((int(off[-1]), ncol), dtype=torch.bool, device="cuda")
    for j in range(len(w.levels) - 1):
        Xj = P[off[j]:off[j + 1]]
        Dj = torch.cdist(Xj, Xj)
        Dj.fill_diagonal_(float("inf"))
        qj = 0.5 * float(Dj.min())
        mask[:, off[j]:off[j + 1]] = torch.cdist(P, Xj) < T * qj
    return mask


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 7])
def test_figures_1_2_3_through_the_gpu_operators(L):
    import torch
    w, M = assembled_jacobi(L)
    nM = norm2(M)
    want = _golden("fig1_mnorm.txt")[L][0]
    assert round(nM, 3) == pytest.approx(want, abs=1.01e-3), (L, nM, want)
    if L <= 5:
        ref = om.jacobi_matrix(w.levels, w.h, w.nu, w.wendland_d, w.wendland_k)[:, :M.shape[1]]
        assert np.abs(M.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    if L < 3:
        return
    fig2 = _golden("fig2_norm_ratio.txt")[L]
    fig3 = _golden("fig3_nnz_ratio.txt")[L]
    big = M.abs() > 1e-8 * float(M.abs().max())
    n0 = int(big.sum())
    for T in range(1, 7):
        mask = survive_mask(w, M.shape[1], T)
        ratio = norm2(torch.where(mask, torch.zeros_like(M), M)) / nM
        nnz = int((big & mask).sum()) / n0
        assert round(ratio, 5) == pytest.approx(fig2[T - 1], abs=1.01e-5), (L, T, ratio)
        assert round(nnz, 5) == pytest.approx(fig3[T - 1], abs=1.01e-5), (L, T, nnz)


def test_convergence_rate_theorem2():
    """Theorem 2 / Corollary 3: ||f - f_L||_{L2} <= C (C_1 mu^tau)^L ||f||, geometric in L.  The
    Franke function fitted on the paper's grids for L = 1..10 (plain FP64, rel_tol 1e-12) and
    evaluated at 65,536 seeded random points (off every grid node: at the cell centres of a
    256^2 grid, which are nodes of the 9- and 10-level grids, the interpolant is exact): the RMS
    errors of L <= 6 equal the oracle's (1e-6 relative), every level lowers the error, and the
    least-squares rate over L = 2..10 is below 1/2 (mu = 1/2 per level here; the oracle measures
    per-level ratios of 0.08-0.3)."""
    import torch
    Qh = inputs.query_random(65536, 2)
    Q = torch.from_numpy(Qh).cuda()
    fq = inputs.franke(Qh)
    errs = []
    for L in range(1, 11):
        w = inputs.franke_grid_hierarchy(L)
        H = ms.Hierarchy.from_workload(w, device=True, precision=ms.MS_PREC_FP64)
        a, st = H.fit(torch.from_numpy(w.f).cuda(), rel_tol=1e-12)
        s = H.evaluate(a, Q).cpu().numpy()
        H.close()
        e = float(np.sqrt(np.mean((s - fq) ** 2)))
        errs.append(e)
        if L <= 6:
            al, _ = om.fit_sequential(w.levels, w.f, w.h, w.nu, 3, 1)
            so = om.evaluate(w.levels, al, w.h, w.nu, 3, 1, Qh)
            eo = float(np.sqrt(np.mean((so - fq) ** 2)))
            assert abs(e - eo) <= 1e-6 * eo, (L, e, eo)
    assert all(b < a for a, b in zip(errs, errs[1:])), f"RMS errors by level: {errs}"
    Ls = np.arange(2, 11)
    rate = float(np.exp(np.polyfit(Ls, np.log(errs[1:]), 1)[0]))
    assert rate < 0.5, (rate, errs)
