"""GPU parity of the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances: the FP64 path must match the oracle's coefficients to 1e-10
relative per level and the approximant to 1e-10; the MIXED path (FP32
mat-vecs, FP64 dots and refinement) to 1e-8 (it is refined to the same FP64
true-residual tolerance).  Element-wise operator checks use 1e-13 (FP64) and
1e-6 (FP32 values) relative to the row's absolute sum.
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


def ragged_halton(sizes, nu=4.0, wendland=(2, 1), seed=77, n_gauss=8):
    allp = inputs.scrambled_halton(max(sizes), 2, seed)
    levels = [np.ascontiguousarray(allp[:n]) for n in sizes]
    h = np.array([n ** -0.5 for n in sizes])
    g = inputs.GaussianMixture(n_gauss, 2, seed + 1, sine=True)
    f = g(np.concatenate(levels))
    return inputs.Workload("ragged", 2, levels, h, nu, wendland[0], wendland[1], f, g)


def oracle_fit(w, f=None):
    a, _ = om.fit_sequential(w.levels, w.f if f is None else f, w.h, w.nu, w.wendland_d, w.wendland_k)
    return a


def split(w, flat):
    off = om.level_offsets(w.levels)
    return [flat[off[l]:off[l + 1]] for l in range(w.L)]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def check_fit(w, prec, tol_coef, rel_tol=1e-12, tol_approx=None, **over):
    tol_approx = tol_coef if tol_approx is None else tol_approx
    H = ms.Hierarchy.from_workload(w, precision=prec, **over)
    alpha, st = H.fit(w.f, rel_tol=rel_tol)
    ref = oracle_fit(w)
    for l, (a, r) in enumerate(zip(split(w, alpha), ref)):
        assert rel(a, r) <= tol_coef, (l, rel(a, r), st)
    Q = inputs.query_grid(64, w.d)
    s_gpu = H.evaluate(alpha, Q)
    s_ref = om.evaluate(w.levels, ref, w.h, w.nu, w.wendland_d, w.wendland_k, Q)
    assert rel(s_gpu, s_ref) <= tol_approx
    for l in range(w.L):
        assert st["rel_residual"][l] <= rel_tol
    H.close()
    return st


# ------------------------------------------------------------------ operators


@pytest.mark.parametrize("prec", [ms.MS_PREC_FP64, ms.MS_PREC_MIXED])
@pytest.mark.parametrize("wl", ["grid", "ragged"])
def test_operators_match_oracle_matrices(wl, prec):
    """Stored entries against the oracle's dense blocks, per row relative to sum |M||x|: FP64
    entries 1e-14 (FP64 accumulation of ~50 products); the MIXED build's FP64 entries come
    from double-float arithmetic (about 48 bits): 1e-13; FP32 copies 2e-6."""
    import torch
    w = inputs.grid_hierarchy_small() if wl == "grid" else ragged_halton([37, 150, 601, 2500])
    H = ms.Hierarchy.from_workload(w, precision=prec, lower_fp32=1)
    off = om.level_offsets(w.levels)
    x = np.random.default_rng(3).standard_normal(w.N)
    # dense oracle blocks
    yA = np.zeros(w.N)
    yB = np.zeros(w.N)
    absA = np.zeros(w.N)
    absB = np.zeros(w.N)
    for k in range(w.L):
        rows = slice(off[k], off[k + 1])
        for j in range(k + 1):
            M = om.kernel_dense(w.levels[k], w.levels[j], w.nu * w.h[j], w.wendland_d, w.wendland_k)
            c = x[off[j]:off[j + 1]]
            if j == k:
                yA[rows] += M @ c
                absA[rows] += np.abs(M) @ np.abs(c)
            else:
                yB[rows] += M @ c
                absB[rows] += np.abs(M) @ np.abs(c)
    xt = torch.from_numpy(x).cuda()
    t64 = 1e-14 if prec == ms.MS_PREC_FP64 else 1e-13
    ops = [(ms.MS_APPLY_A64, yA, absA, t64), (ms.MS_APPLY_B64, yB, absB, t64), (ms.MS_APPLY_B32, yB, absB, 2e-6)]
    if prec == ms.MS_PREC_MIXED:
        ops.append((ms.MS_APPLY_A32, yA, absA, 2e-6))
    for op, ref, scale, tol in ops:
        y = H.apply(op, xt).cpu().numpy()
        err = np.abs(y - ref) / np.maximum(scale, 1e-300)
        assert err.max() <= tol, (op, err.max())
    info = H.info()
    nnzA = sum(int((om.kernel_dense(X, X, w.nu * w.h[l], w.wendland_d, w.wendland_k) != 0).sum())
               for l, X in enumerate(w.levels))
    assert info["nnz_A"] == nnzA
    H.close()


@pytest.mark.parametrize("wl", ["grid", "ragged_nu8_w22", "random3d_w31"])
def test_matrix_free_lower_operators_match_oracle(wl):
    """y = (T_L - D_L) x with B's entries recomputed (the paper's McV without a stored matrix),
    against the oracle's dense blocks, per row relative to sum |B||x|: double-float entries and
    sums (about 48 bits, the fit's lower_op = MATRIX_FREE) 1e-13; FP32 entries and sums 2e-6.
    The handle stores no B (lower_op = MATRIX_FREE), and the CSR lower operators refuse."""
    import torch
    if wl == "grid":
        w = inputs.grid_hierarchy_small()
    elif wl == "ragged_nu8_w22":
        w = ragged_halton([37, 150, 601, 2500], nu=8.0, wendland=(2, 2))
    else:
        w = inputs.random3d_hierarchy(L=3, n_gauss=3)
    H = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, lower_op=ms.MS_OP_MATRIX_FREE)
    assert H.info()["nnz_B"] == 0
    off = om.level_offsets(w.levels)
    x = np.random.default_rng(11).standard_normal(w.N)
    yB = np.zeros(w.N)
    absB = np.zeros(w.N)
    for k in range(1, w.L):
        rows = slice(off[k], off[k + 1])
        for j in range(k):
            M = om.kernel_dense(w.levels[k], w.levels[j], w.nu * w.h[j], w.wendland_d, w.wendland_k)
            yB[rows] += M @ x[off[j]:off[j + 1]]
            absB[rows] += np.abs(M) @ np.abs(x[off[j]:off[j + 1]])
    xt = torch.from_numpy(x).cuda()
    for op, tol in ((ms.MS_APPLY_BMFDF, 1e-13), (ms.MS_APPLY_BMF32, 2e-6)):
        y = H.apply(op, xt).cpu().numpy()
        err = np.abs(y - yB) / np.maximum(absB, 1e-300)
        assert err.max() <= tol, (op, err.max())
        assert np.all(y[:off[1]] == 0.0)
    with pytest.raises(ms.MsError):
        H.apply(ms.MS_APPLY_B64, xt)
    H.close()


@pytest.mark.parametrize("precond", [ms.MS_PRECOND_NONE, ms.MS_PRECOND_EXACT])
@pytest.mark.parametrize("wl", ["nu4_w21", "nu8_w22"])
def test_fit_with_matrix_free_lower_blocks(wl, precond):
    """MIXED fit whose Jacobi updates recompute B's entries (lower_op = MATRIX_FREE) against the
    oracle and against the stored-B MIXED fit.  nu = 4: coefficients 1e-8, approximant 1e-10
    (rel_tol 1e-12); nu = 8, phi_{2,2} (kappa(A_l) ~ 1e5-1e6, so an FP64 residual cannot go much
    below kappa eps ~ 1e-11): rel_tol 1e-11, coefficients 1e-6 and approximant 1e-9, as the
    learned-preconditioner parity test on these levels.  Both fits' approximants agree within
    the approximant tolerance."""
    import torch
    nu, wend, rt, tc, ta = ((4.0, (2, 1), 1e-12, 1e-8, 1e-10) if wl == "nu4_w21" else
                            (8.0, (2, 2), 1e-11, 1e-6, 1e-9))
    w = ragged_halton([37, 150, 601, 2500, 9001], nu=nu, wendland=wend)
    st = check_fit(w, ms.MS_PREC_MIXED, tc, rel_tol=rt, tol_approx=ta, lower_op=ms.MS_OP_MATRIX_FREE,
                   precond=precond)
    assert st["device_status"] == 0
    Hm = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, lower_op=ms.MS_OP_MATRIX_FREE, precond=precond)
    Hc = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, precond=precond)
    Q = inputs.query_grid(64, 2)
    sm = Hm.evaluate(Hm.fit(w.f, rel_tol=rt)[0], Q)
    sc = Hc.evaluate(Hc.fit(w.f, rel_tol=rt)[0], Q)
    assert rel(sm, sc) <= ta
    Hm.close()
    Hc.close()


@pytest.mark.parametrize("wl", ["grid_w21", "halton_nu8_w22", "random3d_w31"])
def test_matrix_free_operator_matches_oracle(wl):
    """y = D_L x with entries recomputed in FP32 from per-cell offsets (no stored matrix),
    against the oracle's dense blocks; FP32 entries and accumulation: 2e-6 of the row's
    absolute sum."""
    import torch
    if wl == "grid_w21":
        w = inputs.grid_hierarchy_small()
    elif wl == "halton_nu8_w22":
        w = inputs.halton_hierarchy(L=3, nu=8.0, wendland=(2, 2), n_gauss=3)
    else:
        w = inputs.random3d_hierarchy(L=2, n_gauss=3)
    H = ms.Hierarchy.from_workload(w)
    off = om.level_offsets(w.levels)
    x = np.random.default_rng(5).standard_normal(w.N)
    y_ref = np.zeros(w.N)
    scale = np.zeros(w.N)
    for l, X in enumerate(w.levels):
        M = om.kernel_dense(X, X, w.nu * w.h[l], w.wendland_d, w.wendland_k)
        c = x[off[l]:off[l + 1]]
        y_ref[off[l]:off[l + 1]] = M @ c
        scale[off[l]:off[l + 1]] = np.abs(M) @ np.abs(c)
    y = H.apply(ms.MS_APPLY_AMF32, torch.from_numpy(x).cuda()).cpu().numpy()
    err = np.abs(y - y_ref) / scale
    assert err.max() <= 2e-6, err.max()
    H.close()


def test_fit_mixed_matrix_free():
    st = check_fit(ragged_halton([37, 150, 601, 2500, 9001]), ms.MS_PREC_MIXED, 1e-8, op=ms.MS_OP_MATRIX_FREE)
    assert sum(st["cg_iterations"]) > 0


def test_sorted_order_is_a_level_preserving_permutation():
    w = ragged_halton([37, 150, 601])
    H = ms.Hierarchy.from_workload(w)
    perm = H.permutation()
    assert sorted(perm.tolist()) == list(range(w.N))
    off = om.level_offsets(w.levels)
    for l in range(w.L):
        seg = perm[off[l]:off[l + 1]]
        assert seg.min() >= off[l] and seg.max() < off[l + 1]
    # deterministic: same inputs, same order
    H2 = ms.Hierarchy.from_workload(w)
    assert np.array_equal(perm, H2.permutation())


# ------------------------------------------------------------------ fits


def test_fit_fp64_grid_hierarchy():
    check_fit(inputs.grid_hierarchy_small(), ms.MS_PREC_FP64, 1e-10)


def test_fit_fp64_ragged_halton():
    check_fit(ragged_halton([37, 150, 601, 2500, 9001]), ms.MS_PREC_FP64, 1e-10)


def test_fit_mixed_ragged_halton():
    st = check_fit(ragged_halton([37, 150, 601, 2500, 9001]), ms.MS_PREC_MIXED, 1e-8)
    assert sum(st["refinements"]) > 0


def test_fit_fp64_halton_phi22_nu8():
    """Ill-conditioned levels (kappa(A_l) ~ 4e5 for nu = 8, phi_{2,2}): a relative residual eps
    bounds the coefficient error by kappa * eps only, so the coefficient bound here is
    kappa * 1e-13 ~ 4e-8 (checked at 1e-8); the approximant stays at 1e-10."""
    w = inputs.halton_hierarchy(L=4, nu=8.0, wendland=(2, 2), n_gauss=5)
    check_fit(w, ms.MS_PREC_FP64, 1e-8, rel_tol=1e-13, tol_approx=1e-10)


def test_fit_d3_random_and_d1():
    w3 = inputs.random3d_hierarchy(L=3, n_gauss=5)
    check_fit(w3, ms.MS_PREC_FP64, 1e-9)
    # jittered 1-D grids (quasi-uniform, so kappa(A_l) stays moderate)
    pts = [((np.arange(n) + 0.25 + 0.5 * inputs.uniform01(11 + l, n)) / n)[:, None]
           for l, n in enumerate([9, 33, 129])]
    g = inputs.GaussianMixture(3, 1, 5)
    w1 = inputs.Workload("d1", 1, pts, np.array([1 / 9, 1 / 33, 1 / 129]), 3.0, 1, 1, g(np.concatenate(pts)), g)
    check_fit(w1, ms.MS_PREC_FP64, 1e-10)


def test_fit_franke_paper_grids():
    check_fit(inputs.franke_grid_hierarchy(5), ms.MS_PREC_FP64, 1e-10)


def test_degenerate_cases():
    # one level; a level with a single point; zero data
    w = ragged_halton([1, 40, 300])
    check_fit(w, ms.MS_PREC_FP64, 1e-10)
    w1 = ragged_halton([500])
    check_fit(w1, ms.MS_PREC_FP64, 1e-10)
    H = ms.Hierarchy.from_workload(w)
    a, st = H.fit(np.zeros(w.N), rel_tol=1e-12)
    assert np.all(a == 0.0)
    with pytest.raises(ms.MsError) as e:
        H.fit(np.full(w.N, np.nan))
    assert e.value.status == ms.MS_ERR_NUMERIC
    with pytest.raises(ms.MsError) as e:
        H.fit(w.f, rel_tol=0.0)
    assert e.value.status == ms.MS_ERR_ARG
    assert H.evaluate(a, np.zeros((0, 2))).shape == (0,)


def _rhs_batch(w, R, seed=999):
    """R right-hand sides: the workload's f, its negative, a zero column, then Gaussian mixtures."""
    cols = [w.f, -w.f, np.zeros(w.N)]
    for r in range(R - 3):
        cols.append(inputs.GaussianMixture(4, w.d, seed + r)(w.points))
    return np.ascontiguousarray(np.stack(cols[:R], axis=1))


@pytest.mark.parametrize("prec,R", [(ms.MS_PREC_FP64, 3), (ms.MS_PREC_FP64, 40), (ms.MS_PREC_MIXED, 40)])
def test_multi_rhs_batch_matches_single_fits_and_oracle(prec, R):
    """All right-hand sides of one call are solved in one launch (up to 32 per launch, every
    (right-hand side, level) pair with its own CG scalars).  The batched launch spreads the rows
    over the CTAs differently from a single fit, so its dot products are summed in another
    (fixed) order: each column matches its single fit to the CG tolerance, not bitwise, and a
    repeated batched call is bitwise identical."""
    w = ragged_halton([37, 150, 601, 2500])
    F = _rhs_batch(w, R)
    H = ms.Hierarchy.from_workload(w, precision=prec)
    A, st = H.fit(F, rel_tol=1e-12)
    A2, _ = H.fit(F, rel_tol=1e-12)
    assert np.array_equal(A, A2)
    assert np.all(A[:, 2] == 0.0)
    assert max(st["rel_residual"][:w.L]) <= 1e-12
    tol = 1e-10 if prec == ms.MS_PREC_FP64 else 1e-8
    for c in sorted({0, 1, 3 % R, R - 1}):
        a, _ = H.fit(np.ascontiguousarray(F[:, c]), rel_tol=1e-12)
        assert rel(A[:, c], a) <= tol, c
    ref = np.concatenate(oracle_fit(w, F[:, [0, R - 1]]))
    assert rel(A[:, 0], ref[:, 0]) <= tol
    assert rel(A[:, R - 1], ref[:, 1]) <= tol
    Q = inputs.query_grid(16, 2)
    S = H.evaluate(A, Q)
    for c in (0, R - 1):
        assert np.array_equal(S[:, c], H.evaluate(np.ascontiguousarray(A[:, c]), Q))
    H.close()


@pytest.mark.parametrize("prec,R,over", [(ms.MS_PREC_FP64, 256, {}),
                                         (ms.MS_PREC_MIXED, 100, {"precond": ms.MS_PRECOND_EXACT})])
def test_many_rhs_in_one_partitioned_launch(prec, R, over):
    """Blocks of 32 right-hand sides share ONE cooperative launch, the grid split into one
    partition of CTAs per block (256 in the row-major SpMM layout, 100 in the right-hand-side-
    major layout with the preconditioner).  Each column matches its single fit to the CG
    tolerance, the zero column stays zero, and a repeated call is bitwise identical."""
    w = ragged_halton([37, 150, 601, 2500])
    F = _rhs_batch(w, R)
    H = ms.Hierarchy.from_workload(w, precision=prec, **over)
    A, st = H.fit(F, rel_tol=1e-12)
    assert st["solve_launches"] == 1 and st["rhs_per_launch"] == R, st
    assert max(st["rel_residual"][:w.L]) <= 1e-12
    A2, _ = H.fit(F, rel_tol=1e-12)
    assert np.array_equal(A, A2)
    assert np.all(A[:, 2] == 0.0)
    tol = 1e-10 if prec == ms.MS_PREC_FP64 else 1e-8
    for c in (0, 31, 32, R - 1):
        a, s1 = H.fit(np.ascontiguousarray(F[:, c]), rel_tol=1e-12)
        assert s1["solve_launches"] == 1 and s1["rhs_per_launch"] == 1
        assert rel(A[:, c], a) <= tol, c
    H.close()


def test_multi_rhs_batch_is_faster_than_single_fits():
    """32 right-hand sides in one launch take far less kernel time than 32 single fits (the
    per-iteration grid barriers and reductions are shared by all of them)."""
    w = ragged_halton([37, 150, 601, 2500])
    F = _rhs_batch(w, 32)
    H = ms.Hierarchy.from_workload(w)
    H.fit(F, rel_tol=1e-10)
    _, st_b = H.fit(F, rel_tol=1e-10)
    t_single = 0.0
    for c in range(32):
        _, s = H.fit(np.ascontiguousarray(F[:, c]), rel_tol=1e-10)
        t_single += s["fit_ms"]
    assert st_b["fit_ms"] < 0.5 * t_single, (st_b["fit_ms"], t_single)
    H.close()


def test_algorithm2_schedule_matches_default():
    """Solving every non-final level in every sweep (Algorithm 2, inter_tol = rel_tol) gives the
    same coefficients as the default schedule, which leaves non-final levels untouched until their
    beta is final; it only runs more CG iterations."""
    w = ragged_halton([37, 150, 601, 2500, 9001])
    a0, s0 = ms.Hierarchy.from_workload(w).fit(w.f, rel_tol=1e-12)
    a1, s1 = ms.Hierarchy.from_workload(w, inter_tol=1e-12).fit(w.f, rel_tol=1e-12)
    assert rel(a1, a0) <= 1e-10
    assert sum(s1["cg_iterations"]) > sum(s0["cg_iterations"])


def test_jacobi_extra_sweep_is_a_fixed_point():
    """beta after L-1 sweeps from beta_0 = f is exact (Theorem 9): one more sweep changes nothing."""
    w = ragged_halton([37, 150, 601, 2500])
    a1, _ = ms.Hierarchy.from_workload(w).fit(w.f, rel_tol=1e-12)
    a2, st = ms.Hierarchy.from_workload(w, jacobi_sweeps=w.L).fit(w.f, rel_tol=1e-12)
    assert st["sweeps"] == w.L
    assert np.array_equal(a1, a2)


def test_device_api_matches_host_api_and_is_deterministic():
    import torch
    w = ragged_halton([37, 150, 601, 2500])
    H = ms.Hierarchy.from_workload(w, device=True)
    a_host, _ = H.fit(w.f, rel_tol=1e-12)
    f = torch.from_numpy(w.f).cuda()
    a_dev, _ = H.fit(f, rel_tol=1e-12)
    torch.cuda.synchronize()
    assert np.array_equal(a_host, a_dev.cpu().numpy())
    Q = torch.from_numpy(inputs.query_grid(32, 2)).cuda()
    s = H.evaluate(a_dev, Q)
    torch.cuda.synchronize()
    assert np.array_equal(s.cpu().numpy(), H.evaluate(a_host, Q.cpu().numpy()))


# ------------------------------------------------------------------ full size (sampled)


@pytest.mark.parametrize("prec", [ms.MS_PREC_FP64, ms.MS_PREC_MIXED])
def test_full_size_halton8_sampled_rows(prec):
    """d=2, 8 Halton levels (1.4M points): rows of T alpha - f sampled and summed by the oracle
    one by one (brute force over every point of the levels involved)."""
    w = inputs.halton_hierarchy(L=8)
    H = ms.Hierarchy.from_workload(w, precision=prec)
    alpha, st = H.fit(w.f, rel_tol=1e-11)
    assert max(st["rel_residual"]) <= 1e-11
    fmax = np.abs(w.f).max()
    rng = np.random.default_rng(8)
    for l in range(w.L):
        idx = rng.choice(len(w.levels[l]), size=min(12, len(w.levels[l])), replace=False)
        for i in idx:
            r = om.row_residual(w.levels, alpha, w.f, w.h, w.nu, 2, 1, l, int(i))
            assert abs(r) <= 1e-8 * fmax, (l, i, r)
    # the approximant reproduces f on the finest level (interpolation property)
    pts = w.levels[-1][rng.choice(len(w.levels[-1]), 64, replace=False)]
    s = H.evaluate(alpha, pts)
    assert np.max(np.abs(s - w.f_fun(pts))) <= 1e-8 * fmax
    H.close()


def test_mixed_falls_back_to_fp64_when_refinement_stalls():
    """A MIXED level whose outer refinement round does not halve the FP64 residual runs its
    inner CG in FP64 from then on.  inner_tol = 0.9 makes every FP32 inner solve stop after a
    10% reduction, so the second round of every level triggers the switch; the fit must then
    match the oracle like the FP64 path."""
    w = ragged_halton([37, 150, 601, 2500])
    H = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, inner_tol=0.9)
    a, st = H.fit(w.f, rel_tol=1e-12)
    assert st["fp64_fallbacks"] >= 3, st
    assert max(st["rel_residual"]) <= 1e-12
    ref = np.concatenate(oracle_fit(w))
    assert rel(a, ref) <= 1e-10
    H.close()


def test_mixed_converges_on_a_nearly_singular_level():
    """Pairs of points 1e-3 h apart make the finest level's A_l ill-conditioned far beyond
    FP32; MIXED (FP32 inner CG with FP64 refinement, FP64 inner CG where refinement stalls)
    still certifies rel_tol and matches the oracle's approximant."""
    sizes = [50, 400, 3000]
    allp = inputs.scrambled_halton(max(sizes), 2, 91)
    levels = [np.ascontiguousarray(allp[:n]) for n in sizes]
    h = np.array([n ** -0.5 for n in sizes])
    idx = np.arange(0, 3000, 100)                      # 30 points get a near-twin
    ang = 2 * np.pi * inputs.uniform01(92, len(idx))
    twins = levels[2][idx] + 1e-3 * h[2] * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    levels[2] = np.ascontiguousarray(np.concatenate([levels[2], np.clip(twins, 0.0, 1.0)]))
    g = inputs.GaussianMixture(6, 2, 93, sine=True)
    w = inputs.Workload("twins", 2, levels, h, 4.0, 2, 1, g(np.concatenate(levels)), g)
    H = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED)
    a, st = H.fit(w.f, rel_tol=1e-11)
    assert max(st["rel_residual"]) <= 1e-11, st
    ref = oracle_fit(w)
    Q = inputs.query_grid(48, 2)
    s_gpu = H.evaluate(a, Q)
    s_ref = om.evaluate(w.levels, ref, w.h, w.nu, 2, 1, Q)
    assert rel(s_gpu, s_ref) <= 1e-6
    H.close()


@pytest.mark.parametrize("over", [{"precond": ms.MS_PRECOND_EXACT}, {"op": ms.MS_OP_MATRIX_FREE}])
def test_multi_rhs_with_preconditioner_or_matrix_free(over):
    """Several right-hand sides with the FSAI preconditioner or the matrix-free operator take the
    right-hand-side-major layout (the row-major SpMM layout serves plain CSR fits); each column
    matches its single fit and the oracle."""
    w = ragged_halton([37, 150, 601, 2500])
    F = _rhs_batch(w, 5)
    H = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_MIXED, **over)
    A, st = H.fit(F, rel_tol=1e-12)
    assert max(st["rel_residual"][:w.L]) <= 1e-12
    assert np.all(A[:, 2] == 0.0)
    for c in (0, 4):
        a, _ = H.fit(np.ascontiguousarray(F[:, c]), rel_tol=1e-12)
        assert rel(A[:, c], a) <= 1e-8, c
    ref = np.concatenate(oracle_fit(w, F[:, [0, 4]]))
    assert rel(A[:, 4], ref[:, 1]) <= 1e-8
    H.close()


def test_evaluate_rejects_queries_of_another_dimension():
    w = inputs.grid_hierarchy_small()
    H = ms.Hierarchy.from_workload(w, precision=ms.MS_PREC_FP64)
    alpha, _ = H.fit(w.f, rel_tol=1e-10)
    with pytest.raises(ms.MsError) as e:
        H.evaluate(alpha, inputs.query_grid(4, 3))
    assert e.value.status == ms.MS_ERR_ARG
    assert H.evaluate(alpha, inputs.query_grid(4, 2)).shape == (16,)
    H.close()
