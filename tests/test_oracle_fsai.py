"""Pins of the preconditioner oracle (oracle/fsai.py) against identities and brute force."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import fsai as of
from oracle import multiscale as om
from paper_2503_04914_gb300 import inputs


def level(nu, wend, L):
    w = inputs.halton_hierarchy(L=L, nu=nu, wendland=wend, n_gauss=3)
    return w.levels[-1], nu * w.h[-1], wend


@pytest.mark.parametrize("nu,wend,L", [(4.0, (2, 1), 3), (8.0, (2, 2), 3)])
def test_fsai_identities(nu, wend, L):
    """Exact FSAI rows satisfy (G A)_{i,j} = 0 for j in P_i \\ {i} and (G A G^T)_ii = 1
    (they solve A_P g = e_1 / sqrt(c)); M = G^T G is SPD."""
    X, delta, (wd, wk) = level(nu, wend, L)
    pat = of.pattern(X, delta)
    rows = of.exact_weights(X, delta, wd, wk, pat)
    G = of.G_matrix(rows, pat, len(X))
    A = om.kernel_dense(X, X, delta, wd, wk)
    GA = G @ A
    scale = np.abs(G).max() * np.abs(A).max()
    for i, nb in enumerate(pat):
        assert np.all(np.abs(GA[i, nb]) <= 1e-9 * scale)
    np.testing.assert_allclose(np.diag(GA @ G.T), 1.0, rtol=1e-9)
    assert np.all(np.diag(G) > 0)
    assert np.all(np.triu(G, 1) == 0)  # lower triangular in input order
    assert np.linalg.eigvalsh(G.T @ G)[0] > 0


def test_pattern_brute_force():
    X, delta, _ = level(4.0, (2, 1), 3)
    pat = of.pattern(X, delta)
    tree = cKDTree(X)
    for i, nb in enumerate(pat):
        cand = [j for j in tree.query_ball_point(X[i], delta * (1 - 1e-12)) if j < i]
        assert len(nb) == min(16, len(cand))
        d = np.linalg.norm(X[nb] - X[i], axis=1)
        assert np.all(nb < i) and np.all(d < delta) and np.all(np.diff(d) >= 0)
        if len(cand) > 16:
            rest = sorted(set(cand) - set(nb.tolist()))
            assert np.min(np.linalg.norm(X[rest] - X[i], axis=1)) >= d[-1]


def test_prefix_patches():
    """Extra training patches: the prefix bound p = i gives the pattern; any p gives the 16
    nearest of the first p points other than i (checked with a k-d tree); the bounds drawn
    from uniform numbers lie in [i + 1, n], hit both ends, and u = 0 gives p = i + 1."""
    X, delta, _ = level(4.0, (2, 1), 3)
    n = len(X)
    pat = of.pattern(X, delta)
    rng = np.random.default_rng(3)
    for i in range(n):
        assert np.array_equal(of.prefix_pattern(X, delta, i, i), pat[i])
    for i in rng.integers(0, n, 60):
        p = int(rng.integers(i + 1, n + 1))
        nb = of.prefix_pattern(X, delta, i, p)
        tree = cKDTree(X[:p])
        cand = [j for j in tree.query_ball_point(X[i], delta * (1 - 1e-12)) if j != i]
        assert len(nb) == min(16, len(cand))
        d = np.linalg.norm(X[nb] - X[i], axis=1)
        assert np.all(nb < p) and np.all(nb != i) and np.all(d < delta) and np.all(np.diff(d) >= 0)
        if len(cand) > 16:
            rest = sorted(set(cand) - set(nb.tolist()))
            assert np.min(np.linalg.norm(X[rest] - X[i], axis=1)) >= d[-1]
    u = inputs.uniform01(inputs.BASE_SEED, n)
    b = of.augment_bounds(n, u)
    i = np.arange(n)
    assert np.all(b >= i + 1) and np.all(b <= n)
    assert np.array_equal(of.augment_bounds(n, np.zeros(n)), i + 1)
    assert np.array_equal(of.augment_bounds(n, np.full(n, np.nextafter(1.0, 0.0))), np.full(n, n))
    assert b[-1] == n


def test_scale_free_weights_are_level_independent():
    """ghat = delta^{-d/2} g depends only on the delta-scaled offsets (eq. kernelscaling)."""
    X, delta, (wd, wk) = level(8.0, (2, 2), 2)
    pat = of.pattern(X, delta)
    g1 = of.scale_free(of.exact_weights(X, delta, wd, wk, pat), delta, 2)
    c = 0.37
    g2 = of.scale_free(of.exact_weights(c * X + 0.1, c * delta, wd, wk, pat), c * delta, 2)
    for a, b in zip(g1, g2):
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10 * np.abs(a).max())


def test_exact_fsai_accelerates_cg():
    X, delta, (wd, wk) = level(4.0, (2, 1), 4)
    pat = of.pattern(X, delta)
    G = of.G_matrix(of.exact_weights(X, delta, wd, wk, pat), pat, len(X))
    A = om.kernel_sparse(X, X, delta, wd, wk)
    b = np.random.default_rng(0).standard_normal(len(X))
    x0, it0 = of.pcg(A, b)
    x1, it1 = of.pcg(A, b, G)
    assert it1 * 5 < it0
    assert np.linalg.norm(x1 - x0) <= 1e-7 * np.linalg.norm(x0)


def _training_data(nu, wend, L, lo, hi):
    X, delta, (wd, wk) = level(nu, wend, L)
    pat = of.pattern(X, delta)
    rows = of.scale_free(of.exact_weights(X, delta, wd, wk, pat), delta, 2)
    T, Mk = of.target_matrix(rows, pat)
    mu, sig = of.standardise(T, Mk)
    Ks = of.patch_matrices(X, delta, wd, wk, pat)[lo:hi]
    Z = of.features(X, delta, pat)[lo:hi]
    Mk = Mk[lo:hi]
    return Z, Mk, Ks, of.exact_q(Ks, Mk), mu, sig, [r for r in rows[lo:hi]]


@pytest.mark.parametrize("m", [1, 3])
def test_gradient_matches_central_differences(m):
    Z, Mk, Ks, qs, mu, sig, _ = _training_data(4.0, (2, 1), 2, 40, 64)
    n_in = Z.shape[1]
    th = of.init_params(n_in, 7, m)
    g = of.grad(th, Z, Mk, Ks, qs, mu, sig, n_in, m)
    rng = np.random.default_rng(1)
    for idx in rng.choice(len(th), 60, replace=False):
        h = 1e-6 * max(1.0, abs(th[idx]))
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (of.loss(tp, Z, Mk, Ks, qs, mu, sig, n_in, m) - of.loss(tm, Z, Mk, Ks, qs, mu, sig, n_in, m)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1e-6, np.abs(g).max()), (idx, fd, g[idx])


def test_exact_q_is_the_exact_rows_self_entry_squared():
    """q* = (K^-1)_11 equals ghat*_self^2 of the unit-energy exact row (two independent routes:
    a Cholesky solve of K, and the exact row computed from the unscaled kernel block)."""
    _, Mk, Ks, qs, _, _, rows = _training_data(8.0, (2, 2), 2, 0, 80)
    for s in range(1, 80):
        assert abs(qs[s] - rows[s][0] ** 2) <= 1e-9 * qs[s]


def test_combination_recovers_the_exact_row_in_its_span(monkeypatch):
    """The FSAI criterion restricted to span(U) gives the exact row whenever it lies in the span
    (for any scaling and mixing of the candidates), and the loss is then 0."""
    _, Mk, Ks, qs, _, _, rows = _training_data(8.0, (2, 2), 2, 0, 80)
    monkeypatch.setattr(of, "RIDGE", 0.0)
    rng = np.random.default_rng(3)
    for s in (10, 33, 71):
        n = int(Mk[s].sum())
        gs = np.zeros(17)
        gs[:n] = rows[s]
        U = np.stack([3.0 * gs] + [rng.standard_normal(17) * Mk[s] for _ in range(2)], axis=1)
        U = U @ rng.standard_normal((3, 3))  # mixed: the span is what counts
        assert n > 3
        g, q, _ = of.combine(U, Ks[s], n)
        assert np.max(np.abs(g - gs)) <= 1e-7 * np.max(np.abs(gs)), s
        assert abs(math.log(qs[s]) - math.log(q)) <= 1e-8


def test_combination_is_optimal_and_normalised_in_the_span():
    """g = combine(U, K, n) has g_self = sqrt(q) > 0 and unit energy less the ridge's shift
    (g^T K g = 1 - RIDGE sum_k S_kk y_k^2 / q), and no unit-energy vector of span(U) has a larger
    self entry (the FSAI criterion); q <= q* (Kaporin's bound), so the loss is >= 0; with m = 1
    it is the candidate rescaled to unit energy with a positive self entry; a patch of n <= m
    points gets the exact row."""
    _, Mk, Ks, qs, _, _, rows = _training_data(8.0, (2, 2), 2, 0, 80)
    rng = np.random.default_rng(5)
    tested = 0
    for s in range(1, 80, 3):
        K = Ks[s]
        n = int(Mk[s].sum())
        U = rng.standard_normal((17, 4)) * Mk[s][:, None]
        g, q, y = of.combine(U, K, n)
        assert g[0] > 0 and abs(g[0] ** 2 - q) <= 1e-9 * q
        if n <= 4:
            assert np.allclose(g[:n], rows[s], rtol=1e-9, atol=1e-12) and abs(q - qs[s]) <= 1e-9 * qs[s]
            continue
        tested += 1
        S = U.T @ K @ U
        assert abs(g @ K @ g - (1.0 - of.RIDGE * np.sum(np.diag(S) * y * y) / q)) <= 1e-9
        assert q <= qs[s] * (1 + 1e-12)
        for _ in range(20):
            v = U @ rng.standard_normal(4)
            v /= math.sqrt(v @ K @ v)
            assert abs(v[0]) <= g[0] * (1 + 1e-5)  # the 1e-6 ridge moves the optimum slightly
        u = U[:, :1]
        g1, _, _ = of.combine(u, K, n)
        ref = np.sign(u[0, 0]) * u[:, 0] / math.sqrt(u[:, 0] @ K @ u[:, 0])
        np.testing.assert_allclose(g1, ref, rtol=1e-5, atol=1e-12)
    assert tested >= 15


def test_loss_is_the_kaporin_gap_and_vanishes_only_at_the_span():
    """loss >= 0 for any parameters; the patch matrices are the oracle's kernel blocks scaled by
    delta^d."""
    X, delta, (wd, wk) = level(8.0, (2, 2), 2)
    pat = of.pattern(X, delta)
    Z, Mk, Ks, qs, mu, sig, _ = _training_data(8.0, (2, 2), 2, 0, len(pat))
    for m, seed in ((1, 1), (4, 2)):
        th = of.init_params(Z.shape[1], seed, m)
        assert of.loss(th, Z, Mk, Ks, qs, mu, sig, Z.shape[1], m) > 0.0
    P = np.concatenate([[60], pat[60]])
    np.testing.assert_allclose(Ks[60][:len(P), :len(P)],
                               om.kernel_dense(X[P], X[P], delta, wd, wk) * delta ** 2, rtol=1e-14)


def test_adam_first_step_is_a_signed_step():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th, m, v = of.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(th[:3], -0.01 * np.sign(g[:3]), rtol=1e-4)
    assert th[3] == 0.0


def test_init_is_uniform_in_fan_in_bounds():
    n_in = 32
    th = of.init_params(n_in, 3)
    parts = of.unpack(th, n_in)
    for p, fan in zip(parts, [32, 32, 64, 64, 64, 64]):
        assert np.abs(p).max() <= 1 / math.sqrt(fan)
        assert np.abs(p).max() >= 0.8 / math.sqrt(fan)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_features_are_invariant_under_rotations_and_reflections(d):
    """The network input is written in a frame fixed by the patch: rotating or reflecting the
    point set leaves the features unchanged, and so it does the exact rows (radial kernel)."""
    rng = np.random.default_rng(11 + d)
    n = {1: 40, 2: 300, 3: 600}[d]
    X = rng.random((n, d))
    delta = {1: 0.12, 2: 0.25, 3: 0.35}[d]
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    Q[:, 0] *= -1 if d > 1 else 1  # an improper orthogonal map for d > 1 (rotation + reflection)
    Xr = X @ Q.T + 0.3
    pat = of.pattern(X, delta)
    assert all(np.array_equal(a, b) for a, b in zip(pat, of.pattern(Xr, delta)))
    Z, Zr = of.features(X, delta, pat), of.features(Xr, delta, pat)
    assert np.max(np.abs(Z - Zr)) <= 1e-12
    w0 = of.exact_weights(X, delta, d, 1, pat)
    w1 = of.exact_weights(Xr, delta, d, 1, pat)
    # relative: 1-D patches of random points are ill-conditioned (large alternating rows)
    assert max(np.max(np.abs(a - b)) / np.max(np.abs(a)) for a, b in zip(w0, w1) if len(a)) <= 1e-8
    # the frame's defining properties: o_1 on the first axis, o_2's last (d=2) coordinate >= 0
    full = [i for i, p in enumerate(pat) if len(p) >= d]
    z = Z[full].reshape(len(full), -1, d)
    assert np.all(z[:, 0, 0] > 0) and np.allclose(z[:, 0, 1:], 0.0, atol=1e-14)
    assert np.all(z[:, d - 1, d - 1] >= -1e-14)
    # lengths are kept
    for i in full[:20]:
        off = (X[pat[i]] - X[i]) / delta
        assert np.allclose(np.linalg.norm(z[full.index(i)][:len(pat[i])], axis=1), np.linalg.norm(off, axis=1))


def test_predicted_rows_are_normalised_like_the_exact_rows():
    """Exact rows satisfy ghat^T K ghat = 1 ((G A G^T)_ii = 1); predicted rows (any m) do too,
    with a positive self entry, and a wider candidate span never does worse on the gap."""
    w = inputs.halton_hierarchy(L=3, nu=4.0, wendland=(2, 1), n_gauss=4)
    X, delta = w.levels[2], w.nu * w.h[2]
    pat = of.pattern(X, delta)
    rows = of.scale_free(of.exact_weights(X, delta, 2, 1, pat), delta, 2)
    Ks = of.patch_matrices(X, delta, 2, 1, pat)
    for i, r in enumerate(rows):
        m = len(r)
        assert abs(r @ Ks[i][:m, :m] @ r - 1.0) <= 1e-9
    Z = of.features(X, delta, pat)
    T, Mk = of.target_matrix(rows, pat)
    mu, sig = of.standardise(T, Mk)
    for m in (1, 4):
        th = of.init_params(32, 3, m)
        pr = of.predict_rows(th, Z, pat, mu, sig, 32, Ks, m)
        for i, r in enumerate(pr):
            n = len(r)
            # unit energy less the 1e-6 ridge's shift rho |y|^2 / q (pinned exactly above; largest
            # where m exceeds the patch size and the candidates are dependent)
            e = r @ Ks[i][:n, :n] @ r
            assert 1.0 - 1e-3 <= e <= 1.0 + 1e-12 and r[0] > 0
    # candidates [u, v]: the gap of their span is at most that of u alone
    th1 = of.init_params(32, 3, 1)
    o1, _ = of.forward(th1, Z, 32, 1)
    o2 = np.concatenate([o1, np.random.default_rng(0).standard_normal(o1.shape)], axis=1)
    U1, U2 = of.candidate_rows(o1, mu, sig, Mk, 1), of.candidate_rows(o2, mu, sig, Mk, 2)
    for i in range(1, len(pat), 13):
        n = 1 + len(pat[i])
        assert of.combine(U2[i], Ks[i], n)[1] >= of.combine(U1[i], Ks[i], n)[1] * (1 - 1e-5)
