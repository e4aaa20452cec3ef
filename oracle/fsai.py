"""CPU FP64 oracle of the learned factorised sparse-approximate-inverse preconditioner.

TEST INFRASTRUCTURE ONLY (imported by the tests and the benchmark's CPU leg, never by
the library).  Plain numpy, FP64, loops over points; shares no code with the CUDA path.

The paper has no preconditioner; this part restates the extension the library
adds to the per-level CG of Theorem 8.  It relies on the locality of A_l^{-1}
(Lemma 5: the entries of A_l^{-1}, and the cardinal functions, decay
exponentially) and on the scaling of eq. kernelscaling.

Definitions (all per level l, points X_l in input order, delta = delta_l, d = dimension):
  * pattern  P_i = {i} + the (up to) K = 16 nearest points j of the same level with
    |x_j - x_i| < delta and input index j < i, ordered by distance, ties by index.
  * exact weights (factorised sparse approximate inverse, Kolotilina-Yeremin):
    g_i = A_P^{-1} e_1 / sqrt(e_1^T A_P^{-1} e_1), A_P = Phi_delta(X_P, X_P), self first;
    G is lower triangular in input order with row i = g_i on P_i, and M = G^T G ~ A^{-1}
    is symmetric positive definite for any G with a positive diagonal.
  * scale-free weights  ghat_i = delta^{-d/2} g_i: since A_P = delta^{-d} K(offsets/delta),
    ghat depends only on the delta-scaled offsets (x_j - x_i)/delta.
  * features  z_i in R^{K d}: the scaled offsets o_k = (x_{n_k} - x_i)/delta of the pattern's
    neighbours in pattern order, zero-padded when fewer than K exist, written in the point's
    canonical frame (canonical_frame below).  The kernel is radial, so A_P, and with it the
    exact row, is unchanged by rotating or reflecting the patch: expressing the offsets in a
    frame fixed by the patch itself removes those d(d-1)/2 + 1 nuisance directions from the
    network's input (measured on the oracle: a network trained on levels 1-4 needs 80 instead
    of 130 PCG iterations on level 5, exact rows 13).
  * network   o = W3 relu(W2 relu(W1 z + b1) + b2) + b3  (hidden width 64, 17 m outputs): m
    candidate rows, u_1 = mu + sigma * o[0:17] (the standardised row, per-entry mean mu and
    deviation sigma of the training targets) and u_k = sigma * o[17 (k-1) : 17 k] for k > 1
    (corrections around it), the outputs of missing neighbours set to zero.
  * row       the factorised-sparse-approximate-inverse row within the span of the candidates
    (combine below): the exact row minimises g^T K g subject to g_self = 1, so restricted to
    g = U c (U = [u_1 .. u_m], K the scaled patch matrix) the minimiser is
    g = U y / sqrt(q), y = S_r^-1 U^T e_1, S = U^T K U, q = e_1^T U y, normalised to g^T K g = 1
    (the value the exact row has, which is (G A G^T)_ii = 1) with g_self = sqrt(q) > 0.  S_r =
    S + 1e-6 diag(S) (a ridge relative to each candidate's own energy: the candidates may be
    nearly dependent in the K metric).  With m = 1 this is the candidate rescaled to unit
    energy; with the exact row in the span it is the exact row.  A patch of n <= m points is
    spanned by any m generic candidates, so its row is the exact row itself (no ridge).
  * loss      the Kaporin-type gap of the row: (1/S) sum_s (log q*_s - log q_s), q* = (K^-1)_11 =
              ghat*_self^2 the value of the exact row.  q <= q* because the exact row maximises
              g_self over g^T K g = 1, so the loss is >= 0 and vanishes exactly when the exact row
              lies in the candidates' span; it does not depend on the scale of the candidates,
              so the network learns a subspace, and the combination is solved exactly per row.
  * Adam      beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.
  * training set  the patches of every point of the training levels, plus R extra patches per
    point: for draw r the patch of point i takes the K nearest points j != i within delta
    among the level's first p points, p = augment_bounds(n, u) for uniform draws u (a
    patch point i would have had if p points had preceded it).  Patch radii then span the
    same range, in units of delta, as the patterns of every level, and the network sees
    (1 + R) times as many geometries of the same training levels (measured on the oracle,
    levels 1-4 to level 5: 82 learned-PCG iterations without them, 49 with R = 4; exact
    rows 16).

Parity: pinned by tests/test_oracle_fsai.py (FSAI identities (G A)_{i,P_i\\{i}} = 0 and
(G A G^T)_ii = 1, scale invariance of ghat, gradients against central differences, PCG
convergence).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import multiscale as om

K_NEIGH = 16
HIDDEN = 64
N_OUT = K_NEIGH + 1


# ----------------------------------------------------------------------------- pattern


def pattern(X: np.ndarray, delta: float, K: int = K_NEIGH):
    """For every point i, the list of its pattern neighbours (input indices), nearest first."""
    n = len(X)
    out = []
    for i in range(n):
        if i == 0:
            out.append(np.zeros(0, dtype=np.int64))
            continue
        d = np.sqrt(np.sum((X[:i] - X[i]) ** 2, axis=1))
        cand = np.nonzero(d < delta)[0]
        order = np.lexsort((cand, d[cand]))  # by distance, then index
        out.append(cand[order][:K].astype(np.int64))
    return out


# ----------------------------------------------------------------------------- exact weights


def prefix_pattern(X: np.ndarray, delta: float, i: int, p: int, K: int = K_NEIGH):
    """The (up to) K nearest points j != i among the first p points of X with |x_j - x_i| < delta,
    nearest first, ties by index.  p = i gives the pattern of point i; p > i gives an extra
    training patch of the same level (the patch point i would have if the level's first p
    points preceded it)."""
    d = np.sqrt(np.sum((X[:p] - X[i]) ** 2, axis=1))
    d[i:i + 1] = np.inf
    cand = np.nonzero(d < delta)[0]
    order = np.lexsort((cand, d[cand]))
    return cand[order][:K].astype(np.int64)


def augment_bounds(n: int, u: np.ndarray) -> np.ndarray:
    """Prefix lengths p_i = i + 1 + floor(u_i (n - i)), capped at n, of the extra training patches
    of points i = 0..n-1 of a level of n points, from uniform draws u_i in [0, 1)."""
    i = np.arange(n)
    m = n - i
    return i + 1 + np.minimum(np.floor(u * m), m - 1).astype(np.int64)


def exact_weights(X: np.ndarray, delta: float, wd: int, wk: int, pat, selfs=None):
    """Rows g_i (self first) of the factorised sparse approximate inverse; selfs[s] is the
    centre of patch s (default: patch s is centred on point s)."""
    rows = []
    for s, nb in enumerate(pat):
        i = s if selfs is None else selfs[s]
        P = np.concatenate([[i], nb])
        AP = om.kernel_dense(X[P], X[P], delta, wd, wk)
        e1 = np.zeros(len(P))
        e1[0] = 1.0
        z = sla.solve(AP, e1, assume_a="pos")
        rows.append(z / math.sqrt(z[0]))
    return rows


def scale_free(rows, delta: float, d: int):
    return [r * delta ** (-0.5 * d) for r in rows]


def G_matrix(rows, pat, n):
    G = np.zeros((n, n))
    for i, (r, nb) in enumerate(zip(rows, pat)):
        G[i, i] = r[0]
        G[i, nb] = r[1:]
    return G


def canonical_frame(off: np.ndarray) -> np.ndarray:
    """Orthonormal rows e_1..e_d fixed by the (nearest-first) offsets off[m, d]:
    e_1 = o_1/|o_1|; e_2 from o_2 by Gram-Schmidt (d = 3), or the perpendicular of e_1 (d = 2);
    e_3 = e_1 x e_2; the last axis is flipped so that o_d has a non-negative coordinate on it
    (d = 1: the sign that makes o_1 positive).  Missing or degenerate offsets fall back to the
    coordinate axes: no offsets -> identity; o_2 parallel to o_1 (d = 3) -> e_2 from the
    coordinate axis least aligned with e_1."""
    m, d = off.shape
    E = np.eye(d)
    if m == 0 or not np.any(off[0]):
        return E
    e1 = off[0] / np.linalg.norm(off[0])
    if d == 1:
        return np.array([[1.0 if off[0, 0] >= 0 else -1.0]])
    if d == 2:
        e2 = np.array([-e1[1], e1[0]])
        if m >= 2 and off[1] @ e2 < 0:
            e2 = -e2
        return np.stack([e1, e2])
    w = off[1] - (off[1] @ e1) * e1 if m >= 2 else np.zeros(3)
    if m >= 2 and np.linalg.norm(w) > 1e-9 * np.linalg.norm(off[1]):
        e2 = w / np.linalg.norm(w)
    else:
        a = int(np.argmin(np.abs(e1)))
        u = np.eye(3)[a]
        e2 = u - (u @ e1) * e1
        e2 /= np.linalg.norm(e2)
    e3 = np.cross(e1, e2)
    if m >= 3 and off[2] @ e3 < 0:
        e3 = -e3
    return np.stack([e1, e2, e3])


def features(X: np.ndarray, delta: float, pat, K: int = K_NEIGH, selfs=None):
    d = X.shape[1]
    Z = np.zeros((len(pat), K * d))
    for s, nb in enumerate(pat):
        i = s if selfs is None else selfs[s]
        off = (X[nb] - X[i]) / delta
        Z[s, :len(nb) * d] = (off @ canonical_frame(off).T).ravel()
    return Z


def target_matrix(ghat_rows, pat):
    """[n, 17] scale-free targets and the validity mask (self always valid)."""
    n = len(pat)
    T = np.zeros((n, N_OUT))
    Mk = np.zeros((n, N_OUT))
    for i, (r, nb) in enumerate(zip(ghat_rows, pat)):
        T[i, :len(r)] = r
        Mk[i, :len(r)] = 1.0
    return T, Mk


# ----------------------------------------------------------------------------- network


def param_shapes(n_in: int, m: int = 1):
    return [(HIDDEN, n_in), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (m * N_OUT, HIDDEN), (m * N_OUT,)]


def unpack(theta: np.ndarray, n_in: int, m: int = 1):
    out, o = [], 0
    for s in param_shapes(n_in, m):
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def n_params(n_in: int, m: int = 1) -> int:
    return sum(int(np.prod(s)) for s in param_shapes(n_in, m))


def init_params(n_in: int, seed: int, m: int = 1) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for every weight and bias of a layer, drawn
    from SplitMix64(seed) in parameter order (W1, b1, W2, b2, W3, b3)."""
    from paper_2503_04914_gb300.inputs import uniform01
    u = uniform01(seed, n_params(n_in, m))
    theta = np.empty(n_params(n_in, m))
    o = 0
    for s, fan in zip(param_shapes(n_in, m), [n_in, n_in, HIDDEN, HIDDEN, HIDDEN, HIDDEN]):
        k = int(np.prod(s))
        b = 1.0 / math.sqrt(fan)
        theta[o:o + k] = -b + 2.0 * b * u[o:o + k]
        o += k
    return theta


def forward(theta, Z, n_in, m: int = 1):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, m)
    a1 = Z @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    o = h2 @ W3.T + b3
    return o, (a1, h1, a2, h2)


def patch_matrices(X: np.ndarray, delta: float, wd: int, wk: int, pat, selfs=None):
    """[n, 17, 17] scaled patch matrices K_i = phi(|x_a - x_b| / delta) on P_i (self first), zero-padded."""
    Ks = np.zeros((len(pat), N_OUT, N_OUT))
    d = X.shape[1]
    for s, nb in enumerate(pat):
        i = s if selfs is None else selfs[s]
        P = np.concatenate([[i], nb])
        m = len(P)
        Ks[s, :m, :m] = om.kernel_dense(X[P], X[P], delta, wd, wk) * delta ** d
    return Ks


RIDGE = 1e-6  # ridge of S = U^T K U, relative to each diagonal entry


def candidate_rows(o, mu, sig, Mk, m):
    """U[s, a, k]: candidate k of sample s, entry a; u_1 = mu + sig o_1, u_k = sig o_k (k > 1),
    zero past the patch."""
    S = len(o)
    U = sig[None, :, None] * o.reshape(S, m, N_OUT).transpose(0, 2, 1)
    U[:, :, 0] += mu[None, :]
    return U * Mk[:, :, None]


def combine(U, K, n):
    """The FSAI row of one patch of n points within span(U) (U [17, m], K [17, 17] the scaled
    patch matrix): g = U y / sqrt(q) with y = (S + RIDGE diag(S))^-1 U^T e_1, S = U^T K U,
    q = e_1^T U y.  For n <= m the exact row K_n^-1 e_1 / sqrt((K_n^-1)_11).  Returns (g, q, y)
    (y = None for the exact row); g = e_1 / sqrt(K_11) when q <= 0 (no candidate has a self entry)."""
    m = U.shape[1]
    if n <= m:
        e = np.zeros(n)
        e[0] = 1.0
        z = sla.solve(K[:n, :n], e, assume_a="pos")
        g = np.zeros(U.shape[0])
        g[:n] = z / math.sqrt(z[0])
        return g, float(z[0]), None
    S = U.T @ K @ U
    y = np.linalg.solve(S + RIDGE * np.diag(np.diag(S)), U[0])
    q = float(U[0] @ y)
    if not q > 0.0:
        g = np.zeros(U.shape[0])
        g[0] = 1.0 / math.sqrt(K[0, 0])
        return g, 0.0, y
    return (U @ y) / math.sqrt(q), q, y


def exact_q(Ks, Mk):
    """q* = (K^-1)_11 of every sample (the exact row's g_self^2 at unit energy)."""
    out = np.empty(len(Ks))
    for s in range(len(Ks)):
        n = int(Mk[s].sum())
        e = np.zeros(n)
        e[0] = 1.0
        out[s] = sla.solve(Ks[s][:n, :n], e, assume_a="pos")[0]
    return out


def loss(theta, Z, Mk, Ks, qstar, mu, sig, n_in, m=1):
    """Mean Kaporin-type gap (log q* - log q) of the rows the network's candidates give."""
    o, _ = forward(theta, Z, n_in, m)
    U = candidate_rows(o, mu, sig, Mk, m)
    tot = 0.0
    for s in range(len(Z)):
        _, q, _ = combine(U[s], Ks[s], int(Mk[s].sum()))
        tot += math.log(qstar[s]) - math.log(max(q, 1e-300))
    return tot / len(Z)


def grad(theta, Z, Mk, Ks, qstar, mu, sig, n_in, m=1):
    """Analytic gradient of loss().  For one sample of more than m points, with S, y, q as in
    combine, r = e_1 - K U y and the ridge's own dependence on U:
    dq/dU = 2 r y^T - 2 RIDGE (K U) diag(y)^2, and d(-log q)/dU = -(dq/dU) / q (patches of n <= m
    points take the exact row: no dependence on U); then backpropagation through the candidate
    map and the three layers."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, m)
    o, (a1, h1, a2, h2) = forward(theta, Z, n_in, m)
    U = candidate_rows(o, mu, sig, Mk, m)
    S = len(Z)
    dU = np.zeros_like(U)
    for s in range(S):
        K = Ks[s]
        _, q, y = combine(U[s], K, int(Mk[s].sum()))
        if y is None or not q > 0.0:
            continue
        KU = K @ U[s]
        r = -K @ (U[s] @ y)
        r[0] += 1.0
        dq = 2.0 * np.outer(r, y) - 2.0 * RIDGE * KU * (y * y)[None, :]
        dU[s] = -dq / q / S
    e = (dU * sig[None, :, None] * Mk[:, :, None]).transpose(0, 2, 1).reshape(S, m * N_OUT)
    gW3 = e.T @ h2
    gb3 = e.sum(0)
    d2 = (e @ W3) * (a2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ Z
    gb1 = d1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def standardise(T, Mk):
    """Per-output mean and standard deviation over the valid targets."""
    cnt = np.maximum(Mk.sum(0), 1.0)
    mu = (T * Mk).sum(0) / cnt
    var = (((T - mu) * Mk) ** 2).sum(0) / cnt
    sig = np.sqrt(np.maximum(var, 1e-30))
    return mu, sig


def predict_rows(theta, Z, pat, mu, sig, n_in, Ks, m=1):
    """Scale-free rows predicted by the network (self first): the combination of its m
    candidate rows that the FSAI criterion selects in their span (combine), g^T K g = 1."""
    o, _ = forward(theta, Z, n_in, m)
    Mk = np.zeros((len(pat), N_OUT))
    for i, nb in enumerate(pat):
        Mk[i, :1 + len(nb)] = 1.0
    U = candidate_rows(o, mu, sig, Mk, m)
    rows = []
    for i, nb in enumerate(pat):
        g, _, _ = combine(U[i], Ks[i], 1 + len(nb))
        rows.append(g[:1 + len(nb)].copy())
    return rows


# ----------------------------------------------------------------------------- PCG


def pcg(A, b, G=None, tol=1e-10, maxiter=100000):
    """CG on A x = b, preconditioned with M = G^T G when G is given; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = G.T @ (G @ r) if G is not None else r.copy()
    p = z.copy()
    rz = float(r @ z)
    bn = float(np.linalg.norm(b))
    for it in range(maxiter):
        q = A @ p
        a = rz / float(p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * bn:
            return x, it + 1
        z = G.T @ (G @ r) if G is not None else r
        rz2 = float(r @ z)
        p = z + (rz2 / rz) * p
        rz = rz2
    return x, maxiter
