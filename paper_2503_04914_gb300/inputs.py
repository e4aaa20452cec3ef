"""Seeded synthetic inputs for the multiscale fit: point hierarchies and data values.

This module holds no arithmetic of the multiscale method itself (no kernel,
no matrix, no solve).  It only produces the inputs the method is applied to:

* point sets X_1..X_L per level (regular grids, scrambled Halton, uniform random),
* the nominal level spacings h_1..h_L the workload recipe prescribes,
* data values f on those points (Gaussian mixtures, the Franke function of
  the paper's Section 5, eq. Franke).

Both the CPU oracle and the CUDA path consume these arrays, so both sides see
bit-identical inputs.  All randomness comes from SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: draw i of a stream with seed s is mix(s + (i+1)*gamma).

Layout convention: points of all levels are concatenated level by level
(level 1 first) into one float64 array of shape [N, d], row-major.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# SplitMix64 constants (the published definition).
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

BASE_SEED = 2503049140


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start..start+n-1 of the SplitMix64 stream with the given seed (uint64)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 draw times 2^-53."""
    z = splitmix64(seed, n, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------

def grid_points(n_side: int, d: int = 2) -> np.ndarray:
    """Regular grid of n_side^d points on [0,1]^d (spacing 1/(n_side-1)), row-major."""
    g = np.linspace(0.0, 1.0, n_side)
    mesh = np.meshgrid(*([g] * d), indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


_PRIMES = (2, 3, 5, 7, 11, 13)


def _digit_count(base: int) -> int:
    # enough digits that base^-D is below double resolution
    return int(math.ceil(53 * math.log(2) / math.log(base)))


def scrambled_halton(n: int, d: int, seed: int, start_index: int = 1) -> np.ndarray:
    """First n points of a scrambled Halton sequence in [0,1)^d.

    Bases are the first d primes.  Scrambling is a random permutation of the
    digit set {0..b-1} for every base b and every digit position p, drawn
    from SplitMix64(seed) (Fisher-Yates, consuming draws in the order
    base 0 position 0, base 0 position 1, ...).  All D_b digit positions
    (D_b = ceil(53 ln2 / ln b)) are permuted, leading zeros included, so the
    map from index to point is one-to-one.  Indices start at start_index (1 by
    default), so nested prefixes give nested point sets.
    """
    idx = np.arange(start_index, start_index + n, dtype=np.int64)
    out = np.empty((n, d), dtype=np.float64)
    draw = 0
    for axis in range(d):
        b = _PRIMES[axis]
        D = _digit_count(b)
        perms = []
        for _p in range(D):
            perm = list(range(b))
            for i in range(b - 1, 0, -1):  # Fisher-Yates
                u = int(splitmix64(seed, 1, draw)[0])
                draw += 1
                j = u % (i + 1)
                perm[i], perm[j] = perm[j], perm[i]
            perms.append(np.asarray(perm, dtype=np.int64))
        rem = idx.copy()
        val = np.zeros(n, dtype=np.float64)
        scale = 1.0 / b
        for p in range(D):
            digit = rem % b
            rem //= b
            val += perms[p][digit] * scale
            scale /= b
        out[:, axis] = val
    return out


def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1)^d from SplitMix64(seed), coordinates drawn point by point."""
    return uniform01(seed, n * d).reshape(n, d)


# ----------------------------------------------------------------------------
# data values
# ----------------------------------------------------------------------------

@dataclass
class GaussianMixture:
    """f(x) = sum_i a_i exp(-|x - c_i|^2 / (2 w_i^2)) (+ optional 0.1 sin(8 pi x) sin(8 pi y)).

    Drawn from SplitMix64(seed) in the order: all centres c (n*d draws, U[0,1)),
    then all widths w (n draws, U[0.05,0.3)), then all amplitudes a (n draws,
    U[-1,1)).
    """
    n: int
    d: int
    seed: int
    sine: bool = False
    c: np.ndarray = field(init=False)
    w: np.ndarray = field(init=False)
    a: np.ndarray = field(init=False)

    def __post_init__(self):
        u = uniform01(self.seed, self.n * self.d + 2 * self.n)
        self.c = u[: self.n * self.d].reshape(self.n, self.d)
        self.w = 0.05 + 0.25 * u[self.n * self.d: self.n * self.d + self.n]
        self.a = -1.0 + 2.0 * u[self.n * self.d + self.n:]

    def __call__(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(x.shape[0], dtype=np.float64)
        for i in range(self.n):
            r2 = np.sum((x - self.c[i]) ** 2, axis=1)
            out += self.a[i] * np.exp(-r2 / (2.0 * self.w[i] ** 2))
        if self.sine:
            out += 0.1 * np.sin(8 * np.pi * x[:, 0]) * np.sin(8 * np.pi * x[:, 1])
        return out


def franke(x: np.ndarray) -> np.ndarray:
    """The Franke test function as printed in Section 5 (eq. Franke), on [0,1]^2."""
    X = 9.0 * x[:, 0]
    Y = 9.0 * x[:, 1]
    return (0.75 * np.exp(-((X - 2) ** 2 + (Y - 2) ** 2) / 4.0)
            + 0.75 * np.exp(-((X + 1) ** 2) / 49.0 - (Y + 1) / 10.0)
            + 0.5 * np.exp(-((X - 7) ** 2 + (Y - 3) ** 2) / 4.0)
            - 0.2 * np.exp(-(X - 4) ** 2 - (Y - 7) ** 2))


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    """One synthetic hierarchy: points per level, nominal spacings, kernel choice, data."""
    name: str
    d: int
    levels: list            # list of [N_l, d] float64 arrays, coarse to fine
    h: np.ndarray           # nominal spacing h_l per level (delta_l = nu * h_l)
    nu: float
    wendland_d: int
    wendland_k: int
    f: np.ndarray           # [N] or [N, nrhs] data values, level-concatenated
    f_fun: object = None    # callable giving f at arbitrary points (first RHS)

    @property
    def n_per_level(self) -> np.ndarray:
        return np.array([len(x) for x in self.levels], dtype=np.int64)

    @property
    def points(self) -> np.ndarray:
        return np.ascontiguousarray(np.concatenate(self.levels, axis=0))

    @property
    def N(self) -> int:
        return int(sum(len(x) for x in self.levels))

    @property
    def L(self) -> int:
        return len(self.levels)


def _seed(cfg_index: int) -> int:
    return BASE_SEED + cfg_index


def grid_hierarchy_small(nrhs: int = 1) -> Workload:
    """d=2 unit square, 4 levels of uniform grids 5^2, 9^2, 17^2, 33^2 (h_j = 2^-(j+1)),
    Wendland phi_{2,1}, nu = 3, f = sum of 5 seeded Gaussians."""
    levels = [grid_points(2 ** (j + 1) + 1, 2) for j in range(1, 5)]
    h = np.array([2.0 ** -(j + 1) for j in range(1, 5)])
    s = _seed(0)
    funs = [GaussianMixture(5, 2, s + 1000 * r) for r in range(nrhs)]
    pts = np.concatenate(levels)
    f = np.stack([g(pts) for g in funs], axis=1)
    return Workload("grid4_d2_nu3_w21", 2, levels, h, 3.0, 2, 1,
                    f[:, 0] if nrhs == 1 else f, funs[0])


def halton_hierarchy(L: int = 8, nu: float = 4.0, wendland=(2, 1), n_gauss: int = 20,
                     sine: bool = True, cfg_index: int = 1, n0: int = 64, nrhs: int = 1) -> Workload:
    """d=2 scrambled Halton points, N_j = n0 * 4^(j-1), nested prefixes of one sequence,
    h_j = N_j^-1/2, delta_j = nu h_j.  f = Gaussian mixture (+ 0.1 sin(8 pi x) sin(8 pi y))."""
    s = _seed(cfg_index)
    ns = [n0 * 4 ** j for j in range(L)]
    allpts = scrambled_halton(ns[-1], 2, s)
    levels = [np.ascontiguousarray(allpts[:n]) for n in ns]
    h = np.array([n ** -0.5 for n in ns])
    funs = [GaussianMixture(n_gauss, 2, s + 1000 * (r + 1), sine=sine) for r in range(nrhs)]
    pts = np.concatenate(levels)
    f = np.stack([g(pts) for g in funs], axis=1)
    name = f"halton{L}_d2_nu{nu:g}_w{wendland[0]}{wendland[1]}"
    return Workload(name, 2, levels, h, nu, wendland[0], wendland[1],
                    f[:, 0] if nrhs == 1 else f, funs[0])


def random3d_hierarchy(L: int = 6, nu: float = 3.0, n_gauss: int = 30, cfg_index: int = 2,
                       n0: int = 125) -> Workload:
    """d=3 uniform random points in [0,1]^3, N_j = n0 * 8^(j-1), independent per level,
    h_j = N_j^-1/3, delta_j = nu h_j, Wendland phi_{3,1}, 30 seeded 3-D Gaussians."""
    s = _seed(cfg_index)
    ns = [n0 * 8 ** j for j in range(L)]
    levels = [uniform_points(n, 3, s + 17 * (j + 1)) for j, n in enumerate(ns)]
    h = np.array([n ** (-1.0 / 3.0) for n in ns])
    g = GaussianMixture(n_gauss, 3, s + 1000)
    f = g(np.concatenate(levels))
    return Workload(f"random{L}_d3_nu{nu:g}_w31", 3, levels, h, nu, 3, 1, f, g)


def franke_grid_hierarchy(L: int = 7) -> Workload:
    """The paper's own experiment (Section 5, Table 1): grids (2^l+1)^2, l = 1..L, on [0,1]^2,
    h_l = fill distance = 2^-l / sqrt(2), nu = 4, Wendland phi_{3,1}, Franke data."""
    levels = [grid_points(2 ** l + 1, 2) for l in range(1, L + 1)]
    h = np.array([2.0 ** -l / math.sqrt(2.0) for l in range(1, L + 1)])
    f = franke(np.concatenate(levels))
    return Workload(f"franke_grid{L}", 2, levels, h, 4.0, 3, 1, f, franke)


def batch_hierarchies(n_h: int = 64, cfg_index: int = 3, lmin: int = 3, lmax: int = 7,
                      finest_lo: int = 4096, finest_hi: int = 262144, nu: float = 4.0):
    """Many independent d=2 Halton hierarchies of uneven depth and size: L ~ U{lmin..lmax},
    finest N_L = round(exp(U[ln finest_lo, ln finest_hi])), N_j = ceil(N_L 4^(j-L)),
    each with its own seed and one Gaussian-mixture RHS."""
    s = _seed(cfg_index)
    u = uniform01(s, 2 * n_h)
    out = []
    for i in range(n_h):
        L = lmin + int(u[2 * i] * (lmax - lmin + 1))
        nL = int(round(math.exp(math.log(finest_lo) + u[2 * i + 1] * (math.log(finest_hi) - math.log(finest_lo)))))
        ns = [int(math.ceil(nL * 4.0 ** (j - L + 1))) for j in range(L)]
        si = s + 7919 * (i + 1)
        allpts = scrambled_halton(ns[-1], 2, si)
        levels = [np.ascontiguousarray(allpts[:n]) for n in ns]
        h = np.array([n ** -0.5 for n in ns])
        g = GaussianMixture(20, 2, si + 1)
        f = g(np.concatenate(levels))
        out.append(Workload(f"batch{i}_L{L}_n{nL}", 2, levels, h, nu, 2, 1, f, g))
    return out


def query_grid(n_side: int, d: int) -> np.ndarray:
    """Uniform query grid on [0,1]^d with n_side points per axis (cell centres)."""
    g = (np.arange(n_side) + 0.5) / n_side
    mesh = np.meshgrid(*([g] * d), indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def query_random(n: int, d: int, seed: int = 2503049199) -> np.ndarray:
    """n seeded uniform query points in [0,1)^d (axis a from SplitMix64 stream seed + a).  Unlike
    the cell centres of query_grid, they avoid the nodes of every dyadic grid, where an
    interpolant is exact."""
    return np.stack([uniform01(seed + a, n) for a in range(d)], axis=1)
