"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module draws random numbers only (numpy PCG64); it holds none of the
method's arithmetic.  Every workload below is shaped like the paper's runs
(35 moments, 1D normal shocks up to Mach 10).
"""
from dataclasses import dataclass

import numpy as np

NP = 35
GAMMA = 5.0 / 3.0
PR = 2.0 / 3.0


@dataclass
class SolveTargets:
    """Raw parameters of the standalone-solve workload, one row per cell.

    Each cell's distribution is exp(-|c|^2/2 + sum a_k c^k - sum b_k c^k) in
    c = (u - v)/sqrt(T), density 1: v ~ N(0, 3^2) per component, T ~
    logU[0.5, 20], 10 cubic coefficients a ~ N(0, 0.05^2), 6 even quartic
    coefficients b ~ U(0.01, 0.1) (the odd quartic terms are zero, so the
    quartic part is negative definite).  The cubic coefficients follow the
    order of the degree-3 statistics: (3,0,0), (2,1,0), (2,0,1), (1,2,0),
    (1,1,1), (1,0,2), (0,3,0), (0,2,1), (0,1,2), (0,0,3).
    """
    v: np.ndarray   # [B, 3]
    T: np.ndarray   # [B]
    a: np.ndarray   # [B, 10]
    b: np.ndarray   # [B, 6]
    redrawn: int = 0            # cells whose first (a, b) draw had a second mode
    bimodal: np.ndarray = None  # redraw=False: mask of the cells with a second mode


_CUBIC = [(3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]
_QUART = [(4, 0, 0), (0, 4, 0), (0, 0, 4), (2, 2, 0), (2, 0, 2), (0, 2, 2)]


def _directions(n_random: int = 256, seed: int = 12345) -> np.ndarray:
    """Fixed unit directions: the 26 lattice directions plus seeded random ones."""
    d = [np.array([i, j, k], float) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1) if (i, j, k) != (0, 0, 0)]
    rng = np.random.Generator(np.random.PCG64(seed))
    d += list(rng.normal(size=(n_random, 3)))
    d = np.array(d)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _unimodal(a: np.ndarray, b: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """True where -t^2/2 + C(e) t^3 - Q(e) t^4 decreases for t > 0 along every
    direction e, i.e. 9 C(e)^2 < 16 Q(e) (no second mode)."""
    mono3 = np.stack([np.prod(dirs ** np.array(k), axis=1) for k in _CUBIC], axis=1)   # [D, 10]
    mono4 = np.stack([np.prod(dirs ** np.array(k), axis=1) for k in _QUART], axis=1)   # [D, 6]
    C = a @ mono3.T
    Q = b @ mono4.T
    return (9.0 * C * C < 16.0 * Q).all(axis=1)


def solve_targets(B: int, seed: int = 0, v_sigma: float = 3.0, a_sigma: float = 0.05,
                  b_lo: float = 0.01, b_hi: float = 0.1, redraw: bool = True) -> SolveTargets:
    """Cells whose density would have a second mode (checked along fixed
    directions) get their (a, b) redrawn until unimodal (redraw=True; the
    count is kept in `redrawn`); redraw=False returns the draws as they come
    and marks the bimodal ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(0.0, v_sigma, size=(B, 3))
    T = np.exp(rng.uniform(np.log(0.5), np.log(20.0), size=B))
    a = rng.normal(0.0, a_sigma, size=(B, 10))
    b = rng.uniform(b_lo, b_hi, size=(B, 6))
    dirs = _directions()
    first = ~_unimodal(a, b, dirs)
    if not redraw:
        return SolveTargets(v=v, T=T, a=a, b=b, redrawn=0, bimodal=first)
    bad = first
    for _ in range(200):
        nb = int(bad.sum())
        if nb == 0:
            break
        a[bad] = rng.normal(0.0, a_sigma, size=(nb, 10))
        b[bad] = rng.uniform(b_lo, b_hi, size=(nb, 6))
        bad = ~_unimodal(a, b, dirs)
    return SolveTargets(v=v, T=T, a=a, b=b, redrawn=int(first.sum()))


def perturbed_hermite_moments(B: int, seed: int = 0, scale: float = 0.05) -> np.ndarray:
    """Moments e_0 + eps in a Hermite gauge: density 1, zero degree-1 and zero
    diagonal degree-2 entries, N(0, scale^2) noise on the other 28 entries.
    Index k of the statistic (a, b, c) follows the library order (total
    degree, then a descending, then b descending)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = np.zeros((B, NP))
    M[:, 0] = 1.0
    noise = rng.normal(0.0, scale, size=(B, NP))
    keep = np.ones(NP, dtype=bool)
    keep[[0, 1, 2, 3, 4, 7, 9]] = False   # e0, e_x, e_y, e_z, (2,0,0), (0,2,0), (0,0,2)
    M[:, keep] += noise[:, keep]
    return M


@dataclass
class ShockProblem:
    mach: float
    ncells: int
    xl: float
    xr: float


def ensemble_problems(nprob: int = 256, seed: int = 1, lo: int = 256, hi: int = 16384,
                      mach_lo: float = 1.2, mach_hi: float = 10.0, dx: float = 0.628):
    """Batched-ensemble workload: cell counts log-uniform, Mach uniform, domain
    = ncells * dx centred on 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nprob))).astype(int)
    ma = rng.uniform(mach_lo, mach_hi, size=nprob)
    return [ShockProblem(float(m), int(n), -0.5 * n * dx, 0.5 * n * dx) for m, n in zip(ma, nc)]


def serving_trace(nreq: int = 512, seed: int = 2, rate: float = 200.0, lo: int = 128, hi: int = 32768,
                  mach_lo: float = 1.5, mach_hi: float = 10.0, dx: float = 0.628):
    """Poisson arrivals (mean `rate` per second) of shock solves."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=nreq)
    t = np.cumsum(gaps)
    nc = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nreq))).astype(int)
    ma = rng.uniform(mach_lo, mach_hi, size=nreq)
    return t, [ShockProblem(float(m), int(n), -0.5 * n * dx, 0.5 * n * dx) for m, n in zip(ma, nc)]
