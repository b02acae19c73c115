"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module only draws random numbers and builds plain configuration records;
it holds none of the method's arithmetic and imports neither the oracle nor the
library.  Every draw is seeded so that both sides see identical inputs.
"""
from __future__ import annotations

import numpy as np

PAPER = dict(J_par=10.0, J_perp=0.1, h=1.0, p=2.5, q=2.0, eta=1.0, dt=0.01, staggered=0.0)
T_C = 1.969


def angles(n_rep: int, Lx: int, Ly: int, seed: int, lo=-np.pi / 2, hi=np.pi / 2) -> np.ndarray:
    """float32 angles uniform in [lo, hi), shape (n_rep, Ly*Lx)."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(lo, hi, size=(n_rep, Ly * Lx)).astype(np.float32)
    # keep every value strictly inside [-pi/2, pi/2) in both precisions
    return np.clip(th, np.float32(-1.5707963), np.float32(1.5707962))


def velocities(n_rep: int, Lx: int, Ly: int, seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed + 7919)
    return (scale * rng.standard_normal(size=(n_rep, Ly * Lx))).astype(np.float32)


def spins_to_theta(spins: np.ndarray) -> np.ndarray:
    """Map a 0/1 spin field to float32 angles (+0.7 for 1, -0.7 for 0)."""
    return np.where(np.asarray(spins) > 0, np.float32(0.7), np.float32(-0.7)).astype(np.float32)


def random_spins(Lx: int, Ly: int, seed: int, p_up: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.random((Ly, Lx)) < p_up).astype(np.int8)


def stripes(Lx: int, Ly: int, width: int, axis: int) -> np.ndarray:
    yy, xx = np.mgrid[0:Ly, 0:Lx]
    c = xx if axis == 0 else yy
    return ((c // width) % 2).astype(np.int8)


def checkerboard(Lx: int, Ly: int) -> np.ndarray:
    yy, xx = np.mgrid[0:Ly, 0:Lx]
    return ((xx + yy) % 2).astype(np.int8)


def spiral(L: int) -> np.ndarray:
    """A one-site-wide rectangular spiral of up spins with a one-site gap
    between its turns: one long component that merges in the worst order for
    a naive union-find."""
    g = np.zeros((L, L), dtype=np.int8)
    dirs = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    x = y = d = 0
    g[0, 0] = 1
    while True:
        for _ in range(2):
            dx, dy = dirs[d]
            ax, ay, bx, by = x + dx, y + dy, x + 2 * dx, y + 2 * dy
            inside_a = 0 <= ax < L and 0 <= ay < L
            inside_b = 0 <= bx < L and 0 <= by < L
            if inside_a and g[ay, ax] == 0 and (not inside_b or g[by, bx] == 0):
                break
            d = (d + 1) % 4
        else:
            break
        x, y = ax, ay
        g[y, x] = 1
    return g


def config(Lx, Ly, n_rep, seed=1, init_mode=0, n_total=10**9, knots=None, field=None, couplings=None, **params):
    p = dict(PAPER)
    p.update(params)
    d = dict(Lx=Lx, Ly=Ly, n_rep=n_rep, seed=seed, init_mode=init_mode, params=p,
             knots=knots if knots is not None else ([0], [T_C]), n_total=n_total)
    if field is not None:
        d["field"] = field
    if couplings is not None:
        d["couplings"] = couplings
    return d


def ar1_field(Lx: int, Ly: int, rho: float, seed: int, axis: int = 1) -> np.ndarray:
    """float64 angles whose rows (axis=1) or columns (axis=0) are periodic AR(1)
    sequences with unit variance and lag-one correlation rho: a field with
    exponentially decaying correlations along one axis (length -1/ln rho)."""
    rng = np.random.default_rng(seed)
    n_lines, n = (Ly, Lx) if axis == 1 else (Lx, Ly)
    # periodic AR(1): circular filter of white noise with the spectrum of the AR(1) process
    w = rng.standard_normal((n_lines, n))
    k = np.arange(n)
    H = np.sqrt(1 - rho ** 2) / (1 - rho * np.exp(-2j * np.pi * k / n))
    z = np.fft.ifft(np.fft.fft(w, axis=1) * H, axis=1).real
    return z if axis == 1 else z.T


def ar1_series(n: int, phi: float, seed: int, n_series: int = 1) -> np.ndarray:
    """(n_series, n) stationary AR(1) series x_{t+1} = phi x_t + sqrt(1 - phi^2) w_t
    with unit variance (float64)."""
    rng = np.random.default_rng(seed)
    x = np.empty((n_series, n))
    x[:, 0] = rng.standard_normal(n_series)
    w = rng.standard_normal((n_series, n))
    s = np.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + s * w[:, t]
    return x
