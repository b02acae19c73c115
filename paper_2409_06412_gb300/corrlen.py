"""Correlation length from the structure factor (arXiv 2409.06412, Sec. VI).

Near k = 0 the structure factor of exponentially decaying correlations is a
Lorentzian (Eq. Lorentzian-Peak), S(k) = a / (1 + (2 pi xi k / N)^2) with k the
DFT index and N the lattice extent in that direction; below T_c the k = 0
value carries a delta peak from the constant part of C(r) and is left out of
the fit window.  This module fits (a, xi) on the host: the structure factors
themselves come from the GPU (``Lattice.structure_factor``), averaged over
replicas by the caller.

The fit linearises 1 / S = 1/a + (4 pi^2 xi^2 / (a N^2)) k^2, solves it by
least squares weighted with S^2 (so that it approximates least squares on S
itself), then polishes (a, xi) with Gauss-Newton steps on the residuals
S(k) - a / (1 + b k^2).
"""
from __future__ import annotations

import math

import numpy as np


def fit_lorentzian(S, N: int, k_lo: int = 1, k_hi: int = 8, iters: int = 50):
    """Fit S[k_lo..k_hi] to a / (1 + (2 pi xi k / N)^2).  Returns (a, xi);
    xi = 0 when the window shows no decay (S not decreasing in k^2)."""
    k = np.arange(k_lo, k_hi + 1, dtype=np.float64)
    y = np.asarray(S, dtype=np.float64)[k_lo:k_hi + 1]
    if k.size < 2 or np.any(y <= 0):
        raise ValueError("need at least two positive values in the fit window")
    k2 = k * k
    w = y * y
    A = np.stack([np.ones_like(k2), k2], axis=1) * w[:, None]
    alpha, beta = np.linalg.lstsq(A, w / y, rcond=None)[0]
    if alpha <= 0 or beta <= 0:
        return float(y[0]), 0.0
    a, b = 1.0 / alpha, beta / alpha  # S = a / (1 + b k^2)
    for _ in range(iters):
        d = 1.0 + b * k2
        r = y - a / d
        J = np.stack([1.0 / d, -a * k2 / (d * d)], axis=1)
        step = np.linalg.lstsq(J, r, rcond=None)[0]
        a, b = a + step[0], max(b + step[1], 1e-300)
        if np.max(np.abs(step) / np.maximum(np.abs([a, b]), 1e-300)) < 1e-15:
            break
    return float(a), float(math.sqrt(b) * N / (2.0 * math.pi))


def correlation_lengths(S_par, S_perp, Lx: int, Ly: int, k_lo: int = 1, k_hi: int = 8):
    """xi_par, xi_perp from replica-averaged structure factors (1-D arrays or
    tensors over k, or (replicas, K) arrays, averaged here)."""
    sp = np.asarray(S_par.cpu() if hasattr(S_par, "cpu") else S_par, dtype=np.float64)
    sq = np.asarray(S_perp.cpu() if hasattr(S_perp, "cpu") else S_perp, dtype=np.float64)
    if sp.ndim == 2:
        sp, sq = sp.mean(axis=0), sq.mean(axis=0)
    return fit_lorentzian(sp, Lx, k_lo, k_hi)[1], fit_lorentzian(sq, Ly, k_lo, k_hi)[1]
