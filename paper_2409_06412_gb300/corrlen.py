"""Correlation length from the structure factor (arXiv 2409.06412, App. C).

Near k = 0 the structure factor of exponentially decaying correlations is a
Lorentzian (Eq. Lorentzian-Peak), S(k) = a / (1 + (2 pi xi k / N)^2) with k the
DFT index and N the lattice extent in that direction; below T_c the k = 0
value carries a delta peak from the constant part of C(r) and is left out of
the fit window.  This module fits (a, xi) on the host: the structure factors
themselves come from the GPU (``Lattice.structure_factor``), averaged over
replicas by the caller.

Two forms of the denominator are offered:
  "continuum": 1 + xi^2 (2 pi k / N)^2, the paper's Eq. Lorentzian-Peak;
  "lattice":   1 + xi^2 4 sin^2(pi k / N), its lattice counterpart: the
               transform of exp(-|r| / l) correlations on a periodic chain
               is exactly this Lorentzian (with xi^2 = rho / (1 - rho)^2,
               rho = exp(-1 / l)), and it equals the continuum form to
               O((k / N)^2) near k = 0.
The lattice form stays exact where the correlation length is a few sites or
less and the peak spans a large part of the Brillouin zone; there the
continuum form would need wavenumbers where it no longer holds.

The fit linearises 1 / S = 1/a + (xi^2 / a) q2(k), solves it by least
squares weighted with S^2 (so that it approximates least squares on S
itself), then polishes (a, xi^2) with Gauss-Newton steps on the residuals
S(k) - a / (1 + xi^2 q2(k)).

Window: given, or chosen from the data (``k_hi=None``): start from every
wavenumber supplied, then set k_hi to the k where (2 pi xi k / N) reaches 1,
i.e. the half-width of the peak, clamped to the supplied range and to at
least three points, and refit until the window stops changing.
"""
from __future__ import annotations

import math

import numpy as np


def _q2(k: np.ndarray, N: int, form: str) -> np.ndarray:
    if form == "lattice":
        return 4.0 * np.sin(np.pi * k / N) ** 2
    if form == "continuum":
        return (2.0 * np.pi * k / N) ** 2
    raise ValueError(f"unknown form {form!r}")


def _fit_window(y: np.ndarray, q2: np.ndarray, iters: int):
    """(a, b) of y = a / (1 + b q2); b <= 0 means no decay."""
    w = y * y
    A = np.stack([np.ones_like(q2), q2], axis=1) * w[:, None]
    alpha, beta = np.linalg.lstsq(A, w / y, rcond=None)[0]
    if alpha <= 0 or beta <= 0:
        return float(np.mean(y)), 0.0
    a, b = 1.0 / alpha, beta / alpha
    for _ in range(iters):
        d = 1.0 + b * q2
        r = y - a / d
        J = np.stack([1.0 / d, -a * q2 / (d * d)], axis=1)
        step = np.linalg.lstsq(J, r, rcond=None)[0]
        a, b = a + step[0], b + step[1]
        if b <= 0:
            return float(a), 0.0
        if np.max(np.abs(step) / np.maximum(np.abs([a, b]), 1e-300)) < 1e-15:
            break
    return float(a), float(b)


def fit_lorentzian(S, N: int, k_lo: int = 1, k_hi: int | None = None, iters: int = 50, form: str = "lattice",
                   return_window: bool = False):
    """Fit S[k_lo..k_hi] to a / (1 + xi^2 q2(k)), q2 as ``form`` selects.
    Returns (a, xi), plus (k_lo, k_hi) with ``return_window``.  xi is NaN
    when the window shows no decay (S not decreasing in q2): a flat window
    carries no length, and zero would be a wrong one."""
    y_all = np.asarray(S, dtype=np.float64)
    K = y_all.shape[0]
    auto = k_hi is None
    hi = K - 1 if auto else int(k_hi)
    if hi > K - 1 or hi - k_lo + 1 < 2:
        raise ValueError("need at least two values in the fit window")
    seen = set()
    while True:
        k = np.arange(k_lo, hi + 1, dtype=np.float64)
        y = y_all[k_lo:hi + 1]
        if np.any(y <= 0):
            raise ValueError("the structure factor must be positive in the fit window")
        a, b = _fit_window(y, _q2(k, N, form), iters)
        xi = math.sqrt(b) if b > 0 else float("nan")
        if not auto or not b > 0:
            break
        seen.add(hi)
        want = int(math.ceil(N / (2.0 * math.pi * xi)))
        want = min(K - 1, max(k_lo + 2, want))
        if want == hi or want in seen:
            break
        hi = want
    out = (float(a), float(xi))
    return out + ((k_lo, hi),) if return_window else out


def correlation_lengths(S_par, S_perp, Lx: int, Ly: int, k_lo: int = 1, k_hi: int | None = None,
                        form: str = "lattice"):
    """xi_par, xi_perp from replica-averaged structure factors (1-D arrays or
    tensors over k, or (replicas, K) arrays, averaged here).  With k_hi None
    each direction's window follows its own correlation length."""
    sp = np.asarray(S_par.cpu() if hasattr(S_par, "cpu") else S_par, dtype=np.float64)
    sq = np.asarray(S_perp.cpu() if hasattr(S_perp, "cpu") else S_perp, dtype=np.float64)
    if sp.ndim == 2:
        sp, sq = sp.mean(axis=0), sq.mean(axis=0)
    return (fit_lorentzian(sp, Lx, k_lo, k_hi, form=form)[1], fit_lorentzian(sq, Ly, k_lo, k_hi, form=form)[1])
