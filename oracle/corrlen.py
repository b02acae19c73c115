"""FP64 oracle of the correlation-length pipeline (arXiv 2409.06412, App. C,
"Correlation Length Extraction").

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it.  It
imports nothing from the library.

Rotors s = (cos(r theta), sin(r theta)); the paper writes (cos theta, sin theta),
so r = 1 is its literal definition, and r is a parameter.  For a lattice
s[j, i] with j the perpendicular index (N_perp rows) and i the parallel index
(N_par columns):

  Eq. S-as-lattice-FT:   S_perp(k) = 1/(N_perp N_par^2) sum_l sum_kappa |s~^kappa_{k,l}|^2,
                         s~_{k,l} = sum_{i,j} s_{i,j} exp(-2 pi i (k j / N_perp + l i / N_par)),
  and the analogue for S_par(l) (sum over k, 1/(N_par N_perp^2)).

  Eq. Lorentzian-Peak:   S_delta(k) ~ 2 xi / (1 + 4 pi^2 xi^2 k^2), k the
                         wavenumber in cycles per site (index / N_delta);
                         fitted here as a / (1 + (2 pi xi k / N_delta)^2)
                         over a window of small k, k = 0 dropped below T_c
                         ("continuum"), or with (2 pi k / N)^2 replaced by
                         the lattice Laplacian's 4 sin^2(pi k / N)
                         ("lattice"), the exact transform of exponentially
                         decaying correlations on a periodic chain.

Every step is the plain definition; numpy's FFT serves as the 2-D transform.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares


def rotors(theta: np.ndarray, r: float = 1.0):
    t = np.asarray(theta, dtype=np.float64)
    return np.cos(r * t), np.sin(r * t)


def structure_factor(theta: np.ndarray, r: float = 1.0):
    """theta: (Ly, Lx) or (B, Ly, Lx).  Returns (S_par[..., Lx], S_perp[..., Ly])
    per Eq. S-as-lattice-FT (rows are the perpendicular direction)."""
    th = np.asarray(theta, dtype=np.float64)
    single = th.ndim == 2
    if single:
        th = th[None]
    B, Ny, Nx = th.shape
    S_par = np.zeros((B, Nx))
    S_perp = np.zeros((B, Ny))
    for b in range(B):
        for comp in rotors(th[b], r):
            F = np.fft.fft2(comp)          # F[k, l]: k over rows (perp), l over columns (par)
            P = np.abs(F) ** 2
            S_perp[b] += P.sum(axis=1) / (Ny * Nx * Nx)
            S_par[b] += P.sum(axis=0) / (Nx * Ny * Ny)
    if single:
        return S_par[0], S_perp[0]
    return S_par, S_perp


def correlation_functions(theta: np.ndarray, r: float = 1.0):
    """Brute-force periodic C_par(x), C_perp(y) (Eq. Ensemble-Avg-as-mean on
    the finite periodic lattice), by explicit loops over the displacement."""
    th = np.asarray(theta, dtype=np.float64)
    Ny, Nx = th.shape
    C_par = np.zeros(Nx)
    C_perp = np.zeros(Ny)
    # s_a . s_b of unit rotors at angles r theta_a, r theta_b is cos(r (theta_a - theta_b))
    for x in range(Nx):
        acc = 0.0
        for j in range(Ny):
            for i in range(Nx):
                acc += np.cos(r * (th[j, i] - th[j, (i + x) % Nx]))
        C_par[x] = acc / (Nx * Ny)
    for y in range(Ny):
        acc = 0.0
        for j in range(Ny):
            for i in range(Nx):
                acc += np.cos(r * (th[j, i] - th[(j + y) % Ny, i]))
        C_perp[y] = acc / (Nx * Ny)
    return C_par, C_perp


def ft_of_correlation(C: np.ndarray) -> np.ndarray:
    """Eq. FT-Corr-delta by a direct sum: S(k) = sum_r C(r) exp(-2 pi i k r / N) (real part)."""
    N = len(C)
    r = np.arange(N)
    return np.array([np.sum(C * np.cos(2 * np.pi * k * r / N)) for k in range(N)])


def lorentzian(k: np.ndarray, a: float, xi: float, N: int, form: str = "continuum") -> np.ndarray:
    k = np.asarray(k, dtype=np.float64)
    if form == "continuum":
        q2 = (2.0 * np.pi * k / N) ** 2
    elif form == "lattice":
        q2 = 4.0 * np.sin(np.pi * k / N) ** 2
    else:
        raise ValueError(form)
    return a / (1.0 + xi * xi * q2)


def exponential_chain_spectrum(rho: float, N: int) -> np.ndarray:
    """S(k), k = 0..N-1, of unit-variance correlations C(r) = rho^|r| on an
    infinite chain sampled at N-periodic wavenumbers: the geometric series
    sum_r rho^|r| e^{-2 pi i k r / N} = (1 - rho^2) / (1 - 2 rho cos(2 pi k / N) + rho^2)."""
    q = 2.0 * np.pi * np.arange(N) / N
    return (1.0 - rho * rho) / (1.0 - 2.0 * rho * np.cos(q) + rho * rho)


def fit_lorentzian(S: np.ndarray, N: int, k_lo: int, k_hi: int, xi0: float = 2.0, form: str = "continuum"):
    """Least-squares fit of S[k_lo..k_hi] to the Lorentzian of ``form``; returns (a, xi)."""
    k = np.arange(k_lo, k_hi + 1, dtype=np.float64)
    y = np.asarray(S, dtype=np.float64)[k_lo:k_hi + 1]
    a0 = float(y[0] / lorentzian(k[:1], 1.0, xi0, N, form)[0])
    res = least_squares(lambda p: lorentzian(k, p[0], p[1], N, form) - y, x0=[a0, xi0],
                        bounds=([0.0, 1e-6], [np.inf, 1e6]), xtol=1e-14, ftol=1e-14, gtol=1e-14)
    return float(res.x[0]), float(res.x[1])
