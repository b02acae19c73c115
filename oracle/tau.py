"""FP64 oracle of the time-series error analysis (arXiv 2409.06412, App. B:
Eq. Autocorrelation-Function, Eq. Autocorrelation-Time, Eq. Time-Series-Var).

TEST INFRASTRUCTURE, like the rest of ``oracle/``.

For a series f_0 .. f_{n-1} sampled every Delta s (here: every record):
  mean        f_bar = (1/n) sum_s f_s
  C(m)        = 1/(n - m) sum_{s=0}^{n-m-1} (f_s - f_bar)(f_{s+m} - f_bar)   (average over the
                available pairs at lag m; C(0) = sigma_f^2)
  tau(M)      = 1/2 + sum_{m=1}^{M} C(m) / C(0)   (the discrete form of
                1/2 int_{-M}^{M} C_f(t)/C_f(0) dt, in units of Delta s)
  tau_C       = tau(M) with the window M chosen as
                  "auto": the smallest M >= 1 with M >= c tau(M) (c = 6), the
                          self-consistent window of the reference the paper
                          cites for this relation (Madras and Sokal); M = n/2
                          if no smaller M qualifies;
                  "half": M = floor(n / 2), the paper's tau_s / 2 taken
                          literally -- on a finite series the mean-subtracted
                          C(m) sum to about zero over all lags, so this window
                          is kept for comparison only;
  sigma_mean^2 = (2 tau_C / Delta s) sigma_f^2 / n
"""
from __future__ import annotations

import numpy as np


def autocorrelation(f: np.ndarray, max_lag: int | None = None) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    n = f.size
    M = n // 2 if max_lag is None else max_lag
    d = f - f.mean()
    C = np.empty(M + 1)
    for m in range(M + 1):
        C[m] = np.dot(d[:n - m], d[m:]) / (n - m)
    return C


def tau_int(f: np.ndarray, window: str = "auto", c: float = 6.0) -> float:
    C = autocorrelation(f)
    if C[0] <= 0:
        return 0.5
    rho = C / C[0]
    M_max = len(C) - 1
    if window == "half":
        return 0.5 + float(np.sum(rho[1:]))
    t = 0.5
    for M in range(1, M_max + 1):
        t += rho[M]
        if M >= c * t:
            return float(t)
    return float(t)


def error_of_mean(f: np.ndarray, window: str = "auto", c: float = 6.0) -> float:
    f = np.asarray(f, dtype=np.float64)
    C0 = autocorrelation(f, 0)[0]
    var = 2.0 * tau_int(f, window, c) * C0 / f.size
    # the literal half-series window can give tau_C < 0 (App. B's integral of
    # a finite series' autocovariance); the error of the mean is then undefined
    return float(np.sqrt(var)) if var >= 0.0 else float("nan")
