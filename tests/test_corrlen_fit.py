"""Host side of the correlation-length pipeline: the library's Lorentzian fit
(paper_2409_06412_gb300.corrlen) recovers exact Lorentzians and agrees with
the oracle's independent least-squares fit on structure factors the oracle
computed (App. C, Eq. Lorentzian-Peak)."""
import math

import numpy as np
import pytest

from oracle import corrlen as ocl
from paper_2409_06412_gb300 import corrlen
from tests.inputs import ar1_field


@pytest.mark.parametrize("a,xi,N", [(3.7, 12.5, 256), (0.4, 1.3, 64), (50.0, 80.0, 1024)])
def test_fit_exact_lorentzian(a, xi, N):
    S = a / (1 + (2 * math.pi * xi * np.arange(N) / N) ** 2)
    a_f, xi_f = corrlen.fit_lorentzian(S, N, 1, 10, form="continuum")
    assert abs(a_f / a - 1) < 1e-9 and abs(xi_f / xi - 1) < 1e-9


def test_fit_agrees_with_oracle_fit():
    rho, eps = 0.85, 0.05
    th = np.stack([eps * ar1_field(256, 64, rho, seed=7 + b) for b in range(6)])
    S_par, _ = ocl.structure_factor(th)
    S = S_par.mean(axis=0)
    for form in ("continuum", "lattice"):
        a1, xi1 = corrlen.fit_lorentzian(S, 256, 1, 10, form=form)
        a2, xi2 = ocl.fit_lorentzian(S, 256, 1, 10, form=form)
        assert abs(xi1 / xi2 - 1) < 1e-6 and abs(a1 / a2 - 1) < 1e-6


def test_fit_rejects_empty_window():
    with pytest.raises(ValueError):
        corrlen.fit_lorentzian(np.ones(8), 8, 3, 3)


@pytest.mark.parametrize("rho,N", [(0.25, 1024), (0.5, 256), (0.95, 512)])
def test_window_follows_the_correlation_length(rho, N):
    """Exact spectra of exponential correlations, K = N / 2 wavenumbers
    supplied: the window chosen from the data ends near N / (2 pi xi), and
    the length is exact whatever the window (lattice form)."""
    S = ocl.exponential_chain_spectrum(rho, N)[:N // 2]
    xi = math.sqrt(rho) / (1 - rho)
    a_f, xi_f, (lo, hi) = corrlen.fit_lorentzian(S, N, return_window=True)
    assert abs(xi_f / xi - 1) < 1e-8
    assert hi == min(N // 2 - 1, max(3, math.ceil(N / (2 * math.pi * xi))))


def test_flat_window_gives_nan_not_zero():
    rng = np.random.default_rng(3)
    S = 1.0 + 1e-3 * rng.standard_normal(64)
    S[np.arange(64) % 2 == 0] += 2e-3  # no decay in k
    _, xi = corrlen.fit_lorentzian(np.sort(S), 1024, 1, 30)  # increasing in k: no peak at 0
    assert math.isnan(xi)


def test_short_length_from_sampled_field_matches_oracle_fit():
    """xi < 1 across the rows of periodic AR(1) columns (rho = 0.3, xi = 0.78):
    the library's automatic window and the oracle's fit on that window agree,
    and both find the generating length within the sampling error."""
    rho, eps, Lx, Ly = 0.3, 0.05, 64, 256
    th = np.stack([eps * ar1_field(Lx, Ly, rho, seed=40 + b, axis=0) for b in range(8)])
    _, S_perp = ocl.structure_factor(th)
    S = S_perp.mean(axis=0)[:Ly // 2]
    _, xi1, (lo, hi) = corrlen.fit_lorentzian(S, Ly, return_window=True)
    _, xi2 = ocl.fit_lorentzian(S, Ly, lo, hi, form="lattice")
    assert abs(xi1 / xi2 - 1) < 1e-6
    assert abs(xi1 / (math.sqrt(rho) / (1 - rho)) - 1) < 0.1
