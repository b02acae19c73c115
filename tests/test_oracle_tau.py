"""Pins of the time-series error analysis oracle (oracle/tau.py, App. B):

- an AR(1) series with lag-one correlation phi has rho(m) = phi^m and
  tau_C = 1/2 + phi / (1 - phi) = (1 + phi) / (2 (1 - phi));
- i.i.d. samples have tau_C = 1/2 and sigma_mean = sigma / sqrt(n);
- the error of the mean predicts the spread of the means of many independent
  series (Eq. Time-Series-Var), where the naive sigma/sqrt(n) does not;
- C(m) is the lag-m covariance: checked against an independent FFT-based
  circular-free estimate on a short series.
"""
import math

import numpy as np
import pytest

from oracle import tau
from tests.inputs import ar1_series


@pytest.mark.parametrize("phi", [0.5, 0.9])
def test_ar1_tau(phi):
    x = ar1_series(20000, phi, seed=3, n_series=8)
    taus = np.array([tau.tau_int(s) for s in x])
    exact = (1 + phi) / (2 * (1 - phi))
    # the windowed estimator is biased low by about exp(-c) and fluctuates by ~ tau sqrt(4 M / n)
    assert abs(taus.mean() / exact - 1) < 0.10


def test_iid_tau_and_error():
    rng = np.random.default_rng(5)
    f = rng.standard_normal(50000) * 2.0 + 1.0
    assert abs(tau.tau_int(f) - 0.5) < 0.15
    assert abs(tau.error_of_mean(f) / (2.0 / math.sqrt(f.size)) - 1) < 0.2


def test_error_of_mean_predicts_spread_of_means():
    phi, n = 0.8, 4000
    x = ar1_series(n, phi, seed=9, n_series=400)
    means = x.mean(axis=1)
    predicted = np.mean([tau.error_of_mean(s) for s in x[:40]])
    assert abs(means.std() / predicted - 1) < 0.2
    naive = 1 / math.sqrt(n)
    assert means.std() / naive > 2.5  # correlated samples: the naive error is far too small


def test_half_window_is_the_literal_sum():
    rng = np.random.default_rng(4)
    f = rng.standard_normal(101)
    C = tau.autocorrelation(f)
    assert abs(tau.tau_int(f, "half") - (0.5 + C[1:].sum() / C[0])) < 1e-12


def test_autocorrelation_matches_fft_estimate():
    rng = np.random.default_rng(2)
    f = rng.standard_normal(257)
    C = tau.autocorrelation(f)
    d = f - f.mean()
    n = f.size
    F = np.fft.rfft(np.concatenate([d, np.zeros(n)]))
    acf = np.fft.irfft(np.abs(F) ** 2)[: n // 2 + 1]  # linear (zero-padded) correlation sums
    np.testing.assert_allclose(C, acf / (n - np.arange(n // 2 + 1)), rtol=1e-10, atol=1e-12)
