"""Pins of the correlation-length oracle (oracle/corrlen.py) against what the
paper and the mathematics fix, independently of the FFT it uses:

- Eq. S-as-lattice-FT equals Eq. FT-Corr-delta applied to the brute-force
  periodic correlation function (Wiener-Khinchin), on non-square lattices in
  both directions and for two rotor multiplicities;
- a perfectly ordered lattice has C(r) = 1: S(0) = N_delta, S(k != 0) = 0;
- a plane wave theta = 2 pi m x / N_par puts S_par = N_par / 2 at k = +-m;
- i.i.d. angles give E S(k != 0) = 1 - |<s>|^2 (here <cos> = 2/pi, <sin> = 0);
- the Lorentzian fit returns (a, xi) exactly on Lorentzian data, and the
  correlation length of an exponentially correlated field (periodic AR(1)
  rows with lag-one correlation rho: S(k) ~ Lorentzian with
  xi = sqrt(rho)/(1 - rho) near k = 0) from S computed on its rotors.
"""
import math

import numpy as np
import pytest

from oracle import corrlen
from tests.inputs import angles, ar1_field


@pytest.mark.parametrize("Lx,Ly,r", [(12, 8, 1.0), (8, 10, 2.0), (16, 4, 1.0)])
def test_structure_factor_is_ft_of_bruteforce_correlation(Lx, Ly, r):
    th = angles(1, Lx, Ly, seed=3).reshape(Ly, Lx).astype(np.float64)
    S_par, S_perp = corrlen.structure_factor(th, r)
    C_par, C_perp = corrlen.correlation_functions(th, r)
    np.testing.assert_allclose(S_par, corrlen.ft_of_correlation(C_par), rtol=0, atol=1e-11)
    np.testing.assert_allclose(S_perp, corrlen.ft_of_correlation(C_perp), rtol=0, atol=1e-11)
    # C(0) = <|s|^2> = 1 and the sum rule sum_k S(k) = N C(0)
    assert abs(C_par[0] - 1) < 1e-12 and abs(C_perp[0] - 1) < 1e-12
    assert abs(S_par.sum() - Lx) < 1e-9 and abs(S_perp.sum() - Ly) < 1e-9


def test_ordered_lattice():
    th = np.full((6, 10), 0.7)
    S_par, S_perp = corrlen.structure_factor(th)
    assert abs(S_par[0] - 10) < 1e-12 and abs(S_perp[0] - 6) < 1e-12
    assert np.max(np.abs(S_par[1:])) < 1e-12 and np.max(np.abs(S_perp[1:])) < 1e-12


@pytest.mark.parametrize("m", [1, 3])
def test_plane_wave(m):
    Lx, Ly = 16, 6
    x = np.arange(Lx)
    th = np.tile(2 * np.pi * m * x / Lx, (Ly, 1))
    S_par, S_perp = corrlen.structure_factor(th)
    expect = np.zeros(Lx)
    expect[m] = expect[Lx - m] = Lx / 2
    np.testing.assert_allclose(S_par, expect, atol=1e-10)
    exp_perp = np.zeros(Ly)
    exp_perp[0] = Ly
    np.testing.assert_allclose(S_perp, exp_perp, atol=1e-10)


def test_plane_wave_in_the_doubled_angle():
    # r = 2: theta = pi m y / N_perp makes the rotor angle 2 theta a wave of wavenumber m
    Lx, Ly, m = 6, 12, 2
    y = np.arange(Ly)
    th = np.tile((np.pi * m * y / Ly)[:, None], (1, Lx))
    S_par, S_perp = corrlen.structure_factor(th, 2.0)
    expect = np.zeros(Ly)
    expect[m] = expect[Ly - m] = Ly / 2
    np.testing.assert_allclose(S_perp, expect, atol=1e-10)


def test_iid_angles_flat_spectrum():
    th = angles(16, 32, 24, seed=11).reshape(16, 24, 32).astype(np.float64)
    S_par, S_perp = corrlen.structure_factor(th)
    expect = 1 - (2 / np.pi) ** 2
    vals = np.concatenate([S_par[:, 1:].ravel(), S_perp[:, 1:].ravel()])
    # each S(k) of one lattice averages N_other |.|^2 terms of a sum of i.i.d. unit vectors
    assert abs(vals.mean() - expect) < 5 * vals.std() / math.sqrt(vals.size)


def test_fit_exact_lorentzian():
    N = 256
    k = np.arange(N)
    S = corrlen.lorentzian(k, 3.7, 12.5, N)
    a, xi = corrlen.fit_lorentzian(S, N, 1, 10)
    assert abs(a - 3.7) < 1e-9 and abs(xi - 12.5) < 1e-9


def test_fit_recovers_exponential_correlation_length():
    rho, eps = 0.9, 0.05
    th = np.stack([eps * ar1_field(512, 128, rho, seed=100 + b) for b in range(8)])
    S_par, S_perp = corrlen.structure_factor(th)
    a, xi = corrlen.fit_lorentzian(S_par.mean(axis=0) / eps ** 2, 512, 1, 12)
    assert abs(xi / (math.sqrt(rho) / (1 - rho)) - 1) < 0.10
    # no correlation across the rows: flat S_perp away from k = 0
    assert abs(S_perp.mean(axis=0)[1:].mean() / eps ** 2 - 1) < 0.05


@pytest.mark.parametrize("rho,N", [(0.2, 64), (0.5, 128), (0.9, 256)])
def test_exponential_chain_spectrum_is_the_transform_of_rho_to_the_r(rho, N):
    # brute force: the N-periodic correlation sum_m rho^|r + m N| (images out
    # to where rho^|r| underflows), transformed by the FFT
    r = np.arange(N)
    C = np.zeros(N)
    for m in range(-60, 61):
        C += rho ** np.abs(r + m * N)
    S_fft = np.fft.fft(C).real
    np.testing.assert_allclose(corrlen.exponential_chain_spectrum(rho, N), S_fft, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("rho,N", [(0.2, 64), (0.5, 128), (0.9, 256), (0.3, 1024)])
def test_lattice_lorentzian_recovers_the_exponential_length(rho, N):
    """On a periodic chain with C(r) = rho^|r| the lattice form of the
    Lorentzian is exact over the whole zone: xi = sqrt(rho) / (1 - rho)
    (C(r) = exp(-r / l), l = -1 / ln rho; xi -> l for l >> 1) and
    a = (1 + rho) / (1 - rho), from any window."""
    S = corrlen.exponential_chain_spectrum(rho, N)
    xi = math.sqrt(rho) / (1 - rho)
    for lo, hi in ((1, N // 2), (1, 5), (N // 8, N // 4)):
        a_f, xi_f = corrlen.fit_lorentzian(S, N, lo, hi, form="lattice")
        assert abs(xi_f / xi - 1) < 1e-8 and abs(a_f / ((1 + rho) / (1 - rho)) - 1) < 1e-8
    # the continuum form of Eq. Lorentzian-Peak agrees near k = 0 when xi >> 1
    if xi > 5:
        _, xi_c = corrlen.fit_lorentzian(S, N, 1, 3, form="continuum")
        assert abs(xi_c / xi - 1) < 1e-3
