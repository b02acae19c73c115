"""Host side of the correlation-length pipeline: the library's Lorentzian fit
(paper_2409_06412_gb300.corrlen) recovers exact Lorentzians and agrees with
the oracle's independent least-squares fit on structure factors the oracle
computed (Sec. VI, Eq. Lorentzian-Peak)."""
import math

import numpy as np
import pytest

from oracle import corrlen as ocl
from paper_2409_06412_gb300 import corrlen
from tests.inputs import ar1_field


@pytest.mark.parametrize("a,xi,N", [(3.7, 12.5, 256), (0.4, 1.3, 64), (50.0, 80.0, 1024)])
def test_fit_exact_lorentzian(a, xi, N):
    S = a / (1 + (2 * math.pi * xi * np.arange(N) / N) ** 2)
    a_f, xi_f = corrlen.fit_lorentzian(S, N, 1, 10)
    assert abs(a_f / a - 1) < 1e-9 and abs(xi_f / xi - 1) < 1e-9


def test_fit_agrees_with_oracle_fit():
    rho, eps = 0.85, 0.05
    th = np.stack([eps * ar1_field(256, 64, rho, seed=7 + b) for b in range(6)])
    S_par, _ = ocl.structure_factor(th)
    S = S_par.mean(axis=0)
    a1, xi1 = corrlen.fit_lorentzian(S, 256, 1, 10)
    a2, xi2 = ocl.fit_lorentzian(S, 256, 1, 10)
    assert abs(xi1 / xi2 - 1) < 1e-6 and abs(a1 / a2 - 1) < 1e-6


def test_fit_rejects_empty_window():
    with pytest.raises(ValueError):
        corrlen.fit_lorentzian(np.ones(8), 8, 3, 3)
