"""Long-run statistics: the GPU's equilibrium observables against the oracle's
within 3 sigma (the benchmark spec's tolerance for long runs).

16 replicas of an L x L lattice at T_c from the ordered start, 10^5 BBK steps
on both sides, (M, E) recorded every 10 steps,
the first 20 % discarded (t0 = 0.2 n).  With the same seed the damped,
equally driven FP32 and FP64 runs stay close (the shared noise keeps
pulling them together), so their difference is far inside 3 sigma; with an
independent seed for the oracle the two runs are independent samples of the
same stationary process and the test is a genuine two-sample comparison.

Per side: <M^2>, <M^4> and <E> are replica means of time averages, each
replica's error of the mean from its integrated autocorrelation time (App. B,
Eq. Time-Series-Var, with the self-consistent window of oracle/tau.py); the
Binder ratio U = <M^4> / <M^2>^2 (Eq. Def-Binder-Cum) gets its error from a
jackknife over the independent replicas.  Each observable must agree within
3 sqrt(sigma_gpu^2 + sigma_oracle^2).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import tau as otau
from paper_2409_06412_gb300 import Config, Lattice, build
from tests import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_STEPS, EVERY, N_REP = 10 ** 5, 10, 16


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()


def _stats(rec: np.ndarray):
    """rec: (replicas, records, 2) of (M, E) -> dict of (value, sigma)."""
    keep = rec[:, int(0.2 * rec.shape[1]):, :]
    M, E = keep[..., 0], keep[..., 1]
    out = {}
    for name, f in (("M2", M ** 2), ("M4", M ** 4), ("E", E)):
        means = f.mean(axis=1)
        sig = np.array([otau.error_of_mean(f[r]) for r in range(f.shape[0])])
        out[name] = (float(means.mean()), float(np.sqrt(np.sum(sig ** 2)) / f.shape[0]))
    m2, m4 = (M ** 2).mean(axis=1), (M ** 4).mean(axis=1)
    R = m2.size
    U = m4.mean() / m2.mean() ** 2
    jack = np.array([np.delete(m4, r).mean() / np.delete(m2, r).mean() ** 2 for r in range(R)])
    out["U"] = (float(U), float(np.sqrt((R - 1) / R * np.sum((jack - jack.mean()) ** 2))))
    return out


@pytest.mark.parametrize("L,oracle_seed", [(32, 1), (32, 2), (64, 2)])
def test_long_run_observables_within_three_sigma(L, oracle_seed):
    """oracle_seed 1: the same noise on both sides; 2: an independent oracle
    run, where the difference is a genuine two-sample comparison."""
    lat = Lattice([Config(Lx=L, Ly=L, n_replicas=N_REP, seed=1, init_mode=1, knots=((0,), (inputs.T_C,)),
                          n_total=N_STEPS)])
    rec_g = lat.step(N_STEPS, record_every=EVERY).cpu().numpy()[:, :N_STEPS // EVERY, :]
    lat.close()
    spec = inputs.config(L, L, N_REP, seed=oracle_seed, n_total=N_STEPS)
    th = [np.stack([oracle.init_theta(L, L, 0, r, oracle_seed, 1) for r in range(N_REP)])]
    om = [np.zeros_like(th[0])]
    rec_o, _ = oracle.run_batch([spec], th, om, [0], N_STEPS, record_every=EVERY)
    rec_o = rec_o[0][:, :N_STEPS // EVERY, :]
    assert np.all(np.isfinite(rec_g)) and rec_g.shape == rec_o.shape
    sg, so = _stats(rec_g), _stats(rec_o)
    lines = []
    for k in ("M2", "M4", "U", "E"):
        (vg, eg), (vo, eo) = sg[k], so[k]
        z = abs(vg - vo) / np.hypot(eg, eo)
        lines.append(f"{k}: gpu {vg:.6g} +- {eg:.2g}, oracle {vo:.6g} +- {eo:.2g}, |z| = {z:.2f}")
    print(f"L = {L}, oracle seed {oracle_seed}: " + "; ".join(lines))
    for k in ("M2", "M4", "U", "E"):
        (vg, eg), (vo, eo) = sg[k], so[k]
        assert eg > 0 and eo > 0
        assert abs(vg - vo) <= 3 * np.hypot(eg, eo), lines
