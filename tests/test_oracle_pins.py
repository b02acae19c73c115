"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No test here retypes an oracle formula: each compares it with a closed form,
a quadrature of the canonical distribution (App. A.2, Eq. Canonical-Dist), a
library routine, brute force on tiny inputs, or an invariant; each is chosen so
that a plausible slip (a dropped factor, a wrong sign or index, reused noise)
fails it.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from tests import inputs

PI = math.pi


# ----------------------------------------------------------------- noise


def test_uniform_endpoints_and_exactness():
    # (m + 1/2) 2^-23 with m the top 23 bits: the extremes are 2^-24 and 1 - 2^-24
    u = oracle.uniform(np.array([0, 0xFFFFFFFF, 0x00000200, 0x80000000], dtype=np.uint32))
    assert u[0] == 2.0 ** -24
    assert u[1] == 1.0 - 2.0 ** -24
    assert u[2] == 1.5 * 2.0 ** -23
    assert u[3] == 0.5 + 2.0 ** -24
    assert np.all(np.float32(u) == u)  # exact in binary32


def test_philox_statistics_and_avalanche():
    n = 1 << 18
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 1] = 0x00010002
    out = oracle.philox(ctr, (1, 0))
    w = out.ravel()
    # every output bit is fair (4n words, sigma = sqrt(4n)/2)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.float64)
    ones = bits.sum(axis=0)
    sigma = math.sqrt(w.size) / 2
    assert np.all(np.abs(ones - w.size / 2) < 5 * sigma)
    # byte histogram chi-square (255 dof)
    hist = np.bincount((w & 0xFF).astype(np.int64), minlength=256)
    e = w.size / 256
    chi2 = ((hist - e) ** 2 / e).sum()
    assert 180 < chi2 < 340
    # avalanche: flipping one counter bit flips ~half of the 128 output bits
    for word in range(4):
        for bit in (0, 7, 31):
            c2 = ctr[:4096].copy()
            c2[:, word] ^= np.uint32(1 << bit)
            o2 = oracle.philox(c2, (1, 0))
            flips = np.unpackbits((out[:4096] ^ o2).view(np.uint8)).reshape(4096, -1).sum(axis=1)
            assert abs(flips.mean() - 64) < 1.0
    # the key matters
    o3 = oracle.philox(ctr[:4096], (2, 0))
    assert np.mean(o3 == out[:4096]) < 1e-3


def test_gaussian_moments_and_box_muller_radius():
    g = np.concatenate([oracle.gauss(7, 3, 5, 1 << 16, k) for k in range(8)])
    n = g.size
    assert abs(g.mean()) < 4 / math.sqrt(n)
    assert abs(g.var() - 1) < 4 * math.sqrt(2 / n)
    kurt = (g ** 4).mean() / g.var() ** 2
    assert abs(kurt - 3) < 4 * math.sqrt(24 / n)
    # the two samples of one Box-Muller pair share the radius -2 ln u of the
    # first word of the pair: check against the raw Philox words
    k, seed, cfg, rep = 11, 7, 3, 5
    gq = oracle.gauss(seed, cfg, rep, 64, k)
    ctr = np.zeros((16, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(16)
    ctr[:, 1] = (cfg << 16) | rep
    ctr[:, 2] = k
    w = oracle.philox(ctr, (seed, 0))
    u = ((w >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    r2 = gq.reshape(16, 4)
    assert np.allclose(r2[:, 0] ** 2 + r2[:, 1] ** 2, -2 * np.log(u[:, 0]), rtol=1e-12)
    assert np.allclose(r2[:, 2] ** 2 + r2[:, 3] ** 2, -2 * np.log(u[:, 2]), rtol=1e-12)
    assert np.allclose(np.arctan2(r2[:, 1], r2[:, 0]) % (2 * PI), (2 * PI * u[:, 1]) % (2 * PI), atol=1e-9)


def test_noise_streams_are_distinct():
    a = oracle.gauss(1, 0, 0, 256, 5)
    for other in (oracle.gauss(1, 0, 1, 256, 5), oracle.gauss(1, 1, 0, 256, 5),
                  oracle.gauss(1, 0, 0, 256, 6), oracle.gauss(2, 0, 0, 256, 5),
                  oracle.gauss(1, 0, 0, 256, 5, tag=1), oracle.gauss(1, 0, 0, 256, 5 + (1 << 32))):
        assert abs(np.corrcoef(a, other)[0, 1]) < 0.3
        assert not np.any(a == other)


# ----------------------------------------------------------------- state space


def test_wrap_interval_and_periodicity():
    x = np.linspace(-20, 20, 100001)
    w = oracle.wrap(x)
    assert np.all(w >= -PI / 2) and np.all(w < PI / 2)
    assert np.allclose(np.sin(2 * w), np.sin(2 * x), atol=1e-12)  # same state mod pi
    inside = (x >= -PI / 2) & (x < PI / 2)
    assert np.array_equal(w[inside], x[inside])
    assert oracle.wrap([PI / 2])[0] == -PI / 2
    assert oracle.wrap([-PI / 2])[0] == -PI / 2


def test_temperature_schedule_linear_quench():
    Tc = 1.969
    knots = ([1000, 1000 + 1500], [1.5 * Tc, 0.0])  # eps(t) = -t / tau_Q with tau_Q = 1000 steps
    for k, expect in [(0, 1.5 * Tc), (1000, 1.5 * Tc), (1500, Tc), (2500, 0.0), (9999, 0.0)]:
        assert oracle.temperature(k, knots) == pytest.approx(expect, abs=1e-12)
    for k in range(1000, 2500, 37):
        eps = (oracle.temperature(k, knots) - Tc) / Tc
        assert eps == pytest.approx(0.5 - (k - 1000) / 1000, abs=1e-12)


def test_init_modes():
    th = oracle.init_theta(16, 8, 0, 0, 1, 1)
    assert np.all(th == 2 * PI / 5)
    M, E = oracle.observe(16, 8, {}, th, np.zeros_like(th))
    # ordered state: every bond cos 0 = 1, cos(p * 2pi/5) = cos(pi) = -1
    assert E == pytest.approx(-10.0 - 0.1 - 1.0, abs=1e-12)
    assert M == pytest.approx(math.sin(4 * PI / 5), abs=1e-12)
    th = oracle.init_theta(64, 64, 2, 3, 9, 0)
    assert np.all(th >= -PI / 2) and np.all(th < PI / 2)
    # uniform on [0, 2 pi) folded twice onto the interval is uniform on it
    assert abs(th.mean()) < 4 * (PI / math.sqrt(12)) / 64
    assert abs(th.var() - PI ** 2 / 12) < 0.05


# ----------------------------------------------------------------- model


def _hamiltonian(Lx, Ly, prm, th, om):
    """Eq. (XY-Hamilton-Kinetic) with Eq. (XY-Hamilton-Field), periodic,
    written over whole arrays with np.roll."""
    t = th.reshape(Ly, Lx)
    w = om.reshape(Ly, Lx)
    q, p = prm["q"], prm["p"]
    return (0.5 * (w ** 2).sum()
            - prm["J_par"] * np.cos(q * (t - np.roll(t, -1, axis=1))).sum()
            - prm["J_perp"] * np.cos(q * (t - np.roll(t, -1, axis=0))).sum()
            + prm["h"] * np.cos(p * t).sum())


@pytest.mark.parametrize("Lx,Ly", [(8, 6), (4, 4), (2, 3), (5, 1)])
def test_force_is_minus_gradient_of_hamiltonian(Lx, Ly):
    prm = dict(inputs.PAPER, J_par=3.0, J_perp=-0.7, h=1.3)
    rng = np.random.default_rng(5)
    th = rng.uniform(-1.2, 1.2, Lx * Ly)
    om = rng.standard_normal(Lx * Ly)
    F = oracle.force(Lx, Ly, prm, th)
    eps = 1e-6
    for i in range(Lx * Ly):
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        dH = (_hamiltonian(Lx, Ly, prm, tp, om) - _hamiltonian(Lx, Ly, prm, tm, om)) / (2 * eps)
        assert F[i] == pytest.approx(-dH, abs=2e-7)
    M, E = oracle.observe(Lx, Ly, prm, th, om)
    assert E * Lx * Ly == pytest.approx(_hamiltonian(Lx, Ly, prm, th, om), rel=1e-12)
    assert M == pytest.approx(np.sin(2 * th).mean(), rel=1e-12)


def test_ground_state_energy_reading_A():
    """T = 0 relaxation from the ordered state plus noise reaches E/N = -J_par - J_perp - h."""
    Lx = Ly = 8
    rng = np.random.default_rng(1)
    th = oracle.init_theta(Lx, Ly, 0, 0, 1, 1) + 0.05 * rng.standard_normal(Lx * Ly)
    om = np.zeros(Lx * Ly)
    oracle.run_lattice(Lx, Ly, 0, 0, 1, {}, ([0], [0.0]), 0, 6000, th, om)
    M, E = oracle.observe(Lx, Ly, {}, th, om)
    assert E == pytest.approx(-11.1, abs=1e-9)
    assert np.allclose(th, 2 * PI / 5, atol=1e-6)


def test_ground_state_energy_reading_B_checkerboard():
    """J -> -J: the ground state is a checkerboard of +-phi*; its energy is the
    minimum over phi of (|J_par| + |J_perp|) cos(4 phi) + h cos(p phi)."""
    Lx = Ly = 8
    Jx, Jy, h, p = 10.0, 0.1, 1.0, 2.5
    phi = np.linspace(0, PI / 2, 2000001)
    f = (Jx + Jy) * np.cos(4 * phi) + h * np.cos(p * phi)
    e_min = f.min()
    phi_star = phi[f.argmin()]
    assert phi_star == pytest.approx(0.7995, abs=2e-3)
    assert e_min == pytest.approx(-10.4989, abs=2e-3)
    yy, xx = np.mgrid[0:Ly, 0:Lx]
    sign = np.where((xx + yy) % 2 == 0, 1.0, -1.0).ravel()
    rng = np.random.default_rng(2)
    th = sign * 0.7 + 0.05 * rng.standard_normal(Lx * Ly)
    om = np.zeros(Lx * Ly)
    prm = dict(J_par=-Jx, J_perp=-Jy)
    oracle.run_lattice(Lx, Ly, 0, 0, 1, prm, ([0], [0.0]), 0, 8000, th, om)
    M, E = oracle.observe(Lx, Ly, prm, th, om)
    assert E == pytest.approx(e_min, abs=1e-8)
    assert np.allclose(np.abs(th), phi_star, atol=1e-5)
    # staggered order parameter is the sign-corrected one
    Ms, _ = oracle.observe(Lx, Ly, dict(prm, staggered=1.0), th, om)
    assert abs(Ms) == pytest.approx(abs(math.sin(2 * phi_star)), abs=1e-5)
    assert abs(M) < 1e-9


def test_monotone_energy_descent_at_zero_temperature():
    """dE/dt = -eta sum omega^2 <= 0 without noise; BBK keeps it up to O(dt^2)."""
    Lx = Ly = 8
    excess = []
    for dt in (0.01, 0.005):
        th = inputs.angles(1, Lx, Ly, 3)[0].astype(np.float64)
        om = np.zeros(Lx * Ly)
        n = int(round(5.0 / dt))
        rec = oracle.run_lattice(Lx, Ly, 0, 0, 1, dict(dt=dt), ([0], [0.0]), 0, n, th, om, 1)
        E = rec[:, 1]
        dE = np.diff(E)
        assert E[-1] < E[0] - 1.0
        excess.append(max(dE.max(), 0.0))
        assert dE.max() < 1e-3 * abs(E).max()
    # any positive excursion is a discretisation effect: it shrinks at least ~4x when dt halves
    if excess[0] > 1e-12:
        assert excess[1] < excess[0] / 3.0


# ----------------------------------------------------------------- canonical distribution


def _sample_angles(Lx, Ly, n_rep, prm, T, n_burn, n_steps, every, seed=1):
    samples = []
    om_samples = []
    for r in range(n_rep):
        th = oracle.init_theta(Lx, Ly, 0, r, seed, 0)
        om = np.zeros(Lx * Ly)
        oracle.run_lattice(Lx, Ly, 0, r, seed, prm, ([0], [T]), 0, n_burn, th, om)
        k = n_burn
        while k < n_burn + n_steps:
            oracle.run_lattice(Lx, Ly, 0, r, seed, prm, ([0], [T]), k, every, th, om)
            k += every
            samples.append(th.copy())
            om_samples.append(om.copy())
    return np.array(samples), np.array(om_samples)


@pytest.mark.parametrize("T", [0.5, 2.0, 10.0])
def test_single_angle_boltzmann(T):
    """J = 0: each angle follows p(theta) ~ exp(-h cos(p theta) / T) on [-pi/2, pi/2)."""
    prm = dict(J_par=0.0, J_perp=0.0, h=1.0)
    th, om = _sample_angles(32, 32, 1, prm, T, 500, 8000, 40)
    x = th.ravel()
    edges = np.linspace(-PI / 2, PI / 2, 41)
    hist, _ = np.histogram(x, bins=edges)
    Z = integrate.quad(lambda t: math.exp(-math.cos(2.5 * t) / T), -PI / 2, PI / 2)[0]
    prob = np.array([integrate.quad(lambda t: math.exp(-math.cos(2.5 * t) / T), a, b)[0] / Z
                     for a, b in zip(edges[:-1], edges[1:])])
    expect = prob * x.size
    # samples are correlated in time: allow an effective-sample inflation of 4
    z = (hist - expect) / np.sqrt(4 * expect)
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    # equipartition <omega^2> = T (pins one Gaussian per time point shared by both kicks)
    w2 = (om ** 2).mean()
    assert w2 == pytest.approx(T, rel=0.03)


def test_equipartition_halves_with_fresh_draws_reading():
    """If each half-kick drew a fresh Gaussian the injected variance would halve:
    <omega^2> = T/2.  The oracle's shared-sample reading must give T."""
    prm = dict(J_par=0.0, J_perp=0.0, h=0.0)
    _, om = _sample_angles(32, 32, 1, prm, 3.0, 500, 4000, 20)
    assert (om ** 2).mean() == pytest.approx(3.0, rel=0.03)


def test_two_by_two_lattice_boltzmann():
    """2 x 2 periodic lattice (each bond counted twice by the forward-bond sum):
    averages against 4-D quadrature of exp(-H_XY / T)."""
    prm = dict(J_par=1.0, J_perp=0.4, h=1.0)
    T = 1.5
    th, _ = _sample_angles(2, 2, 64, prm, T, 400, 6000, 20)
    t = th.reshape(-1, 4)
    n = 36
    g = -PI / 2 + (np.arange(n) + 0.5) * PI / n
    a, b, c, d = np.meshgrid(g, g, g, g, indexing="ij")
    # sites: 0=(0,0) 1=(1,0) 2=(0,1) 3=(1,1); x-bonds 0-1, 2-3; y-bonds 0-2, 1-3; each twice
    H = (-2 * prm["J_par"] * (np.cos(2 * (a - b)) + np.cos(2 * (c - d)))
         - 2 * prm["J_perp"] * (np.cos(2 * (a - c)) + np.cos(2 * (b - d)))
         + prm["h"] * (np.cos(2.5 * a) + np.cos(2.5 * b) + np.cos(2.5 * c) + np.cos(2.5 * d)))
    w = np.exp(-(H - H.min()) / T)
    w /= w.sum()
    checks = {
        "cos2(t0-t1)": (np.cos(2 * (a - b)), np.cos(2 * (t[:, 0] - t[:, 1]))),
        "cos2(t0-t2)": (np.cos(2 * (a - c)), np.cos(2 * (t[:, 0] - t[:, 2]))),
        "cos(p t0)": (np.cos(2.5 * a), np.cos(2.5 * t[:, 0])),
        "sin^2 2t0": (np.sin(2 * a) ** 2, np.sin(2 * t[:, 0]) ** 2),
        "sin2t0 sin2t3": (np.sin(2 * a) * np.sin(2 * d), np.sin(2 * t[:, 0]) * np.sin(2 * t[:, 3])),
    }
    for name, (f_grid, f_samp) in checks.items():
        exact = (w * f_grid).sum()
        err = f_samp.std() / math.sqrt(f_samp.size / 4.0)
        assert abs(f_samp.mean() - exact) < 5 * err + 2e-3, (name, f_samp.mean(), exact, err)


def test_j0_observable_closed_forms():
    """J = 0 sites are independent: <M^2> = s2/N, <M^4> = (3(N-1)s2^2 + m4)/N^3 and
    <E> = T/2 + h<cos p theta>, with s2 = <sin^2 2t>, m4 = <sin^4 2t> by quadrature."""
    T = 2.0
    L = 4
    N = L * L
    cfg = inputs.config(L, L, 96, seed=3, J_par=0.0, J_perp=0.0, h=1.0, knots=([0], [T]))
    th = np.stack([oracle.init_theta(L, L, 0, r, 3, 0) for r in range(96)])
    om = np.zeros_like(th)
    step = [0]
    rec, mom = oracle.run_batch([cfg], [th], [om], step, 12000, record_every=20, t0=1000)
    assert step[0] == 12000
    p = lambda t: math.exp(-math.cos(2.5 * t) / T)
    Z = integrate.quad(p, -PI / 2, PI / 2)[0]
    s2 = integrate.quad(lambda t: p(t) * math.sin(2 * t) ** 2, -PI / 2, PI / 2)[0] / Z
    m4 = integrate.quad(lambda t: p(t) * math.sin(2 * t) ** 4, -PI / 2, PI / 2)[0] / Z
    cp = integrate.quad(lambda t: p(t) * math.cos(2.5 * t), -PI / 2, PI / 2)[0] / Z
    cnt = mom[0, 0]
    M2 = mom[0, 1] / cnt
    M4 = mom[0, 2] / cnt
    Emean = mom[0, 3] / cnt
    r = rec[0][:, 50:, :]
    Ms = r[:, :, 0].ravel()
    Es = r[:, :, 1].ravel()
    n_eff = Ms.size / 3.0
    assert M2 == pytest.approx(s2 / N, abs=5 * (Ms ** 2).std() / math.sqrt(n_eff))
    assert M4 == pytest.approx((3 * (N - 1) * s2 ** 2 + m4) / N ** 3, abs=5 * (Ms ** 4).std() / math.sqrt(n_eff))
    assert Emean == pytest.approx(T / 2 + cp, abs=5 * Es.std() / math.sqrt(n_eff))
    assert abs(mom[0, 5] / cnt - np.abs(Ms).mean()) < 1e-3


# ----------------------------------------------------------------- paper benchmarks


def _msd_closed_form(t, eta, T, w2, m=1.0):
    """Eq. (MSD-HO), evaluated in complex arithmetic (lambda_+- complex when eta < 2 omega)."""
    root = np.sqrt(complex(eta * eta - 4 * w2))
    lp, lm = 0.5 * (eta + root), 0.5 * (eta - root)
    pre = eta * T / (m * (lp - lm) ** 2)
    val = pre * ((lp + lm) / (lp * lm) + 4 / (lp + lm) * (np.exp(-(lp + lm) * t) - 1)
                 - np.exp(-2 * lp * t) / lp - np.exp(-2 * lm * t) / lm)
    return val.real


@pytest.mark.parametrize("dt", [0.05, 0.01])
@pytest.mark.parametrize("eta", [1.0, 5.0, 20.0])
def test_benchmark_harmonic_msd(dt, eta):
    """App. A.2 benchmark 1: omega^2 = 20, T = 20, m = 1, 1e5 paths."""
    n_paths = 100000
    t_end = 3.0
    n = int(round(t_end / dt))
    msd = oracle.harmonic_msd(n_paths, n, dt, eta, 20.0, 20.0)
    t = dt * np.arange(n + 1)
    exact = _msd_closed_form(t, eta, 20.0, 20.0)
    assert abs(exact[-1] - 1.0) < 0.02 or eta < 2  # T / omega^2 = 1 in the long-time limit
    # statistical error of a mean of x^2 over Gaussian paths, at the equilibrium scale
    # T / omega^2 = 1, plus an O(dt) allowance for the discretisation ("small
    # deviations" at dt = 0.05, Fig. 8): at early times the one-step scheme has an
    # O(1) relative error on a tiny value, so the bound is absolute
    sigma_eq = math.sqrt(2.0) * 1.0 / math.sqrt(n_paths)
    dev = np.abs(msd - exact)
    assert dev.max() < 5 * sigma_eq + 0.3 * dt, dev.max()
    assert np.mean(np.abs(msd[n // 2:] - exact[n // 2:]) / exact[n // 2:]) < 0.02


def test_benchmark_pair_cross_section():
    """App. A.2 benchmark 2 (Fig. 9): two sites, one bond J = 40, h = 100, p = 2.5,
    eta = 1, T = 100; theta_1 histogram (100 bins) in the slice theta_2 in
    [0.975, 1.125] against the canonical density.  A 2 x 1 periodic lattice
    counts the bond twice, so it runs with J_par = J / 2."""
    J, h, T = 40.0, 100.0, 100.0
    prm = dict(J_par=J / 2, J_perp=0.0, h=h, p=2.5)
    n_pairs = 1024
    Lx = 2 * n_pairs  # independent pairs side by side would couple; run them as replicas instead
    del Lx
    samples = []
    every = 100
    for r in range(n_pairs):
        th = oracle.init_theta(2, 1, 0, r, 11, 0)
        om = np.zeros(2)
        oracle.run_lattice(2, 1, 0, r, 11, prm, ([0], [T]), 0, 500, th, om)
        k = 500
        for _ in range(60):
            oracle.run_lattice(2, 1, 0, r, 11, prm, ([0], [T]), k, every, th, om)
            k += every
            samples.append(th.copy())
    s = np.array(samples)
    sel = (s[:, 1] >= 0.975) & (s[:, 1] <= 1.125)
    t1 = s[sel, 0]
    assert t1.size > 2000
    edges = np.linspace(-PI / 2, PI / 2, 101)
    hist, _ = np.histogram(t1, bins=edges)

    def dens(a, b):
        return integrate.dblquad(
            lambda t2, t1_: math.exp(-(-J * math.cos(2 * (t1_ - t2)) + h * math.cos(2.5 * t1_)
                                       + h * math.cos(2.5 * t2)) / T),
            a, b, 0.975, 1.125)[0]

    prob = np.array([dens(a, b) for a, b in zip(edges[:-1], edges[1:])])
    prob /= prob.sum()
    expect = prob * t1.size
    m = expect > 5
    chi2 = (((hist - expect) ** 2)[m] / expect[m]).sum() / m.sum()
    assert chi2 < 2.0, chi2
    # mean of theta_1 in the slice within 4 sigma
    mu = (prob * 0.5 * (edges[1:] + edges[:-1])).sum()
    assert abs(t1.mean() - mu) < 4 * t1.std() / math.sqrt(t1.size / 2)


# ----------------------------------------------------------------- resume and domains


def test_resume_is_bit_identical():
    L = 8
    cfg = dict(Lx=L, Ly=L, cfg=1, seed=5)
    th0 = inputs.angles(1, L, L, 4)[0].astype(np.float64)
    a_th, a_om = th0.copy(), np.zeros(L * L)
    rec_a = oracle.run_lattice(L, L, 1, 0, 5, {}, ([0, 300], [3.0, 1.0]), 0, 300, a_th, a_om, 7)
    b_th, b_om = th0.copy(), np.zeros(L * L)
    rec_b1 = oracle.run_lattice(L, L, 1, 0, 5, {}, ([0, 300], [3.0, 1.0]), 0, 113, b_th, b_om, 7)
    rec_b2 = oracle.run_lattice(L, L, 1, 0, 5, {}, ([0, 300], [3.0, 1.0]), 113, 187, b_th, b_om, 7)
    assert np.array_equal(a_th, b_th) and np.array_equal(a_om, b_om)
    assert np.array_equal(rec_a, np.concatenate([rec_b1, rec_b2]))
    del cfg


def _periodic_components(spins):
    Ly, Lx = spins.shape
    idx = np.arange(Lx * Ly).reshape(Ly, Lx)
    rows, cols = [], []
    for dy, dx in ((0, 1), (1, 0)):
        nb = np.roll(np.roll(idx, -dy, axis=0), -dx, axis=1)
        same = spins == np.roll(np.roll(spins, -dy, axis=0), -dx, axis=1)
        rows.append(idx[same])
        cols.append(nb[same])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    g = coo_matrix((np.ones(r.size), (r, c)), shape=(Lx * Ly, Lx * Ly))
    _, comp = connected_components(g, directed=False)
    # canonical label: smallest site index of each component
    mins = np.full(comp.max() + 1, Lx * Ly)
    np.minimum.at(mins, comp, np.arange(Lx * Ly))
    return mins[comp]


@pytest.mark.parametrize("case", ["random", "stripes_x", "stripes_y", "checker", "uniform", "spiral", "sparse"])
def test_ccl_against_graph_library(case):
    L = 24
    if case == "random":
        s = inputs.random_spins(L, L + 8, 4)
    elif case == "stripes_x":
        s = inputs.stripes(L, L, 3, 0)
    elif case == "stripes_y":
        s = inputs.stripes(L, L, 5, 1)
    elif case == "checker":
        s = inputs.checkerboard(L, L)
    elif case == "uniform":
        s = np.ones((L, L), dtype=np.int8)
    elif case == "spiral":
        s = inputs.spiral(L)
    else:
        s = inputs.random_spins(L, L, 9, p_up=0.1)
    Ly, Lx = s.shape
    th = inputs.spins_to_theta(s)
    lab, hist = oracle.ccl(Lx, Ly, th)
    ref = _periodic_components(s)
    assert np.array_equal(lab, ref.astype(np.int32))
    sizes = np.bincount(ref)[np.unique(ref)]
    vals, cnts = np.unique(sizes, return_counts=True)
    assert np.array_equal(hist, np.stack([vals, cnts], axis=1))
    assert hist[:, 0] @ hist[:, 1] == Lx * Ly
    if case == "checker":
        assert hist.tolist() == [[1, Lx * Ly]]
    if case == "uniform":
        assert hist.tolist() == [[Lx * Ly, 1]]
    if case == "stripes_x":
        # stripes of width 3 on a 24-periodic ring: 8 vertical bands, each one component
        assert hist.tolist() == [[3 * L, 8]]


def test_ccl_zero_angle_counts_as_up():
    th = np.array([0.0, -0.0, -1e-7, 1e-7], dtype=np.float32)
    lab, _ = oracle.ccl(4, 1, th)
    # theta >= 0 (both signed zeros) is up: sites 0,1,3 are up and 3-0 wrap
    assert lab.tolist() == [0, 0, 2, 0]


# ----------------------------------------------------------------- adjoint


def _fd_grad(Lx, Ly, prm, knots, n, th0, om0, wE, wM, rel=1e-5, field=None, couplings=None):
    names = ("J_par", "J_perp", "h", "eta")
    g = []
    for nm in names:
        base = prm[nm]
        eps = rel * max(1.0, abs(base))
        vals = []
        for s in (+1, -1):
            p2 = dict(prm)
            p2[nm] = base + s * eps
            obj, _, _, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, p2, knots, 0, n, th0, om0, wE, wM, field=field,
                                                  couplings=couplings)
            vals.append(obj)
        g.append((vals[0] - vals[1]) / (2 * eps))
    return np.array(g)


@pytest.mark.parametrize("wE,wM", [(1.0, 0.0), (0.0, 1.0), (0.7, 0.3)])
def test_adjoint_matches_finite_differences_smooth_field(wE, wM):
    """p = 2: cos(p theta) is pi-periodic, the dynamics is smooth, so the
    pathwise gradient equals central differences up to O(eps^2)."""
    Lx, Ly = 6, 4
    prm = dict(inputs.PAPER, J_par=2.0, J_perp=0.5, h=1.0, p=2.0, eta=0.8)
    th0 = inputs.angles(1, Lx, Ly, 8)[0].astype(np.float64)
    om0 = 0.3 * inputs.velocities(1, Lx, Ly, 8)[0].astype(np.float64)
    knots = ([0, 150], [1.0, 0.5])
    obj, grad, _, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, 150, th0, om0, wE, wM)
    fd = _fd_grad(Lx, Ly, prm, knots, 150, th0, om0, wE, wM)
    assert np.allclose(grad, fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fd).max())), (grad, fd)


def test_adjoint_matches_finite_differences_paper_field_low_T():
    """p = 2.5 away from the kink at +-pi/2: same agreement."""
    Lx, Ly = 8, 4
    prm = dict(inputs.PAPER, h=3.0)
    th0 = oracle.init_theta(Lx, Ly, 0, 0, 1, 1) + 0.05 * inputs.velocities(1, Lx, Ly, 2)[0]
    om0 = np.zeros(Lx * Ly)
    knots = ([0], [0.05])
    obj, grad, th1, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, 200, th0, om0, 1.0, 0.5)
    assert np.abs(th1).max() < PI / 2 - 0.1
    fd = _fd_grad(Lx, Ly, prm, knots, 200, th0, om0, 1.0, 0.5)
    assert np.allclose(grad, fd, rtol=1e-6, atol=1e-8 * max(1.0, np.abs(fd).max())), (grad, fd)


@pytest.mark.parametrize("field", [None, ([5, 30], [0.4, 2.5])])
def test_adjoint_forward_equals_stepper(field):
    """The adjoint's forward trajectory and objective are the stepper's (two
    loops written apart; with a field schedule each must give every time
    point its own field)."""
    Lx, Ly = 8, 8
    th0 = inputs.angles(1, Lx, Ly, 1)[0].astype(np.float64)
    om0 = np.zeros(Lx * Ly)
    knots = ([0], [inputs.T_C])
    obj, grad, th1, om1 = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, {}, knots, 0, 40, th0, om0, 0.6, 0.4, field=field)
    th, om = th0.copy(), om0.copy()
    oracle.run_lattice(Lx, Ly, 0, 0, 3, {}, knots, 0, 40, th, om, field=field)
    assert np.array_equal(th, th1) and np.array_equal(om, om1)
    # objective = sum over k = 1..n of the stepper's records
    th, om = th0.copy(), om0.copy()
    rec = oracle.run_lattice(Lx, Ly, 0, 0, 3, {}, knots, 0, 41, th, om, 1, field=field)
    expect = (0.6 * rec[1:, 1] + 0.4 * np.abs(rec[1:, 0])).sum()
    assert obj == pytest.approx(expect, rel=1e-13)


# ---------------------------------------------------------------- nonlinear quench schedule
# (Sec. V: eps(t) = t^gamma / tau_Q^gamma; gamma = 1 is Eq. Linear-Quench)

def test_power_quench_gamma_one_is_the_linear_ramp():
    Tc, kc, tq, ei, ef = 1.969, 500.0, 200.0, 0.5, -1.0
    power = {"power": (Tc, kc, tq, 1.0, ei, ef)}
    # the same ramp as knots: eps = +0.5 at k = kc - 0.5 tq, eps = -1 at k = kc + tq
    lin = ((int(kc - ei * tq), int(kc - ef * tq)), (Tc * (1 + ei), Tc * (1 + ef)))
    for k in (0, 350, 400, 401, 499, 500, 523, 650, 699, 700, 701, 5000):
        assert abs(oracle.temperature(k, power) - oracle.temperature(k, lin)) < 1e-12


@pytest.mark.parametrize("gamma", [2.0, 3.0])
def test_power_quench_closed_form(gamma):
    Tc, kc, tq, ei, ef = 2.0, 1000.0, 300.0, 0.6, -0.9
    sched = {"power": (Tc, kc, tq, gamma, ei, ef)}
    for k in (700, 900, 999, 1000, 1001, 1100, 1250):
        t = k - kc
        eps = -math.copysign(abs(t / tq) ** gamma, t) if t != 0 else 0.0
        eps = min(ei, max(ef, eps))
        assert abs(oracle.temperature(k, sched) - Tc * (1 + eps)) < 1e-12
    # clamped outside the ramp, continuous and non-increasing throughout
    ks = np.arange(0, 3000)
    T = np.array([oracle.temperature(int(k), sched) for k in ks])
    assert abs(T[0] - Tc * (1 + ei)) < 1e-12 and abs(T[-1] - Tc * (1 + ef)) < 1e-12
    assert np.all(np.diff(T) <= 1e-15)
    assert np.max(np.abs(np.diff(T))) < Tc * gamma * 1.5 / tq  # no jumps: |dT/dk| <= Tc gamma max|eps|^(1-1/gamma) / tq


# ---------------------------------------------------------------- path sensitivity (test infrastructure)


def _state_after(Lx, Ly, prm, knots, th0, om0, k0, j):
    th, om = th0.copy(), om0.copy()
    oracle.run_lattice(Lx, Ly, 0, 0, 5, prm, knots, k0, j, th, om)
    return th, om


def test_theta_sensitivity_matches_finite_differences():
    """lt_s(j) = d theta_t(n) / d theta_s(j) and lv_s(j) = d theta_t(n) /
    d wh_s(j) against central differences of the oracle's own trajectory:
    the angle perturbed after step j - 1 (the second half-kick of that step
    then sees the perturbed force), the half-step velocity of step j
    perturbed through omega_j (wh_j = (1 - a) omega_j + ...)."""
    Lx, Ly, n, k0 = 6, 4, 12, 3
    prm = dict(J_par=2.0, J_perp=0.7, h=1.0, p=2.0, eta=0.8, dt=0.02)
    knots = ([0], [0.2])
    rng = np.random.default_rng(5)
    th0 = rng.uniform(-0.5, 0.5, Lx * Ly)
    om0 = 0.3 * rng.standard_normal(Lx * Ly)
    target = 9
    _, lt, lv = oracle.theta_sensitivity(Lx, Ly, 0, 0, 5, prm, knots, k0, n, th0, om0, [target], fields=True)
    a = 0.5 * prm["eta"] * prm["dt"]
    eps = 1e-6
    for j, s in ((1, target), (4, target + 1), (7, 2), (n, target), (n, 3)):
        th_j, om_j = _state_after(Lx, Ly, prm, knots, th0, om0, k0, j)
        out = []
        for sgn in (1.0, -1.0):
            th_p, om_p = th_j.copy(), om_j.copy()
            th_p[s] += sgn * eps
            # omega_j was formed with F(theta_j): redo that half-kick's force term
            dF = oracle.force(Lx, Ly, prm, th_p) - oracle.force(Lx, Ly, prm, th_j)
            om_p += 0.5 * prm["dt"] * dF / (1 + a)
            th_e, om_e = _state_after(Lx, Ly, prm, knots, th_p, om_p, k0 + j, n - j)
            out.append(th_e[target])
        fd = (out[0] - out[1]) / (2 * eps)
        assert abs(fd - lt[j - 1, s]) <= 1e-6 * abs(fd) + 1e-9, (j, s, fd, lt[j - 1, s])
    for j, s in ((0, target), (3, target - 1), (6, 15), (n - 1, target)):
        th_j, om_j = _state_after(Lx, Ly, prm, knots, th0, om0, k0, j)
        out = []
        for sgn in (1.0, -1.0):
            om_p = om_j.copy()
            om_p[s] += sgn * eps / (1 - a)
            th_e, _ = _state_after(Lx, Ly, prm, knots, th_j.copy(), om_p, k0 + j, n - j)
            out.append(th_e[target])
        fd = (out[0] - out[1]) / (2 * eps)
        assert abs(fd - lv[j, s]) <= 1e-6 * abs(fd) + 1e-9, (j, s, fd, lv[j, s])


def test_theta_sensitivity_sums_and_free_rotor_closed_form():
    """J = h = 0 and T = 0: free damped rotors, theta_n = theta_j + dt sum_{m>=j} wh_m
    with wh_{m+1} = r wh_m, r = (1 - a) / (1 + a).  So lt_s(j) = delta_st and
    lv_t(j) = dt (1 - r^(n - j)) / (1 - r); the weighted sums follow in closed form."""
    Lx, Ly, n = 8, 2, 20
    prm = dict(J_par=0.0, J_perp=0.0, h=0.0, eta=1.5, dt=0.05)
    th0 = np.linspace(-1.0, 1.0, Lx * Ly)
    om0 = np.full(Lx * Ly, 0.1)
    t = 5
    a = 0.5 * 1.5 * 0.05
    r = (1 - a) / (1 + a)
    want_lv = np.array([0.05 * (1 - r ** (n - j)) / (1 - r) for j in range(n)])
    out, tth, tom, lt, lv = oracle.theta_sensitivity(Lx, Ly, 0, 0, 1, prm, ([0], [0.0]), 0, n, th0, om0, [t, 2],
                                                     trajectory=True, fields=True)
    np.testing.assert_allclose(lv[:, t], want_lv, rtol=1e-12)
    assert np.abs(np.delete(lv, t, axis=1)).max() == 0.0
    assert np.all(lt[:, t] == 1.0) and np.abs(np.delete(lt, t, axis=1)).max() == 0.0
    np.testing.assert_allclose(out[0], [n + want_lv.sum(), math.sqrt(n + (want_lv ** 2).sum())], rtol=1e-12)
    assert abs(out[1][0] - out[0][0]) < 1e-12  # another rotor, the same sums
    # the trajectory of a free rotor: omega_j = omega_0 r^j, theta_j = theta_0 + dt (1 - a) omega_0 (1 - r^j) / (1 - r)
    j = np.arange(n + 1)
    np.testing.assert_allclose(tom[:, t], 0.1 * r ** j, rtol=1e-12)
    np.testing.assert_allclose(tth[:, t], th0[t] + 0.05 * 0.1 * (1 - a) * (1 - r ** j) / (1 - r), rtol=1e-12)
    # weights: sum |l| w over the fields
    rng = np.random.default_rng(2)
    wt, wv = rng.random((n, Lx * Ly)), rng.random((n, Lx * Ly))
    out_w = oracle.theta_sensitivity(Lx, Ly, 0, 0, 1, prm, ([0], [0.0]), 0, n, th0, om0, [t], wt=wt, wv=wv)
    np.testing.assert_allclose(out_w[0], [wt[:, t].sum() + (want_lv * wv[:, t]).sum(),
                                          math.sqrt((wt[:, t] ** 2).sum() + ((want_lv * wv[:, t]) ** 2).sum())],
                               rtol=1e-12)


def test_first_order_bound_holds_for_binary32_state_rounding():
    """The propagation behind the parity tests' first-order bound, on the CPU:
    a run that rounds its state to binary32 after every step makes local
    errors of at most U |theta_j| in the angles and U |omega_j| in the
    full-step velocities (hence (1 - a) U |omega_j| in the next half-step
    velocity); after 100 steps from a random start at T_c every site must lie
    within sum |lambda| w of the exact run, and the sum must not be vacuous
    (within a factor 1000 of the largest deviation)."""
    Lx, Ly, n = 16, 12, 100
    prm = dict(inputs.PAPER)
    knots = ([0], [inputs.T_C])
    th0 = inputs.angles(1, Lx, Ly, seed=12)[0].astype(np.float64)
    om0 = np.zeros(Lx * Ly)
    U = 2.0 ** -24
    a = 0.5 * prm["eta"] * prm["dt"]
    ex_t, ex_w = th0.copy(), om0.copy()
    oracle.run_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, n, ex_t, ex_w)
    r_t, r_w = th0.copy(), om0.copy()
    for k in range(n):
        oracle.run_lattice(Lx, Ly, 0, 0, 3, prm, knots, k, 1, r_t, r_w)
        r_t[:] = r_t.astype(np.float32)
        r_w[:] = r_w.astype(np.float32)
    d = np.abs(r_t - ex_t) % math.pi
    d = np.minimum(d, math.pi - d)
    _, tth, tom = oracle.theta_sensitivity(Lx, Ly, 0, 0, 3, prm, knots, 0, n, th0, om0, [], trajectory=True)
    wt = U * np.abs(tth[1:])
    wv = (1 - a) * U * np.abs(tom[:n])
    wv[0] = 0.0  # the start is exact
    sites = np.arange(Lx * Ly)
    bound = oracle.theta_sensitivity(Lx, Ly, 0, 0, 3, prm, knots, 0, n, th0, om0, sites, wt=wt, wv=wv)[:, 0]
    assert np.all(d <= bound), (d / bound).max()
    assert d.max() > 1e-3 * bound.max()



# ---------------------------------------------------------------- field schedule (orthogonal quench)


def test_field_schedule_is_linear_interpolation():
    """s(k) through the knots and constant outside them: numpy's interpolation
    of the same knots, at the knots, between them and beyond both ends."""
    field = ([10, 40, 41, 200], [0.5, 2.0, -1.0, 3.25])
    ks = np.arange(-5, 260)
    got = np.array([oracle.field_scale(int(k), field) for k in ks])
    want = np.interp(ks.astype(np.float64), np.array(field[0], dtype=np.float64), np.array(field[1]))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    assert oracle.field_scale(123, None) == 1.0


def test_field_schedule_scales_the_field_exactly():
    """A schedule of ones changes nothing, and a constant scale 2 with h = 1
    is the run with h = 2 (h s(k) enters the force and the energy exactly)."""
    Lx, Ly, n = 8, 6, 60
    prm = dict(inputs.PAPER)
    knots = ([0], [inputs.T_C])
    th0 = inputs.angles(1, Lx, Ly, 4)[0].astype(np.float64)
    runs = []
    for p_, field in ((prm, None), (prm, ([0, 30], [1.0, 1.0])), (dict(prm, h=0.5), ([0], [2.0])),
                      (dict(prm, h=1.0), None)):
        th, om = th0.copy(), np.zeros(Lx * Ly)
        rec = oracle.run_lattice(Lx, Ly, 0, 0, 7, p_, knots, 0, n, th, om, record_every=5, field=field)
        runs.append((th, om, rec))
    for a, b in ((0, 1), (2, 3)):
        assert all(np.array_equal(x, y) for x, y in zip(runs[a], runs[b]))


def test_single_angle_boltzmann_at_the_held_field():
    """J = 0: a ramp of the field from 0.25 h to 2 h over 400 steps, then held:
    the angles follow exp(-2 h cos(p theta) / T) of the field now applied."""
    T, h = 1.0, 1.0
    prm = dict(J_par=0.0, J_perp=0.0, h=h)
    field = ([0, 400], [0.25, 2.0])
    Lx, Ly = 32, 32
    th = oracle.init_theta(Lx, Ly, 0, 0, 9, 0)
    om = np.zeros(Lx * Ly)
    oracle.run_lattice(Lx, Ly, 0, 0, 9, prm, ([0], [T]), 0, 900, th, om, field=field)
    samples, k = [], 900
    while k < 900 + 8000:
        oracle.run_lattice(Lx, Ly, 0, 0, 9, prm, ([0], [T]), k, 40, th, om, field=field)
        k += 40
        samples.append(th.copy())
    x = np.array(samples).ravel()
    edges = np.linspace(-PI / 2, PI / 2, 41)
    hist, _ = np.histogram(x, bins=edges)
    dens = lambda t: math.exp(-2.0 * h * math.cos(2.5 * t) / T)
    Z = integrate.quad(dens, -PI / 2, PI / 2)[0]
    expect = np.array([integrate.quad(dens, a, b)[0] / Z for a, b in zip(edges[:-1], edges[1:])]) * x.size
    z = (hist - expect) / np.sqrt(4 * expect)
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    # and not the distribution of the starting field 0.25 h
    dens0 = lambda t: math.exp(-0.25 * h * math.cos(2.5 * t) / T)
    Z0 = integrate.quad(dens0, -PI / 2, PI / 2)[0]
    exp0 = np.array([integrate.quad(dens0, a, b)[0] / Z0 for a, b in zip(edges[:-1], edges[1:])]) * x.size
    assert np.abs((hist - exp0) / np.sqrt(4 * exp0)).max() > 10.0


def test_adjoint_with_field_schedule_matches_finite_differences():
    """p = 2 (smooth) with a field ramp and a temperature ramp: d/dh at the
    fixed profile s(k) and the other three components against central
    differences."""
    Lx, Ly = 6, 4
    prm = dict(inputs.PAPER, J_par=2.0, J_perp=0.5, h=1.2, p=2.0, eta=0.8)
    th0 = inputs.angles(1, Lx, Ly, 18)[0].astype(np.float64)
    om0 = 0.3 * inputs.velocities(1, Lx, Ly, 18)[0].astype(np.float64)
    knots = ([0, 150], [1.0, 0.5])
    field = ([20, 120], [0.3, 1.7])
    obj, grad, _, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, 150, th0, om0, 0.6, 0.4, field=field)
    fd = _fd_grad(Lx, Ly, prm, knots, 150, th0, om0, 0.6, 0.4, field=field)
    assert np.allclose(grad, fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fd).max())), (grad, fd)
    # the schedule matters: without it d/dh differs
    _, g1, _, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, 150, th0, om0, 0.6, 0.4)
    assert abs(g1[2] - grad[2]) > 1e-3 * abs(grad[2])


# ---------------------------------------------------------------- anisotropic quench: coupling profiles
# (Sec. V: the two directional couplings quenched at different
# rates, J_par(k) = J_par a(k), J_perp(k) = J_perp b(k))

def test_coupling_schedule_scales_the_couplings_exactly():
    """Profiles of ones change nothing; constant scales a = 2, b = 1/2 are the
    run with J_par doubled and J_perp halved (both enter the force and the
    energy exactly), and swapping the two profiles is a different run."""
    Lx, Ly, n = 8, 6, 60
    prm = dict(inputs.PAPER)
    knots = ([0], [inputs.T_C])
    th0 = inputs.angles(1, Lx, Ly, 4)[0].astype(np.float64)
    runs = []
    for p_, cpl in ((prm, None), (prm, ([0, 30], [1.0, 1.0], [1.0, 1.0])),
                    (prm, ([0], [2.0], [0.5])), (dict(prm, J_par=2 * prm["J_par"], J_perp=0.5 * prm["J_perp"]), None),
                    (prm, ([0], [0.5], [2.0]))):
        th, om = th0.copy(), np.zeros(Lx * Ly)
        rec = oracle.run_lattice(Lx, Ly, 0, 0, 7, p_, knots, 0, n, th, om, record_every=5, couplings=cpl)
        runs.append((th, om, rec))
    for a, b in ((0, 1), (2, 3)):
        assert all(np.array_equal(x, y) for x, y in zip(runs[a], runs[b]))
    assert not np.array_equal(runs[2][0], runs[4][0])


def test_coupling_ramp_gives_every_time_point_its_couplings():
    """The adjoint's forward loop and the stepper give every time point its
    own couplings: the same trajectory and objective under a ramp of both."""
    Lx, Ly = 8, 8
    th0 = inputs.angles(1, Lx, Ly, 1)[0].astype(np.float64)
    om0 = np.zeros(Lx * Ly)
    knots = ([0], [inputs.T_C])
    cpl = ([5, 30], [1.0, 0.3], [0.2, 3.0])
    obj, _, th1, om1 = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, {}, knots, 0, 40, th0, om0, 0.6, 0.4, couplings=cpl)
    th, om = th0.copy(), om0.copy()
    rec = oracle.run_lattice(Lx, Ly, 0, 0, 3, {}, knots, 0, 41, th, om, 1, couplings=cpl)
    th, om = th0.copy(), om0.copy()
    oracle.run_lattice(Lx, Ly, 0, 0, 3, {}, knots, 0, 40, th, om, couplings=cpl)
    assert np.array_equal(th, th1) and np.array_equal(om, om1)
    expect = (0.6 * rec[1:, 1] + 0.4 * np.abs(rec[1:, 0])).sum()
    assert obj == pytest.approx(expect, rel=1e-13)


def test_adjoint_with_coupling_schedule_matches_finite_differences():
    """p = 2 (smooth), both couplings ramped at different rates together with
    a temperature ramp and a field ramp: d/dJ_par and d/dJ_perp at the fixed
    profiles, and the other two components, against central differences."""
    Lx, Ly = 6, 4
    prm = dict(inputs.PAPER, J_par=2.0, J_perp=0.5, h=1.2, p=2.0, eta=0.8)
    th0 = inputs.angles(1, Lx, Ly, 28)[0].astype(np.float64)
    om0 = 0.3 * inputs.velocities(1, Lx, Ly, 28)[0].astype(np.float64)
    knots = ([0, 150], [1.0, 0.5])
    field = ([20, 120], [0.3, 1.7])
    cpl = ([10, 90, 140], [1.5, 0.6, 1.0], [0.4, 2.2, 1.3])
    obj, grad, _, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, 150, th0, om0, 0.6, 0.4, field=field,
                                             couplings=cpl)
    fd = _fd_grad(Lx, Ly, prm, knots, 150, th0, om0, 0.6, 0.4, field=field, couplings=cpl)
    assert np.allclose(grad, fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fd).max())), (grad, fd)
    # the profiles matter: without them d/dJ differ
    _, g1, _, _ = oracle.adjoint_lattice(Lx, Ly, 0, 0, 3, prm, knots, 0, 150, th0, om0, 0.6, 0.4, field=field)
    assert abs(g1[0] - grad[0]) > 1e-3 * abs(grad[0]) and abs(g1[1] - grad[1]) > 1e-3 * abs(grad[1])
