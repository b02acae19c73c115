"""GPU structure factors (xy_structure_factor) against the oracle's literal
2-D transform (App. C, Eq. S-as-lattice-FT), element by element."""
import numpy as np
import pytest
import torch

from oracle import corrlen as ocl
from paper_2409_06412_gb300 import PAPER_PARAMS, XY_INIT_USER, Config, Lattice, XYError
from paper_2409_06412_gb300 import corrlen
from tests.inputs import angles, ar1_field

pytestmark = pytest.mark.gpu


def lattice_from(shapes_thetas):
    cfgs, ths = [], []
    for (Lx, Ly, th) in shapes_thetas:
        th = np.asarray(th, dtype=np.float32).reshape(-1, Ly * Lx)
        cfgs.append(Config(Lx=Lx, Ly=Ly, n_replicas=th.shape[0], seed=3, init_mode=XY_INIT_USER,
                           params=dict(PAPER_PARAMS), knots=((0,), (1.969,)), n_total=10 ** 6))
        ths.append(th.reshape(-1))
    t = torch.from_numpy(np.concatenate(ths)).cuda()
    return Lattice(cfgs, theta=t, omega=torch.zeros_like(t))


def check(S_gpu, S_ref, N):
    S_gpu = S_gpu.cpu().numpy()
    # FP32 line sums of unit-bounded terms: relative 1e-5 of the largest value
    tol = 2e-5 * max(1.0, float(np.max(np.abs(S_ref)))) + 1e-6
    assert np.max(np.abs(S_gpu - S_ref)) < tol, (np.max(np.abs(S_gpu - S_ref)), tol)


@pytest.mark.parametrize("Lx,Ly,n,K,r", [
    (64, 64, 2, 16, 1.0),
    (256, 128, 1, 13, 1.0),   # Lx > 128, non-square, a partial group of wavenumbers
    (12, 20, 3, 12, 2.0),     # rows narrower than a warp, doubled angle
    (1024, 32, 1, 32, 1.0),   # long rows, K = Ly
    (40, 8, 2, 1, 1.0),       # K = 1
])
def test_structure_factor_matches_oracle(Lx, Ly, n, K, r):
    th = angles(n, Lx, Ly, seed=Lx + Ly).reshape(n, Ly, Lx)
    lat = lattice_from([(Lx, Ly, th)])
    S_par, S_perp = lat.structure_factor(0, n, K, r)
    o_par, o_perp = ocl.structure_factor(th.astype(np.float64), r)
    check(S_par, o_par[:, :K], Lx)
    check(S_perp, o_perp[:, :K], Ly)


def test_mixed_shapes_in_one_call_and_host_outputs():
    a = angles(2, 64, 32, seed=1).reshape(2, 32, 64)
    b = np.full((1, 16, 16), 0.7, dtype=np.float32)                 # ordered: S(0) = N, else 0
    x = np.arange(128)
    c = np.tile(np.float32(2 * np.pi * 3 * x / 128 - np.pi), (1, 8, 1)).reshape(1, 8, 128)  # wave k = 3
    c = ((c + np.pi / 2) % np.pi - np.pi / 2).astype(np.float32)    # as a stored angle, rotor r = 2 sees k = 6
    lat = lattice_from([(64, 32, a), (16, 16, b), (128, 8, c)])
    K = 8
    S_par, S_perp = lat.structure_factor(0, 4, K, 1.0)
    refs = [ocl.structure_factor(t.astype(np.float64), 1.0) for t in (a[0], a[1], b[0], c[0])]
    for i, (rp, rq) in enumerate(refs):
        check(S_par[i], rp[:K], 0)
        check(S_perp[i], rq[:K], 0)
    assert abs(S_par[2, 0].item() - 16) < 1e-4 and float(S_par[2, 1:].abs().max()) < 1e-6
    # the same through host buffers
    hp = np.zeros((4, K))
    hq = np.zeros((4, K))
    from paper_2409_06412_gb300 import _lib
    _lib.call("xy_structure_factor", lat._h, 0, 4, K, 1.0, hp.ctypes.data, hq.ctypes.data)
    np.testing.assert_array_equal(hp, S_par.cpu().numpy())
    np.testing.assert_array_equal(hq, S_perp.cpu().numpy())
    # the doubled angle of the wave lattice peaks at k = 6
    S6, _ = lat.structure_factor(3, 1, 8, 2.0)
    assert int(np.argmax(S6[0].cpu().numpy())) == 6


def test_structure_factor_rejects_bad_arguments():
    lat = lattice_from([(16, 8, angles(1, 16, 8, seed=2))])
    with pytest.raises(XYError):
        lat.structure_factor(0, 1, 9)   # K > min(Lx, Ly)
    with pytest.raises(XYError):
        lat.structure_factor(0, 2, 4)   # range past the last lattice


def test_correlation_length_of_correlated_rows():
    # exponentially correlated rows (xi_par = sqrt(rho)/(1 - rho) ~ 9.5), uncorrelated columns
    rho, eps = 0.9, 0.05
    th = np.stack([eps * ar1_field(512, 128, rho, seed=100 + b) for b in range(8)]).astype(np.float32)
    lat = lattice_from([(512, 128, th)])
    S_par, S_perp = lat.structure_factor(0, 8, 16, 1.0)
    o_par, o_perp = ocl.structure_factor(th.astype(np.float64))
    check(S_par, o_par[:, :16], 512)
    xi_par, xi_perp = corrlen.correlation_lengths(S_par, S_perp, 512, 128, 1, 12)
    _, xi_o = ocl.fit_lorentzian(o_par.mean(axis=0), 512, 1, 12, form="lattice")
    assert abs(xi_par / xi_o - 1) < 1e-3
    assert abs(xi_par / (np.sqrt(rho) / (1 - rho)) - 1) < 0.10
    assert np.isnan(xi_perp) or xi_perp < 1.0  # uncorrelated columns: no decay, or a length below a site


def test_correlation_length_below_one_site():
    """Periodic AR(1) columns with rho = 0.3 (xi_perp = sqrt(rho)/(1 - rho) =
    0.78): S_perp over the whole half zone from the GPU, the window chosen
    from the data; the fit agrees with the oracle's fit of the oracle's
    S_perp on the same window and finds the generating length."""
    rho, eps, L = 0.3, 0.05, 256
    th = np.stack([eps * ar1_field(L, L, rho, seed=200 + b, axis=0) for b in range(8)]).astype(np.float32)
    lat = lattice_from([(L, L, th)])
    K = L // 2
    S_par, S_perp = lat.structure_factor(0, 8, K, 1.0)
    o_par, o_perp = ocl.structure_factor(th.astype(np.float64))
    check(S_perp, o_perp[:, :K], L)
    _, xi, (lo, hi) = corrlen.fit_lorentzian(S_perp.cpu().numpy().mean(axis=0), L, return_window=True)
    _, xi_o = ocl.fit_lorentzian(o_perp.mean(axis=0)[:K], L, lo, hi, form="lattice")
    assert abs(xi / xi_o - 1) < 1e-3, (xi, xi_o, lo, hi)
    assert abs(xi / (np.sqrt(rho) / (1 - rho)) - 1) < 0.10, xi
    assert np.isnan(corrlen.correlation_lengths(S_par, S_perp, L, L)[0])  # rows uncorrelated: no length


def test_full_size_lattice_after_dynamics():
    # a 1024 x 1024 lattice after 200 steps at T_c from the ordered state
    lat = Lattice([Config(Lx=1024, Ly=1024, n_replicas=1, seed=1, init_mode=1, knots=((0,), (1.969,)),
                          n_total=10 ** 6)])
    lat.step(200)
    S_par, S_perp = lat.structure_factor(0, 1, 24, 1.0)
    th = lat.theta.cpu().numpy().reshape(1024, 1024).astype(np.float64)
    o_par, o_perp = ocl.structure_factor(th)
    check(S_par[0], o_par[:24], 1024)
    check(S_perp[0], o_perp[:24], 1024)
