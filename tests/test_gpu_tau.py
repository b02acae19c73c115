"""GPU autocorrelation times (xy_autocorr_time) against the oracle
(oracle/tau.py, App. B) on the same series: synthetic AR(1) series with
known tau and the records of a lattice run."""
import numpy as np
import pytest
import torch

from oracle import tau as otau
from paper_2409_06412_gb300 import Config, Lattice, XYError
from paper_2409_06412_gb300 import sampling
from tests.inputs import ar1_series

pytestmark = pytest.mark.gpu


def as_records(series_M, series_E=None):
    B, n = series_M.shape
    r = np.zeros((B, n, 2))
    r[:, :, 0] = series_M
    r[:, :, 1] = series_E if series_E is not None else -series_M
    return torch.from_numpy(r).cuda()


def oracle_row(f, c=6.0):
    window = "auto" if c > 0 else "half"
    C0 = otau.autocorrelation(f, 0)[0]
    return np.array([f.mean(), C0, otau.tau_int(f, window, c), otau.error_of_mean(f, window, c)])


@pytest.mark.parametrize("phi,n,c", [(0.5, 3000, 6.0), (0.95, 20000, 6.0), (0.3, 1001, 0.0), (0.9, 777, 4.0)])
def test_ar1_series_match_oracle(phi, n, c):
    x = ar1_series(n, phi, seed=int(phi * 100) + n, n_series=5) * 0.3 + 0.1
    out = sampling.autocorr_time(as_records(x), "M", "f", 0, n, c).cpu().numpy()
    for b in range(5):
        ref = oracle_row(x[b], c)
        np.testing.assert_allclose(out[b, :2], ref[:2], rtol=1e-12, atol=1e-14)
        assert abs(out[b, 2] - ref[2]) < 1e-4 * max(1.0, abs(ref[2])), (out[b], ref)
        if ref[2] > 1e-3:  # the literal half window can sum to tau <= 0, where sigma_mean is undefined
            assert abs(out[b, 3] / ref[3] - 1) < 1e-4


@pytest.mark.parametrize("transform,g", [("f2", lambda v: v * v), ("f4", lambda v: v ** 4), ("abs", np.abs)])
def test_transforms_and_second_component(transform, g):
    x = ar1_series(2048, 0.7, seed=4, n_series=3)
    e = ar1_series(2048, 0.2, seed=5, n_series=3)
    rec = as_records(x, e)
    out = sampling.autocorr_time(rec, "M", transform, 100, 1500).cpu().numpy()
    for b in range(3):
        ref = oracle_row(g(x[b, 100:1600]))
        np.testing.assert_allclose(out[b, :2], ref[:2], rtol=1e-12)
        assert abs(out[b, 2] - ref[2]) < 1e-4 * max(1.0, ref[2])
    outE = sampling.autocorr_time(rec, "E").cpu().numpy()
    for b in range(3):
        ref = oracle_row(e[b])
        assert abs(outE[b, 2] - ref[2]) < 1e-4 * max(1.0, ref[2])


def test_records_of_a_run_and_host_output():
    lat = Lattice([Config(Lx=32, Ly=32, n_replicas=4, seed=2, init_mode=1, knots=((0,), (1.969,)),
                          n_total=10 ** 6)])
    rec = lat.step(4000, record_every=10)
    R = rec.shape[1]
    n = R - 1  # the last slot of a window ending between records stays empty
    rec = rec[:, :n].contiguous()
    out = sampling.autocorr_time(rec, "M", "f2", 50).cpu().numpy()
    h = rec.cpu().numpy()
    for b in range(4):
        ref = oracle_row(h[b, 50:, 0] ** 2)
        np.testing.assert_allclose(out[b, :2], ref[:2], rtol=1e-12)
        assert abs(out[b, 2] - ref[2]) < 1e-4 * max(1.0, ref[2])
    host = np.zeros((4, 4))
    from paper_2409_06412_gb300 import _lib
    import ctypes
    _lib.call("xy_autocorr_time", ctypes.c_void_p(rec.data_ptr()), 4, n, 0, 1, 50, n - 50, 6.0,
              host.ctypes.data_as(ctypes.c_void_p), None)
    np.testing.assert_array_equal(host, out)
    assert sampling.suggest_record_every(out[0, 2], 10) >= 100


def test_bad_arguments_are_rejected():
    rec = as_records(np.zeros((2, 10)))
    with pytest.raises(XYError):
        sampling.autocorr_time(rec, "M", "f", 5, 6)   # skip + n > R
    with pytest.raises(XYError):
        sampling.autocorr_time(rec, "M", "f", 0, 1)   # n < 2
