"""xy_label_domains_static: domain labelling with no allocation.

Callers whose memory pool owns the whole GPU, or that cannot afford an
allocation or cudaFree's synchronisation, label domains with this entry
point: it uses a fixed working array inside the library instead of
cudaMalloc.  It must give exactly what xy_label_domains gives (labels, size
histogram, number of sizes are integers, so the comparison is bit-exact, the
same bar as the other labelling tests), including on a second call right
after the first, since the working array keeps the previous call's contents.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_06412_gb300 import _lib, build
from tests import inputs
from tests.gpu_helpers import make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _reference(lat, b_first, b_count, hist_cap):
    labels, hist, n_sizes = lat.label_domains(b_first, b_count, hist_cap=hist_cap)
    torch.cuda.synchronize()
    return labels, hist, n_sizes


def _static(theta, Lx, Ly, n_lat, hist_cap):
    N = Lx * Ly
    labels = torch.full((n_lat, N), -7, dtype=torch.int32, device="cuda")
    hist = torch.full((n_lat, hist_cap, 2), -7, dtype=torch.int64, device="cuda")
    n_sizes = torch.full((n_lat,), -7, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    rc = _lib.load().xy_label_domains_static(ctypes.c_void_p(theta.data_ptr()), Lx, Ly, n_lat,
                                             ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(hist.data_ptr()),
                                             hist_cap, ctypes.c_void_p(n_sizes.data_ptr()),
                                             ctypes.c_void_p(st.cuda_stream))
    assert rc == _lib.XY_OK, _lib.load().xy_last_error()
    return labels, hist, n_sizes


def _batch(kind, Lx, Ly, n, seed):
    if kind == "random":
        s = [inputs.random_spins(Lx, Ly, seed + i) for i in range(n)]
    elif kind == "sparse":
        s = [inputs.random_spins(Lx, Ly, seed + i, p_up=0.1) for i in range(n)]
    else:
        s = [inputs.stripes(Lx, Ly, 2 + i, i % 2) for i in range(n)]
    return np.stack([inputs.spins_to_theta(x).ravel() for x in s])


def test_static_labelling_matches_allocating_entry_point_twice():
    # first call: 4 random-spin lattices of 256 x 128
    th1 = _batch("random", 256, 128, 4, 10)
    lat1, _, _ = make_pair([inputs.config(256, 128, 4)], [th1])
    ref1 = _reference(lat1, 0, 4, 4096)
    got1 = _static(lat1.theta, 256, 128, 4, 4096)
    # second call, right after, on other shapes and patterns: nothing of the
    # first call's working memory may leak into it
    th2 = np.concatenate([_batch("stripes", 64, 32, 3, 0), _batch("sparse", 64, 32, 2, 5)])
    lat2, _, _ = make_pair([inputs.config(64, 32, 5)], [th2])
    ref2 = _reference(lat2, 0, 5, 1024)
    got2 = _static(lat2.theta, 64, 32, 5, 1024)
    torch.cuda.synchronize()
    for ref, got in ((ref1, got1), (ref2, got2)):
        for r, g in zip(ref, got):
            assert torch.equal(r, g)


def test_static_labelling_at_the_size_limit():
    """Exactly XY_STATIC_CCL_MAX_SITES sites in several lattices (8 of 512 x
    512): the far end of the working array (the last lattices' size counts
    and the error word after them) is in use, and the result is still
    bit-identical to the allocating entry point's, on two calls in a row."""
    n, L = 8, 512
    assert n * L * L == _lib.XY_STATIC_CCL_MAX_SITES
    th = np.concatenate([_batch("random", L, L, n // 2, 30), _batch("sparse", L, L, n // 2, 40)])
    lat, _, _ = make_pair([inputs.config(L, L, n)], [th])
    ref = _reference(lat, 0, n, 1 << 14)
    for _ in range(2):
        got = _static(lat.theta, L, L, n, 1 << 14)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            assert torch.equal(r, g)


def test_static_labelling_rejects_host_pointers():
    lib = _lib.load()
    theta_h = np.zeros(64, dtype=np.float32)
    labels_d = torch.zeros(64, dtype=torch.int32, device="cuda")
    theta_d = torch.zeros(64, dtype=torch.float32, device="cuda")
    labels_h = np.zeros(64, dtype=np.int32)
    for th, lab in ((theta_h.ctypes.data, labels_d.data_ptr()), (theta_d.data_ptr(), labels_h.ctypes.data)):
        rc = lib.xy_label_domains_static(ctypes.c_void_p(th), 8, 8, 1, ctypes.c_void_p(lab), None, 0, None, None)
        assert rc == _lib.XY_EINVAL
        assert b"device memory" in lib.xy_last_error()
    hist_h = np.zeros((1, 4, 2), dtype=np.int64)
    rc = lib.xy_label_domains_static(ctypes.c_void_p(theta_d.data_ptr()), 8, 8, 1, ctypes.c_void_p(labels_d.data_ptr()),
                                     ctypes.c_void_p(hist_h.ctypes.data), 4, None, None)
    assert rc == _lib.XY_EINVAL


def test_static_labelling_rejects_oversize_calls():
    lib = _lib.load()
    theta = torch.zeros(16, dtype=torch.float32, device="cuda")
    labels = torch.zeros(16, dtype=torch.int32, device="cuda")
    too_many = _lib.XY_STATIC_CCL_MAX_SITES // (1024 * 1024) + 1
    rc = lib.xy_label_domains_static(ctypes.c_void_p(theta.data_ptr()), 1024, 1024, too_many,
                                     ctypes.c_void_p(labels.data_ptr()), None, 0, None, None)
    assert rc == _lib.XY_EINVAL
    assert b"XY_STATIC_CCL_MAX_SITES" in lib.xy_last_error()
