"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs and identical counter-based noise.

Tolerances (stated by the method's specification): max circular |dtheta| <=
1e-4 rad after 100 steps; observables, moments and the full-step velocity are
checked at FP32 accuracy; domain labels bit-exact; adjoint gradients within
1e-3 relative of the oracle's FP64 adjoint.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest
import torch

import oracle
from paper_2409_06412_gb300 import (XY_ADJOINT_AUTO, XY_ADJOINT_BACKWARD, XY_ADJOINT_RECOMPUTE, XY_PATH_BATCHED,
                                    XY_PATH_PLAIN, XYError, build, debug_noise, debug_philox)
from paper_2409_06412_gb300.lattice import Config, Lattice
from tests import inputs
from tests.gpu_helpers import (assert_grads_close, circ_diff, inputs_params, make_pair, parity_report, split_state,
                               stepwise_parity, theta_parity)

pytestmark = pytest.mark.gpu
PI = math.pi
TC = inputs.T_C


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()


# ------------------------------------------------------------------ noise


def _counters(n, seed=0):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    c[:16] = 0
    c[16:32] = 0xFFFFFFFF
    c[:32, 0] = np.arange(32)
    return c


def test_philox_bits_match_oracle():
    total = 0
    for chunk in range(6):
        c = _counters(1 << 24, seed=chunk)
        key = (0x9E3779B9 + chunk, 0xDEADBEEF ^ chunk)
        g = debug_philox(torch.from_numpy(c.view(np.int32)).cuda(), *key).cpu().numpy().view(np.uint32)
        o = oracle.philox(c, key)
        assert np.array_equal(g, o), f"chunk {chunk}: {np.argwhere(g != o)[:4]}"
        total += c.shape[0]
    assert total >= 10 ** 8


def test_philox_bits_match_curand():
    """Independent implementation: cuRAND's Philox4x32-10 block function."""
    src = os.path.join(os.path.dirname(__file__), "cuda", "curand_philox_ref.cu")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "curand_ref.so")
    subprocess.check_call([build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, src])
    ref = ctypes.CDLL(so)
    ref.curand_philox_ref.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                      ctypes.c_void_p]
    c = _counters(1 << 22, seed=99)
    key = (12345, 678910)
    ct = torch.from_numpy(c.view(np.int32)).cuda()
    out = torch.empty_like(ct)
    torch.cuda.synchronize()
    assert ref.curand_philox_ref(ct.data_ptr(), key[0], key[1], c.shape[0], out.data_ptr()) == 0
    mine = debug_philox(ct, *key)
    torch.cuda.synchronize()
    assert torch.equal(mine, out)
    # and the oracle's
    assert np.array_equal(oracle.philox(c[:65536], key), out[:65536].cpu().numpy().view(np.uint32))


def test_gaussians_match_oracle():
    n_quads = 1 << 18
    words, g = debug_noise(7, 3, 5, 123456789012, 0, n_quads)
    o = oracle.gauss(7, 3, 5, 4 * n_quads, 123456789012)
    g = g.cpu().numpy().astype(np.float64)
    d = np.abs(g - o)
    # FP32 Box-Muller with the hardware log2 (absolute error 2^-22 near 1):
    # the radius error is ~3e-7 / r, so tiny radii carry larger absolute error
    w = words.cpu().numpy().view(np.uint32)
    u0 = ((w[:, [0, 0, 2, 2]] >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    r = np.sqrt(-2 * np.log(u0)).ravel()
    tol = 4e-6 * (1 + np.abs(o)) + 4e-7 / r
    assert np.all(d <= tol), (d / tol).max()
    assert np.quantile(d, 0.9999) < 2e-5


# ------------------------------------------------------------------ init


def test_init_modes_match_oracle():
    cfgs = [Config(Lx=64, Ly=32, n_replicas=3, seed=11, init_mode=0),
            Config(Lx=128, Ly=8, n_replicas=2, seed=12, init_mode=1)]
    lat = Lattice(cfgs)
    torch.cuda.synchronize()
    th = split_state(lat, lat.theta)
    for r in range(3):
        o = oracle.init_theta(64, 32, 0, r, 11, 0)
        assert circ_diff(th[0][r], o).max() < 1e-6
    assert np.all(th[1] == np.float32(2 * PI / 5))
    assert torch.all(lat.omega == 0)


# ------------------------------------------------------------------ stepping parity

MIXED = [
    # (Lx, Ly, n_rep): kernel chosen by the batched path
    (64, 64, 1),     # resident, 1024 threads, one row per band
    (128, 128, 2),   # resident, 1024 threads, 4 rows per band
    (256, 64, 2),    # strip, 2 strips per row, edge columns from global memory
    (32, 2048, 1),   # strip, 4 row groups per warp (sub-warp shuffles)
    (128, 256, 1),   # strip, full-row warps
    (12, 10, 2),     # plain (ragged width)
    (4, 1, 3),       # plain (degenerate: self-neighbours in y, x wraps onto the quad)
    (132, 6, 1),     # plain (width not a multiple of 128)
]


def _mixed_specs(T=TC, n_total=10 ** 9, **prm):
    return [inputs.config(Lx, Ly, n, seed=1 + i, n_total=n_total, knots=([0], [T]), **prm)
            for i, (Lx, Ly, n) in enumerate(MIXED)]


def _mixed_thetas(specs, seed=5):
    return [inputs.angles(s["n_rep"], s["Lx"], s["Ly"], seed + i) for i, s in enumerate(specs)]


@pytest.mark.parametrize("path", [XY_PATH_BATCHED, XY_PATH_PLAIN])
def test_mixed_batch_parity_100_steps(path):
    """100 steps: every site within 1e-4 rad of the oracle except sites near a
    cusp event (the FP32 and FP64 angles on opposite sides of the wrap cut at
    +-pi/2, where the field force jumps); such events are listed."""
    specs = _mixed_specs()
    thetas = _mixed_thetas(specs)
    lat, o_th, o_om = make_pair(specs, thetas, path=path)
    res = stepwise_parity(lat, specs, o_th, o_om, 100)
    assert res["step_now"] == [100] * len(specs)
    report = parity_report(res)
    print(report)
    for rec in res["ill"]:
        print("  FP32-conditioned (config, replica, site, |dtheta|, bound, rms):", rec)
    assert not res["unexplained"], (res["unexplained"][:10], report)
    assert res["frac_within_tol"] > 1 - 1e-3, report
    # full-step angular velocity away from events
    om = split_state(lat, lat.omega_full())
    hit = {(ev[0], ev[1]) for ev in res["events"]} | {(rec[0], rec[1]) for rec in res["ill"]}
    for c, s in enumerate(specs):
        for r in range(s["n_rep"]):
            if (c, r) not in hit:
                assert np.abs(om[c][r] - o_om[c][r]).max() < 2e-3, (c, r)


@pytest.mark.parametrize("path", [XY_PATH_BATCHED, XY_PATH_PLAIN])
def test_ordered_start_parity_100_steps(path):
    """From the ordered state the benchmark workloads start in (theta =
    2 pi / 5 at T_c), 100 steps on the resident, strip and plain kernels:
    every site within 1e-4 rad of the oracle except sites next to a cusp
    event, which T_c reaches within 100 steps; such sites are listed."""
    shapes = [(64, 64, 2), (256, 64, 2), (32, 256, 1), (12, 10, 2)]
    specs = [inputs.config(Lx, Ly, n, seed=31 + i, knots=([0], [TC])) for i, (Lx, Ly, n) in enumerate(shapes)]
    thetas = [np.full((s["n_rep"], s["Lx"] * s["Ly"]), np.float32(2 * PI / 5)) for s in specs]
    lat, o_th, o_om = make_pair(specs, thetas, path=path)
    res = stepwise_parity(lat, specs, o_th, o_om, 100)
    report = parity_report(res)
    print(report)
    assert not res["unexplained"], (res["unexplained"][:10], report)
    assert res["frac_within_tol"] > 1 - 1e-3, report


def test_plain_method_workload_parity():
    """64 x 64, one replica, seed 1, theta uniform from the library's own
    initialisation (noise stream tag 1), T_c, 100 steps."""
    lat = Lattice([Config(Lx=64, Ly=64, n_replicas=1, seed=1, init_mode=0, knots=((0,), (TC,)))])
    spec = inputs.config(64, 64, 1, seed=1)
    o_th = [oracle.init_theta(64, 64, 0, 0, 1, 0).reshape(1, -1)]
    torch.cuda.synchronize()
    assert circ_diff(split_state(lat, lat.theta)[0], o_th[0]).max() < 1e-6
    o_om = [np.zeros_like(o_th[0])]
    res = stepwise_parity(lat, [spec], o_th, o_om, 100)
    print(parity_report(res))
    assert not res["unexplained"], res["unexplained"][:10]
    assert res["frac_within_tol"] > 1 - 1e-3


def test_records_and_moments_parity():
    """Observables of a 100-step call against the oracle's, lattice by
    lattice; lattices whose trajectory met a cusp event compare at a looser
    bound after the event."""
    specs = _mixed_specs()
    thetas = _mixed_thetas(specs, seed=15)
    lat, o_th, o_om = make_pair(specs, thetas)
    rec = lat.step(100, record_every=10, t0=20)
    mom, steps = lat.observe()
    assert list(steps) == [100] * len(specs)
    step_now = [0] * len(specs)
    o_rec, o_mom = oracle.run_batch(specs, o_th, o_om, step_now, 100, record_every=10, t0=20)
    g = rec.cpu().numpy()
    b = 0
    loose = 0
    for c, s in enumerate(specs):
        for r in range(s["n_rep"]):
            mine, ref = g[b, :10], o_rec[c][r]
            assert ref.shape == (10, 2)
            dm = np.abs(mine[:, 0] - ref[:, 0])
            de = np.abs(mine[:, 1] - ref[:, 1]) / (1 + np.abs(ref[:, 1]))
            if dm.max() > 2e-5 or de.max() > 2e-5:
                loose += 1
                assert dm.max() < 2e-3 and de.max() < 2e-4, (c, r, dm.max(), de.max())
            assert np.isnan(g[b, 10]).all()  # R = n // record_every + 1; the last slot stays untouched
            b += 1
    assert loose <= 2, loose
    assert np.array_equal(mom[:, 0], o_mom[:, 0])
    assert np.allclose(mom, o_mom, rtol=2e-4, atol=1e-7)


def test_records_further_apart_than_a_graph_chunk():
    """Records every 50 steps (more than a 32-step graph chunk) of a call
    that starts at step 7: the recording steps run alone with the recording
    kernel, the stretches between them as non-recording chunks.  Records
    match the oracle's; the state is bit-identical to a run without records."""
    specs = _mixed_specs()
    thetas = _mixed_thetas(specs, seed=17)
    lat, o_th, o_om = make_pair(specs, thetas)
    ref, _, _ = make_pair(specs, thetas)
    lat.step(7)
    ref.step(7)
    rec = lat.step(130, record_every=50).cpu().numpy()  # k = 50 and 100
    ref.step(130)
    torch.cuda.synchronize()
    assert torch.equal(lat.theta, ref.theta) and torch.equal(lat.omega, ref.omega)
    step_now = [0] * len(specs)
    oracle.run_batch(specs, o_th, o_om, step_now, 7)
    o_rec, _ = oracle.run_batch(specs, o_th, o_om, step_now, 130, record_every=50)
    b, loose = 0, 0
    for c, s in enumerate(specs):
        for r in range(s["n_rep"]):
            mine, want = rec[b, :2], o_rec[c][r]
            assert want.shape == (2, 2)
            dm = np.abs(mine[:, 0] - want[:, 0])
            de = np.abs(mine[:, 1] - want[:, 1]) / (1 + np.abs(want[:, 1]))
            if dm.max() > 2e-5 or de.max() > 2e-5:
                loose += 1
                assert dm.max() < 2e-3 and de.max() < 2e-4, (c, r, dm.max(), de.max())
            assert np.isnan(rec[b, 2]).all()
            b += 1
    assert loose <= 2, loose


def test_plain_and_batched_are_bit_identical():
    specs = _mixed_specs()
    thetas = _mixed_thetas(specs, seed=9)
    a, _, _ = make_pair(specs, thetas, path=XY_PATH_BATCHED)
    b, _, _ = make_pair(specs, thetas, path=XY_PATH_PLAIN)
    for lat in (a, b):
        lat.step(37)
        lat.step(40)  # odd, then even: parity fix-up both ways, and a graph chunk
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta)
    assert torch.equal(a.omega, b.omega)


def test_resume_and_snapshot_are_bit_identical():
    specs = _mixed_specs(T=3.0)
    thetas = _mixed_thetas(specs, seed=13)
    a, _, _ = make_pair(specs, thetas)
    b, _, _ = make_pair(specs, thetas)
    a.step(90, record_every=9)
    b.step(13, record_every=9)
    snap = b.save()
    b.step(77, record_every=9)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)
    # reload the snapshot and redo the second part
    b.load(snap)
    b.step(77, record_every=9)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)
    ma, sa = a.observe()
    mb, sb = b.observe()
    assert np.array_equal(sa, sb)


def test_uneven_run_lengths_in_one_batch():
    totals = [30, 77, 100, 5, 0, 64, 99, 1]
    specs = _mixed_specs()
    for s, n in zip(specs, totals):
        s["n_total"] = n
    thetas = _mixed_thetas(specs, seed=21)
    lat, o_th, o_om = make_pair(specs, thetas)
    lat.step(60)
    lat.step(60)
    _, steps = lat.observe()
    assert list(steps) == totals
    # the same run step by step against the oracle
    lat2, o_th, o_om = make_pair(specs, thetas)
    res = stepwise_parity(lat2, specs, o_th, o_om, 120)
    print(parity_report(res))
    assert res["step_now"] == totals
    assert not res["unexplained"], (res["unexplained"][:10], res["events"][:10], res["ill"][:10])
    assert res["frac_within_tol"] > 1 - 1e-3
    torch.cuda.synchronize()
    assert torch.equal(lat.theta, lat2.theta) and torch.equal(lat.omega, lat2.omega)


def test_quench_schedule_parity():
    """Linear ramp eps(t) = -t / tau_Q from 1.5 T_c after an equilibration segment."""
    tau_q = 40
    knots = ([20, 20 + int(1.5 * tau_q)], [1.5 * TC, 0.0])
    specs = [inputs.config(Lx, Ly, n, seed=3 + i, knots=knots, n_total=20 + int(1.5 * tau_q),
                           eta=[0.1, 1.0, 10.0][i % 3], h=[0.5, 1.0, 2.0][i % 3])
             for i, (Lx, Ly, n) in enumerate([(64, 64, 2), (256, 64, 1), (12, 10, 1)])]
    thetas = _mixed_thetas(specs, seed=31)
    lat, o_th, o_om = make_pair(specs, thetas)
    rec = lat.step(200, record_every=5)
    step_now = [0] * 3
    o_rec, _ = oracle.run_batch(specs, o_th, o_om, step_now, 200, record_every=5)
    worst, bad = theta_parity(split_state(lat, lat.theta), o_th)
    assert worst <= 1e-4, (worst, bad[:10])
    g = rec.cpu().numpy()
    assert np.abs(g[0, :16, 1] - o_rec[0][0][:, 1]).max() < 1e-4


@pytest.mark.parametrize("gamma", [2.0, 3.0])
def test_nonlinear_quench_parity(gamma):
    """Nonlinear quench eps = -sign(t) |t / tau_Q|^gamma (Sec. V) crossing T_c
    inside a 100-step window, on the batched and the plain path, classified
    like every trajectory parity test (cusp events, FP32 conditioning)."""
    sched = {"power": (TC, 45, 40.0, gamma, 0.5, -0.9)}
    specs = [inputs.config(Lx, Ly, n, seed=5 + i, knots=sched, n_total=400, eta=[0.5, 1.0][i % 2])
             for i, (Lx, Ly, n) in enumerate([(64, 64, 2), (256, 32, 1), (12, 10, 1)])]
    thetas = _mixed_thetas(specs, seed=33)
    for path in (XY_PATH_BATCHED, XY_PATH_PLAIN):
        lat, o_th, o_om = make_pair(specs, thetas, path=path)
        res = stepwise_parity(lat, specs, o_th, o_om, 100)
        print(path, parity_report(res))
        assert res["step_now"] == [100] * len(specs)
        assert not res["unexplained"], (path, res["unexplained"][:10], res["events"][:10], res["ill"][:10])
        assert res["frac_within_tol"] > 1 - 1e-3
    # the schedule survives a snapshot
    lat2, _, _ = make_pair(specs, thetas)
    lat2.step(60)
    blob = lat2.save()
    lat2.step(100)
    a = lat2.theta.clone()
    lat2.load(blob)
    lat2.step(100)
    assert torch.equal(a, lat2.theta)


FIELD = ([10, 80], [0.5, 2.0])  # an orthogonal quench: the field ramps from h / 2 to 2 h


@pytest.mark.parametrize("path", [XY_PATH_BATCHED, XY_PATH_PLAIN])
def test_field_schedule_parity(path):
    """The field schedule h_k = h s(k) (orthogonal quench) with a temperature
    ramp at the same time, on the resident, strip and plain kernels: 100
    steps one at a time against the oracle, classified like every trajectory
    test; then records of (M, E), which carry h_k in E_k."""
    knots = ([0, 100], [1.3 * TC, 0.6 * TC])
    shapes = [(64, 64, 2), (256, 32, 1), (12, 10, 1)]
    specs = [inputs.config(Lx, Ly, n, seed=61 + i, knots=knots, field=FIELD) for i, (Lx, Ly, n) in enumerate(shapes)]
    thetas = _mixed_thetas(specs, seed=63)
    lat, o_th, o_om = make_pair(specs, thetas, path=path)
    res = stepwise_parity(lat, specs, o_th, o_om, 100)
    print(path, parity_report(res))
    assert res["step_now"] == [100] * len(specs)
    assert not res["unexplained"], (res["unexplained"][:10], res["events"][:10])
    assert res["frac_within_tol"] > 1 - 1e-3
    lat2, o_th2, o_om2 = make_pair(specs, thetas, path=path)
    rec = lat2.step(60, record_every=6).cpu().numpy()
    o_rec, _ = oracle.run_batch(specs, o_th2, o_om2, [0, 0, 0], 60, record_every=6)
    b = 0
    for c, s_ in enumerate(specs):
        for r in range(s_["n_rep"]):
            dm = np.abs(rec[b, :10, 0] - o_rec[c][r][:, 0]).max()
            de = (np.abs(rec[b, :10, 1] - o_rec[c][r][:, 1]) / (1 + np.abs(o_rec[c][r][:, 1]))).max()
            assert dm < 2e-5 and de < 2e-5, (c, r, dm, de)
            b += 1


def test_field_schedule_removed_and_snapshot():
    """Removing the schedule restores the bits of a run that never had one;
    the schedule survives a snapshot."""
    specs = [inputs.config(256, 32, 1, seed=71), inputs.config(64, 64, 1, seed=72)]
    thetas = _mixed_thetas(specs, seed=73)
    a, _, _ = make_pair(specs, thetas)
    b, _, _ = make_pair([dict(s, field=FIELD) for s in specs], thetas)
    b.set_field_schedule(0, [], [])
    b.set_field_schedule(1, [], [])
    a.step(50)
    b.step(50)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)
    c, _, _ = make_pair([dict(s, field=FIELD) for s in specs], thetas)
    c.step(30)
    blob = c.save()
    c.step(60)
    t1 = c.theta.clone()
    c.load(blob)
    c.step(60)
    torch.cuda.synchronize()
    assert torch.equal(t1, c.theta)
    with pytest.raises(XYError):
        c.set_field_schedule(0, [5, 5], [1.0, 2.0])


@pytest.mark.parametrize("mode", ["recompute", "backward"])
def test_adjoint_with_field_schedule_matches_oracle(mode):
    """d/d(J_par, J_perp, h, eta) with a field ramp (d/dh at the fixed profile
    s(k)) against the oracle's FP64 adjoint, every component within 1e-3."""
    prm = dict(J_par=2.0, J_perp=0.5, h=1.0, p=2.0, eta=0.8)
    knots = ([0, 100], [1.0, 0.5])
    field = ([5, 70], [0.3, 1.8])
    if mode == "recompute":
        shapes = [(16, 8, 2), (128, 4, 1), (12, 10, 1)]
    else:
        shapes = [(16, 8, 2), (128, 4, 1), (256, 6, 1)]
    specs = [inputs.config(Lx, Ly, n, seed=3 + i, knots=knots, field=field, **prm) for i, (Lx, Ly, n) in enumerate(shapes)]
    thetas = _mixed_thetas(specs, seed=81)
    lat, o_th, o_om = make_pair(specs, thetas)
    lat.set_adjoint_mode(XY_ADJOINT_RECOMPUTE if mode == "recompute" else XY_ADJOINT_BACKWARD)
    obj, grads = lat.adjoint(100, checkpoint_every=30, w_E=0.7, w_M=0.3)
    o_obj, o_grads = _oracle_adjoint(specs, o_th, o_om, 100, 0.7, 0.3)
    assert obj == pytest.approx(o_obj, rel=1e-5, abs=2e-6)
    assert_grads_close(grads, o_grads, 1e-3)


# an anisotropic quench: J_par ramps down by half while J_perp triples
COUPLINGS = ([15, 85], [1.0, 0.5], [0.6, 3.0])


@pytest.mark.parametrize("path", [XY_PATH_BATCHED, XY_PATH_PLAIN])
def test_coupling_schedule_parity(path):
    """Coupling profiles J_par a(k), J_perp b(k) (anisotropic quench) with a
    temperature ramp and a field ramp at the same time, on the resident,
    strip and plain kernels: 100 steps one at a time against the oracle,
    classified like every trajectory test; then records of (M, E), which
    carry the couplings of step k in E_k."""
    knots = ([0, 100], [1.3 * TC, 0.6 * TC])
    shapes = [(64, 64, 2), (256, 32, 1), (12, 10, 1)]
    specs = [inputs.config(Lx, Ly, n, seed=91 + i, knots=knots, field=FIELD, couplings=COUPLINGS)
             for i, (Lx, Ly, n) in enumerate(shapes)]
    thetas = _mixed_thetas(specs, seed=93)
    lat, o_th, o_om = make_pair(specs, thetas, path=path)
    res = stepwise_parity(lat, specs, o_th, o_om, 100)
    print(path, parity_report(res))
    assert res["step_now"] == [100] * len(specs)
    assert not res["unexplained"], (res["unexplained"][:10], res["events"][:10])
    assert res["frac_within_tol"] > 1 - 1e-3
    lat2, o_th2, o_om2 = make_pair(specs, thetas, path=path)
    rec = lat2.step(60, record_every=6).cpu().numpy()
    o_rec, _ = oracle.run_batch(specs, o_th2, o_om2, [0, 0, 0], 60, record_every=6)
    b = 0
    for c, s_ in enumerate(specs):
        for r in range(s_["n_rep"]):
            dm = np.abs(rec[b, :10, 0] - o_rec[c][r][:, 0]).max()
            de = (np.abs(rec[b, :10, 1] - o_rec[c][r][:, 1]) / (1 + np.abs(o_rec[c][r][:, 1]))).max()
            assert dm < 2e-5 and de < 2e-5, (c, r, dm, de)
            b += 1


def test_coupling_schedule_removed_and_snapshot():
    """Removing the profiles restores the bits of a run that never had them;
    they survive a snapshot; bad knots are refused."""
    specs = [inputs.config(256, 32, 1, seed=95), inputs.config(64, 64, 1, seed=96)]
    thetas = _mixed_thetas(specs, seed=97)
    a, _, _ = make_pair(specs, thetas)
    b, _, _ = make_pair([dict(s, couplings=COUPLINGS) for s in specs], thetas)
    b.set_coupling_schedule(0, [], [], [])
    b.set_coupling_schedule(1, [], [], [])
    a.step(50)
    b.step(50)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)
    c, _, _ = make_pair([dict(s, couplings=COUPLINGS) for s in specs], thetas)
    c.step(30)
    blob = c.save()
    c.step(60)
    t1 = c.theta.clone()
    c.load(blob)
    c.step(60)
    torch.cuda.synchronize()
    assert torch.equal(t1, c.theta)
    with pytest.raises(XYError):
        c.set_coupling_schedule(0, [5, 5], [1.0, 2.0], [1.0, 1.0])
    with pytest.raises(XYError):
        c.set_coupling_schedule(0, [5], [float("nan")], [1.0])


@pytest.mark.parametrize("kind", ["field", "couplings"])
def test_schedule_set_between_calls(kind):
    """A schedule set after the stepper has run (and captured its graphs)
    without one takes effect: the run equals one that had the schedule from
    the start, its scales exactly 1 up to the first knot, bit for bit."""
    specs = [inputs.config(256, 32, 2, seed=101), inputs.config(64, 64, 1, seed=102)]
    thetas = _mixed_thetas(specs, seed=103)
    sched = dict(field=([40, 80], [1.0, 2.0])) if kind == "field" else dict(couplings=([40, 80], [1.0, 0.5], [1.0, 3.0]))
    a, _, _ = make_pair([dict(s, **sched) for s in specs], thetas)
    b, _, _ = make_pair(specs, thetas)
    a.step(40)
    b.step(40)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)
    for c in range(len(specs)):
        if kind == "field":
            b.set_field_schedule(c, *sched["field"])
        else:
            b.set_coupling_schedule(c, *sched["couplings"])
    a.step(70)
    b.step(70)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)
    # and the schedule does act: a run without it differs
    c0, _, _ = make_pair(specs, thetas)
    c0.step(110)
    torch.cuda.synchronize()
    assert not torch.equal(c0.theta, b.theta)


@pytest.mark.parametrize("mode", ["recompute", "backward"])
def test_adjoint_with_coupling_schedule_matches_oracle(mode):
    """d/d(J_par, J_perp, h, eta) with both couplings ramped at different rates
    and a field ramp (d/dJ and d/dh at the fixed profiles) against the
    oracle's FP64 adjoint, every component within 1e-3."""
    prm = dict(J_par=2.0, J_perp=0.5, h=1.0, p=2.0, eta=0.8)
    knots = ([0, 100], [1.0, 0.5])
    field = ([5, 70], [0.3, 1.8])
    cpl = ([10, 60, 95], [1.4, 0.6, 1.0], [0.5, 2.0, 1.2])
    if mode == "recompute":
        shapes = [(16, 8, 2), (128, 4, 1), (12, 10, 1)]
    else:
        shapes = [(16, 8, 2), (128, 4, 1), (256, 6, 1)]
    specs = [inputs.config(Lx, Ly, n, seed=13 + i, knots=knots, field=field, couplings=cpl, **prm)
             for i, (Lx, Ly, n) in enumerate(shapes)]
    thetas = _mixed_thetas(specs, seed=83)
    lat, o_th, o_om = make_pair(specs, thetas)
    lat.set_adjoint_mode(XY_ADJOINT_RECOMPUTE if mode == "recompute" else XY_ADJOINT_BACKWARD)
    obj, grads = lat.adjoint(100, checkpoint_every=30, w_E=0.7, w_M=0.3)
    o_obj, o_grads = _oracle_adjoint(specs, o_th, o_om, 100, 0.7, 0.3)
    assert obj == pytest.approx(o_obj, rel=1e-5, abs=2e-6)
    assert_grads_close(grads, o_grads, 1e-3)


def test_staggered_order_parameter():
    specs = [inputs.config(64, 64, 2, seed=4, J_par=-10.0, J_perp=-0.1, staggered=1.0)]
    thetas = _mixed_thetas(specs, seed=41)
    lat, o_th, o_om = make_pair(specs, thetas)
    rec = lat.step(50, record_every=5)
    step_now = [0]
    o_rec, _ = oracle.run_batch(specs, o_th, o_om, step_now, 50, record_every=5)
    assert np.abs(rec.cpu().numpy()[:, :10, 0] - np.stack(o_rec[0])[:, :, 0]).max() < 2e-5


# ------------------------------------------------------------------ edge cases


def test_edge_cases_and_errors():
    lat = Lattice([Config(Lx=8, Ly=8, n_replicas=1)])
    th0 = lat.theta.clone()
    lat.step(0)
    torch.cuda.synchronize()
    assert torch.equal(lat.theta, th0)
    rec = lat.step(3, record_every=10)  # one record at k = 0
    assert rec.shape == (1, 1, 2) and torch.isfinite(rec).all()
    with pytest.raises(XYError):
        lat.set_params(0, dt=-1.0)
    with pytest.raises(XYError):
        lat.set_schedule(0, [5, 5], [1.0, 1.0], 10)
    with pytest.raises(XYError):
        lat.set_schedule(0, [0], [-1.0], 10)
    with pytest.raises(XYError):
        lat.step(-1)
    with pytest.raises(XYError):
        Lattice([Config(Lx=6, Ly=4)])
    with pytest.raises(XYError):
        lat.label_domains(0, 2)
    assert lat.kernel_launches() > 0


# ------------------------------------------------------------------ failure detection


def test_union_timeout_is_reported_and_recoverable():
    """A union-find bound of one step makes the labelling of a percolating
    pattern run out: the call returns XY_ETIMEOUT (no fault, no hang) and the
    next call with the default bound is exact again."""
    from paper_2409_06412_gb300 import _lib
    spins = inputs.random_spins(512, 512, seed=91, p_up=0.7)
    th = torch.from_numpy(inputs.spins_to_theta(spins).ravel()).cuda()
    lat = Lattice([Config(Lx=512, Ly=512, n_replicas=1, init_mode=_lib.XY_INIT_USER)], theta=th,
                  omega=torch.zeros_like(th))
    _lib.call("xy_debug_set_union_limit", 1)
    try:
        with pytest.raises(XYError) as ei:
            lat.label_domains(0, 1)
        assert ei.value.code == _lib.XY_ETIMEOUT
    finally:
        _lib.call("xy_debug_set_union_limit", 0)
    labels, _, _ = lat.label_domains(0, 1)
    lab_o, _ = oracle.ccl(512, 512, inputs.spins_to_theta(spins).ravel())
    assert np.array_equal(labels[0].cpu().numpy(), lab_o)
    lat.close()


def test_non_finite_state_is_reported():
    """A NaN angle in the caller's state spreads to the observables; the FP64
    moments come back as XY_ENAN from xy_observe."""
    from paper_2409_06412_gb300 import _lib
    th = torch.from_numpy(inputs.angles(1, 16, 8, 93).ravel()).cuda()
    th[37] = float("nan")
    lat = Lattice([Config(Lx=16, Ly=8, n_replicas=1, init_mode=_lib.XY_INIT_USER)], theta=th,
                  omega=torch.zeros_like(th))
    lat.step(10, record_every=5)
    with pytest.raises(XYError) as ei:
        lat.observe()
    assert ei.value.code == _lib.XY_ENAN
    lat.close()


def test_failed_allocation_is_reported_and_recoverable():
    """An adjoint whose checkpoints cannot be allocated (1e9 steps with a
    checkpoint every step: 1 TB) returns XY_ENOMEM before launching anything
    on them; the object stays usable."""
    from paper_2409_06412_gb300 import _lib
    specs = [inputs.config(16, 8, 1, seed=3)]
    lat, _, _ = make_pair(specs, _mixed_thetas(specs))
    with pytest.raises(XYError) as ei:
        lat.adjoint(10 ** 9, checkpoint_every=1)
    assert ei.value.code == _lib.XY_ENOMEM
    _, steps = lat.observe()
    assert list(steps) == [0]
    lat.step(5)
    obj, grads = lat.adjoint(10, checkpoint_every=5)
    assert np.isfinite(obj) and np.all(np.isfinite(grads))
    lat.close()


# ------------------------------------------------------------------ domains


@pytest.mark.parametrize("case", ["random", "stripes_x", "stripes_y", "checker", "uniform", "spiral", "sparse",
                                  "tiny"])
def test_domain_labels_bit_exact(case):
    L = 96
    s = {
        "random": lambda: inputs.random_spins(L, L, 4),
        "stripes_x": lambda: inputs.stripes(L, L, 3, 0),
        "stripes_y": lambda: inputs.stripes(L, L, 5, 1),
        "checker": lambda: inputs.checkerboard(L, L),
        "uniform": lambda: np.ones((L, L), np.int8),
        "spiral": lambda: inputs.spiral(L),
        "sparse": lambda: inputs.random_spins(L, L, 9, p_up=0.08),
        "tiny": lambda: inputs.random_spins(4, 1, 3),
    }[case]()
    Ly, Lx = s.shape
    th = inputs.spins_to_theta(s).reshape(1, -1)
    spec = inputs.config(Lx, Ly, 1)
    lat, _, _ = make_pair([spec], [th])
    labels, hist, n_sizes = lat.label_domains(hist_cap=Lx * Ly)
    lab_o, hist_o = oracle.ccl(Lx, Ly, th[0])
    assert np.array_equal(labels[0].cpu().numpy(), lab_o)
    k = int(n_sizes[0])
    assert k == hist_o.shape[0]
    assert np.array_equal(hist[0, :k].cpu().numpy(), hist_o)
    assert torch.all(hist[0, k:] == 0)


def test_domain_labels_after_quench_and_host_outputs():
    knots = ([50, 350], [1.5 * TC, 0.0])
    specs = [inputs.config(256, 128, 3, seed=8, knots=knots, n_total=350)]
    thetas = _mixed_thetas(specs, seed=51)
    lat, _, _ = make_pair(specs, thetas)
    lat.step(350)
    labels, hist, n_sizes = lat.label_domains(hist_cap=4096)
    th = split_state(lat, lat.theta)[0].astype(np.float32)
    for r in range(3):
        lab_o, hist_o = oracle.ccl(256, 128, th[r])
        assert np.array_equal(labels[r].cpu().numpy(), lab_o)
        k = int(n_sizes[r])
        assert np.array_equal(hist[r, :k].cpu().numpy(), hist_o)
    # host output buffers through the raw ABI
    from paper_2409_06412_gb300 import _lib
    lab_h = np.zeros((3, 256 * 128), np.int32)
    hist_h = np.zeros((3, 8, 2), np.int64)
    ns_h = np.zeros(3, np.int64)
    rc = _lib.load().xy_label_domains(lat._h, 0, 3, lab_h.ctypes.data_as(ctypes.c_void_p),
                                      hist_h.ctypes.data_as(ctypes.c_void_p), 8,
                                      ns_h.ctypes.data_as(ctypes.c_void_p))
    assert np.array_equal(lab_h, labels.cpu().numpy())
    assert np.array_equal(ns_h, n_sizes.cpu().numpy())
    if ns_h.max() > 8:
        assert rc == _lib.XY_EINVAL  # more distinct sizes than hist_cap
    assert np.array_equal(hist_h[:, :8], hist[:, :8].cpu().numpy())
    # with kernel timing on, each call records one span of its passes and the
    # labels do not change
    lat.set_kernel_timing(True)
    for _ in range(2):
        lab_t, _, _ = lat.label_domains(hist_cap=4096)
    ms, n = lat.kernel_timing()
    lat.set_kernel_timing(False)
    assert n[_lib.XY_KCLASS_LABELS] == 2 and ms[_lib.XY_KCLASS_LABELS] > 0
    assert np.array_equal(lab_t.cpu().numpy(), labels.cpu().numpy())


# ------------------------------------------------------------------ adjoint


def _oracle_adjoint(specs, o_th, o_om, n, wE, wM):
    B = sum(s["n_rep"] for s in specs)
    obj, grads = 0.0, []
    for c, s in enumerate(specs):
        g = np.zeros(4)
        for r in range(s["n_rep"]):
            ob, gr, _, _ = oracle.adjoint_lattice(s["Lx"], s["Ly"], c, r, s["seed"], s["params"], s["knots"], 0, n,
                                                  o_th[c][r], o_om[c][r], wE, wM, field=s.get("field"),
                                                  couplings=s.get("couplings"))
            obj += ob
            g += gr
        grads.append(g / (B * n))
    return obj / (B * n), np.array(grads)


@pytest.mark.parametrize("mode", ["recompute", "backward"])
@pytest.mark.parametrize("field", ["smooth_p2", "paper_p2.5_lowT", "staggered_af"])
def test_adjoint_matches_oracle(field, mode):
    if field == "smooth_p2":
        prm = dict(J_par=2.0, J_perp=0.5, h=1.0, p=2.0, eta=0.8)
        knots = ([0, 100], [1.0, 0.5])
    elif field == "staggered_af":
        # the antiferromagnetic reading: negative couplings, |M| of the
        # staggered order parameter sigma = (-1)^(x+y)
        prm = dict(J_par=-2.0, J_perp=-0.5, h=1.0, p=2.0, eta=0.8, staggered=1.0)
        knots = ([0, 100], [1.0, 0.5])
    else:
        prm = dict(h=3.0)
        knots = ([0], [0.05])
    if mode == "recompute":
        # band reverse kernel (16 x 8 with sub-warp rows, 128 x 4) and the
        # per-quad fallback (12 x 10, a width the band decomposition does not
        # take), each segment recomputed forward
        specs = [inputs.config(16, 8, 2, seed=3, knots=knots, **prm),
                 inputs.config(128, 4, 1, seed=4, knots=knots, **prm),
                 inputs.config(12, 10, 1, seed=4, knots=knots, **prm)]
    else:
        # states integrated backward inside the reverse kernel: sub-warp rows,
        # one full-warp row, and two 128-column strips side by side (one row
        # per band: every row is a halo row of the neighbouring bands)
        specs = [inputs.config(16, 8, 2, seed=3, knots=knots, **prm),
                 inputs.config(128, 4, 1, seed=4, knots=knots, **prm),
                 inputs.config(256, 6, 1, seed=5, knots=knots, **prm)]
    if field in ("smooth_p2", "staggered_af"):
        thetas = _mixed_thetas(specs, seed=61)
    else:
        thetas = [np.full((s["n_rep"], s["Lx"] * s["Ly"]), np.float32(2 * PI / 5)) +
                  0.05 * inputs.velocities(s["n_rep"], s["Lx"], s["Ly"], 62 + i) for i, s in enumerate(specs)]
        thetas = [t.astype(np.float32) for t in thetas]
    lat, o_th, o_om = make_pair(specs, thetas)
    lat.set_adjoint_mode(XY_ADJOINT_RECOMPUTE if mode == "recompute" else XY_ADJOINT_BACKWARD)
    n, K = 100, 30
    obj, grads = lat.adjoint(n, checkpoint_every=K, w_E=0.7, w_M=0.3)
    o_obj, o_grads = _oracle_adjoint(specs, o_th, o_om, n, 0.7, 0.3)
    # the objective averages per-site terms of size |J| ~ 2 in FP32 partial
    # sums; where they nearly cancel (antiferromagnetic couplings) the bound is
    # that rounding, 1e-6 of the terms, not a fraction of the small sum
    assert obj == pytest.approx(o_obj, rel=1e-5, abs=2e-6)
    assert_grads_close(grads, o_grads, 1e-3)
    _, steps = lat.observe()
    assert list(steps) == [n, n, n]


def test_adjoint_modes_agree_on_wide_strips():
    """Backward integration against the stored recompute on lattices of 3, 2
    and 16 strips of 128 columns at T_c from the ordered state, with n a multiple of
    the checkpoint interval (the last segment ends at the final state) and
    not: gradients and objective agree to rounding of the recovered states,
    and the state after the call is the same forward state."""
    specs = [inputs.config(384, 32, 2, seed=7, knots=([0], [TC])), inputs.config(256, 16, 3, seed=8, knots=([0], [TC])),
             inputs.config(2048, 8, 1, seed=9, knots=([0], [TC]))]  # 16 strips: 512 threads, 64 KB of staging
    thetas = [np.full((s["n_rep"], s["Lx"] * s["Ly"]), np.float32(2 * PI / 5)) +
              0.02 * inputs.velocities(s["n_rep"], s["Lx"], s["Ly"], 80 + i) for i, s in enumerate(specs)]
    thetas = [t.astype(np.float32) for t in thetas]
    for n, K in ((120, 40), (130, 40)):
        res = {}
        for mode in (XY_ADJOINT_RECOMPUTE, XY_ADJOINT_BACKWARD):
            lat, _, _ = make_pair(specs, thetas)
            lat.step(20)
            lat.set_adjoint_mode(mode)
            obj, grads = lat.adjoint(n, checkpoint_every=K, w_E=1.0, w_M=1.0)
            res[mode] = (obj, grads, lat.theta.cpu().numpy().copy())
            lat.close()
        (o1, g1, t1), (o2, g2, t2) = res[XY_ADJOINT_RECOMPUTE], res[XY_ADJOINT_BACKWARD]
        assert np.array_equal(t1, t2)
        assert o2 == pytest.approx(o1, rel=1e-6)
        assert_grads_close(g2, g1, 1e-4, what=f"n = {n}")


@pytest.mark.parametrize("n,K", [(1, 1), (1, 100), (5, 1), (7, 100), (9, 3)])
def test_adjoint_schedules_agree_on_short_windows(n, K):
    """Degenerate windows: one step, a checkpoint every step, a checkpoint
    interval longer than the window, n a multiple of K."""
    specs = [inputs.config(256, 8, 2, seed=21, knots=([0], [TC])), inputs.config(32, 16, 3, seed=22, knots=([0], [TC]))]
    thetas = _mixed_thetas(specs, seed=23)
    res = {}
    for mode in (XY_ADJOINT_RECOMPUTE, XY_ADJOINT_BACKWARD):
        lat, _, _ = make_pair(specs, thetas)
        lat.set_adjoint_mode(mode)
        res[mode] = lat.adjoint(n, checkpoint_every=K, w_E=0.6, w_M=0.4) + (lat.theta.cpu().numpy().copy(),)
        lat.close()
    (o1, g1, t1), (o2, g2, t2) = res[XY_ADJOINT_RECOMPUTE], res[XY_ADJOINT_BACKWARD]
    assert np.array_equal(t1, t2)
    assert o2 == pytest.approx(o1, rel=1e-6)
    assert_grads_close(g2, g1, 1e-4)


def test_backward_adjoint_rejects_other_shapes():
    specs = [inputs.config(12, 10, 1, seed=4, knots=([0], [1.0]))]
    lat, _, _ = make_pair(specs, _mixed_thetas(specs))
    lat.set_adjoint_mode(XY_ADJOINT_BACKWARD)
    with pytest.raises(XYError):
        lat.adjoint(10, checkpoint_every=5)
    with pytest.raises(XYError):
        lat.set_adjoint_mode(7)
    lat.set_adjoint_mode(XY_ADJOINT_AUTO)  # falls back to the recompute for this shape
    obj, grads = lat.adjoint(10, checkpoint_every=5)
    assert np.isfinite(obj) and np.all(np.isfinite(grads))


def test_adjoint_autograd_function():
    from paper_2409_06412_gb300.autograd import bbk_objective
    specs = [inputs.config(16, 8, 2, seed=3, knots=([0], [1.0]), p=2.0, J_par=2.0, J_perp=0.5)]
    thetas = _mixed_thetas(specs, seed=71)
    lat, o_th, o_om = make_pair(specs, thetas)
    J = torch.tensor([2.0], dtype=torch.float64, requires_grad=True)
    Jp = torch.tensor([0.5], dtype=torch.float64, requires_grad=True)
    h = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    eta = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    obj = bbk_objective(lat, J, Jp, h, eta, n=40, checkpoint_every=10, w_E=1.0, w_M=0.0)
    obj.backward()
    o_obj, o_grads = _oracle_adjoint(specs, o_th, o_om, 40, 1.0, 0.0)
    assert float(obj.detach()) == pytest.approx(o_obj, rel=1e-5)
    got = np.array([J.grad.item(), Jp.grad.item(), h.grad.item(), eta.grad.item()])
    assert_grads_close(got[None], o_grads[:1], 1e-3)


def _perturbed_ordered(specs, seed, spread=0.05):
    """Angles near the ordered state 2 pi / 5 (the workloads' start) with
    Gaussian spread, and full-step velocities at equipartition for T_c."""
    th = [(np.full((s["n_rep"], s["Lx"] * s["Ly"]), np.float32(2 * PI / 5)) +
           spread * inputs.velocities(s["n_rep"], s["Lx"], s["Ly"], seed + i)).astype(np.float32)
          for i, s in enumerate(specs)]
    om = [inputs.velocities(s["n_rep"], s["Lx"], s["Ly"], seed + 100 + i, scale=math.sqrt(TC)) for i, s in enumerate(specs)]
    return th, om


def _central_differences(spec, th, om, n, K, mode, eps_rel=(1e-3, 1e-3, 1e-3, 1e-3), wE=1.0, wM=1.0):
    """GPU adjoint and central differences of the GPU objective over the four
    parameters, every evaluation from the same full-step state (theta_0,
    omega_0), which is what the adjoint holds fixed: the priming to the stored
    half-step velocity is redone with the perturbed parameters."""
    names = ("J_par", "J_perp", "h", "eta")

    def run(prm):
        sp = [dict(spec, params=dict(spec["params"], **prm))]
        lat, _, _ = make_pair(sp, th, om)
        lat.set_adjoint_mode(mode)
        out = lat.adjoint(n, checkpoint_every=K, w_E=wE, w_M=wM)
        lat.close()
        return out

    base = {k: inputs_params(spec)[k] for k in names}
    _, g = run(base)
    fd = np.zeros(4)
    for i, nm in enumerate(names):
        eps = eps_rel[i] * abs(base[nm])
        op, _ = run(dict(base, **{nm: base[nm] + eps}))
        om_, _ = run(dict(base, **{nm: base[nm] - eps}))
        fd[i] = (op - om_) / (2 * eps)
    return g[0], fd


@pytest.mark.parametrize("mode", [XY_ADJOINT_BACKWARD, XY_ADJOINT_RECOMPUTE])
@pytest.mark.parametrize("field", ["p2_at_Tc", "p2.5_below_the_cut"])
def test_adjoint_matches_central_differences(field, mode):
    """The GPU adjoint against central differences of the GPU objective
    (epsilon = 1e-3 relative to each parameter), component by component
    within 1e-3 relative, on the differentiation workload's shape (64
    lattices of 256 x 256, the paper's couplings) over 50 steps with a
    checkpoint every 25, from near the ordered state.

    The pathwise derivative exists where the dynamics is smooth: with p = 2
    the field force h p sin(p theta) is continuous across the wrap cut at
    +-pi/2 (as the couplings always are, q = 2), so at T_c every crossing of
    the cut is smooth; with the paper's p = 2.5 the force jumps there by
    2 h p sin(1.25 pi), and the test runs below the temperatures at which
    sites reach the cut within the window (T = 0.2, 0.314 rad from 2 pi / 5
    at a thermal spread of ~0.035 rad).  At T_c with p = 2.5 a perturbation
    of 1e-3 shifts some of the many crossings by a step and the difference
    quotient picks up those jumps; the adjoint is the derivative almost
    everywhere and leaves them out (measured there: 0.1-1 % apart).

    Epsilon is 1e-3 of J_par, J_perp and h, and 1e-2 of eta.  The kernels
    take eta through the FP32 constants 1 - eta dt / 2 and 1 / (1 + eta dt / 2):
    a change of 1e-3 in eta moves them by 5e-6 while their rounding is
    3e-8, so the effective perturbation is off by up to 0.6 % per evaluation
    (measured: the eta quotient's error times epsilon stays at ~5e-7 of the
    objective from epsilon = 1e-3 to 1e-5).  At 1e-2 that quantisation is
    below 6e-4 and the truncation error of the central difference ~1e-4.
    The J_par, J_perp and h constants round at ~1e-4 of a 1e-3 step."""
    if field == "p2_at_Tc":
        spec = inputs.config(256, 256, 64, seed=41, knots=([0], [TC]), p=2.0)
        th, om = _perturbed_ordered([spec], 300)
    else:
        T = 0.2
        spec = inputs.config(256, 256, 64, seed=42, knots=([0], [T]))
        th, _ = _perturbed_ordered([spec], 310, spread=0.02)
        om = [inputs.velocities(64, 256, 256, 320, scale=math.sqrt(T))]
    g, fd = _central_differences(spec, th, om, 50, 25, mode, eps_rel=(1e-3, 1e-3, 1e-3, 1e-2))
    print(f"{field}: adjoint {g}, central differences {fd}, relative {np.abs(g - fd) / np.abs(fd)}")
    assert_grads_close(g[None], fd[None], 1e-3)


def test_adjoint_auto_schedule_follows_the_damping_bound():
    """Backward integration undoes the damping, which amplifies FP32 rounding
    by about exp(eta dt K) per segment: XY_ADJOINT_AUTO integrates backward
    up to eta dt K = 5 and recomputes above it.  At eta = 5 (eta dt K = 5)
    AUTO is the backward schedule, bit for bit, and agrees with the
    recompute per component within 1e-4; at eta = 10 (eta dt K = 10) AUTO is
    the recompute, bit for bit."""
    for eta, expect in ((5.0, XY_ADJOINT_BACKWARD), (10.0, XY_ADJOINT_RECOMPUTE)):
        specs = [inputs.config(256, 32, 2, seed=51, knots=([0], [TC]), eta=eta)]
        th, om = _perturbed_ordered(specs, 400)
        res = {}
        for mode in (XY_ADJOINT_AUTO, XY_ADJOINT_BACKWARD, XY_ADJOINT_RECOMPUTE):
            lat, _, _ = make_pair(specs, th, om)
            lat.set_adjoint_mode(mode)
            res[mode] = lat.adjoint(150, checkpoint_every=100, w_E=1.0, w_M=1.0)
            lat.close()
        assert res[XY_ADJOINT_AUTO][0] == res[expect][0]
        assert np.array_equal(res[XY_ADJOINT_AUTO][1], res[expect][1])
        if eta == 5.0:
            assert_grads_close(res[XY_ADJOINT_BACKWARD][1], res[XY_ADJOINT_RECOMPUTE][1], 1e-4)


# ------------------------------------------------------------------ full size, sampled


def test_static_criticality_full_size_sampled():
    """The static-criticality batch at full size (L = 128..1024, 32
    temperatures x 16 replicas each, ordered start) in the benchmark's launch
    configuration; one sampled lattice per L is replayed by the oracle."""
    Ls = [128, 256, 512, 1024]
    temps = np.linspace(0.9, 1.1, 32) * TC
    cfgs, specs = [], []
    for L in Ls:
        for T in temps:
            cfgs.append(Config(Lx=L, Ly=L, n_replicas=16, seed=1, init_mode=1, knots=((0,), (float(T),)),
                               n_total=10 ** 5))
            specs.append(dict(Lx=L, Ly=L, n_rep=16, seed=1, params=dict(inputs.PAPER), knots=([0], [float(T)]),
                              n_total=10 ** 5))
    lat = Lattice(cfgs)
    n = 12
    rec = lat.step(n, record_every=4)
    torch.cuda.synchronize()
    picks = [(0, 3), (40, 7), (77, 15), (127, 0)]  # (config, replica) with L = 128, 256, 512, 1024
    for c, r in picks:
        s = specs[c]
        th = oracle.init_theta(s["Lx"], s["Ly"], c, r, 1, 1)
        om = np.zeros_like(th)
        o_rec = oracle.run_lattice(s["Lx"], s["Ly"], c, r, 1, s["params"], s["knots"], 0, n, th, om, 4)
        b = sum(cc.n_replicas for cc in cfgs[:c]) + r
        g = lat.lattice_view(lat.theta, b).cpu().numpy().ravel()
        assert circ_diff(g, th).max() < 1e-5
        assert np.abs(rec[b, :3, 0].cpu().numpy() - o_rec[:, 0]).max() < 2e-5
    assert torch.isfinite(rec[:, :3]).all()
