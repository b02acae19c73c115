"""Full-size batches of the dynamic-exponent and Kibble-Zurek workloads in the
batched launch configuration, checked on sampled lattices that the FP64
oracle replays whole.

Dynamic exponent z: L in {256, 512, 1024, 2048} x 256 replicas, ordered
start at T_c, M recorded every 10 steps (2.85e9 sites of state and second
buffer, 22.8 GB).  Kibble-Zurek: L = 1024, 16 log-spaced tau_Q in
[1e2, 1e5] steps x eta in {0.1, 1, 10} x h in {0.5, 1, 2} x 64 replicas =
9216 lattices, 1e3 equilibration steps at 1.5 T_c then a linear ramp to 0
over 1.5 tau_Q steps (each setting has its own run length), uniform random
start (1.93e10 sites of state and second buffer, 155 GB).
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_2409_06412_gb300 import XY_INIT_ORDERED, XY_INIT_UNIFORM, build
from paper_2409_06412_gb300.lattice import Config, Lattice
from tests import inputs
from tests.gpu_helpers import assert_grads_close, circ_diff

pytestmark = pytest.mark.gpu
PI = math.pi
TC = inputs.T_C


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()


def _free_gb():
    free, _ = torch.cuda.mem_get_info()
    return free / 2 ** 30


def test_dynamic_z_full_size_sampled():
    Ls = [256, 512, 1024, 2048]
    cfgs = [Config(Lx=L, Ly=L, n_replicas=256, seed=1, init_mode=XY_INIT_ORDERED, knots=((0,), (TC,)),
                   n_total=10 ** 5) for L in Ls]
    if _free_gb() < 2 * 8 * sum(c.sites for c in cfgs) / 2 ** 30 + 8:
        pytest.skip("not enough free device memory for the full-size batch")
    lat = Lattice(cfgs)
    n, re = 11, 10  # records at steps 0 and 10
    rec = lat.step(n, record_every=re).cpu().numpy()[:, :2]
    torch.cuda.synchronize()
    picks = [(0, 255), (1, 17), (2, 128), (3, 3)]  # (config, replica), one per L
    params = dict(inputs.PAPER)

    def replay(pick):
        c, r = pick
        L = Ls[c]
        th = oracle.init_theta(L, L, c, r, 1, XY_INIT_ORDERED)
        om = np.zeros_like(th)
        o_rec = oracle.run_lattice(L, L, c, r, 1, params, ([0], [TC]), 0, n, th, om, re)
        return th, o_rec

    with ThreadPoolExecutor(max_workers=len(picks)) as ex:
        results = list(ex.map(replay, picks))
    for (c, r), (th, o_rec) in zip(picks, results):
        b = 256 * c + r
        g = lat.lattice_view(lat.theta, b).cpu().numpy().ravel()
        assert circ_diff(g, th).max() < 1e-5, (c, r)
        assert o_rec.shape[0] == 2
        assert np.abs(rec[b, :, 0] - o_rec[:, 0]).max() < 2e-5
        assert np.abs(rec[b, :, 1] - o_rec[:, 1]).max() < 2e-4 * max(1.0, np.abs(o_rec[:, 1]).max())
    assert np.isfinite(rec).all()
    _, steps = lat.observe()
    assert list(steps) == [n] * len(Ls)
    lat.close()


def _kz_configs():
    tau_q = np.round(np.logspace(2, 5, 16)).astype(np.int64)
    n_eq = 1000
    cfgs = []
    for tq in tau_q:
        ramp = int(round(1.5 * tq))
        for eta in (0.1, 1.0, 10.0):
            for h in (0.5, 1.0, 2.0):
                cfgs.append(Config(Lx=1024, Ly=1024, n_replicas=64, seed=1, init_mode=XY_INIT_UNIFORM,
                                   params=dict(eta=eta, h=h),
                                   knots=((0, n_eq, n_eq + ramp), (1.5 * TC, 1.5 * TC, 0.0)),
                                   n_total=n_eq + ramp))
    return cfgs


def test_kibble_zurek_full_size_sampled():
    cfgs = _kz_configs()
    assert len(cfgs) * 64 == 9216
    if _free_gb() < 2 * 8 * sum(c.sites for c in cfgs) / 2 ** 30 + 12:
        pytest.skip("not enough free device memory for the full-size batch")
    lat = Lattice(cfgs)
    N = 1024 * 1024
    picks = [(0, 0), (70, 33), (143, 63)]  # (config, replica): tau_Q = 1e2 / ~2.5e3 / 1e5, all eta and h corners
    bs = [64 * c + r for c, r in picks]
    # domain labels of the random initial state, bit-exact against the oracle's flood fill
    labels, _, _ = lat.label_domains(bs[1], 1, hist_cap=1 << 16)
    th0 = [lat.lattice_view(lat.theta, b).cpu().numpy().ravel().copy() for b in bs]
    lab_o, _ = oracle.ccl(1024, 1024, th0[1])
    assert np.array_equal(labels[0].cpu().numpy().ravel(), lab_o)
    # step one BBK step at a time over the whole batch; the oracle replays the
    # sampled lattices from the same initial angles
    n = 6
    o_th = [t.astype(np.float64) for t in th0]
    o_om = [np.zeros(N) for _ in picks]
    events = [[] for _ in picks]
    for k in range(n):
        lat.step(1)

        def one(i):
            c, r = picks[i]
            cf = cfgs[c]
            oracle.run_lattice(1024, 1024, c, r, 1, dict(inputs.PAPER, **cf.params), cf.knots, k, 1, o_th[i], o_om[i])

        with ThreadPoolExecutor(max_workers=len(picks)) as ex:
            list(ex.map(one, range(len(picks))))
        for i, b in enumerate(bs):
            g = lat.lattice_view(lat.theta, b).cpu().numpy().ravel().astype(np.float64)
            raw = np.abs(g - o_th[i])
            events[i] += list(np.nonzero((raw > PI / 2) & (circ_diff(g, o_th[i]) < 1e-3))[0])
    for i, b in enumerate(bs):
        g = lat.lattice_view(lat.theta, b).cpu().numpy().ravel()
        d = circ_diff(g, o_th[i])
        assert (d <= 1e-4).mean() > 1 - 1e-4
        # sites beyond 1e-4 rad lie next to a cusp event (the two sides on
        # opposite ends of the wrap cut at +-pi/2 after some step)
        ev = np.array(sorted(set(int(e) for e in events[i])), dtype=np.int64)
        for s in np.nonzero(d > 1e-4)[0]:
            x, y = s % 1024, s // 1024
            dx = np.abs(ev % 1024 - x)
            dy = np.abs(ev // 1024 - y)
            near = (np.minimum(dx, 1024 - dx) <= 16) & (np.minimum(dy, 1024 - dy) <= 4)
            assert ev.size and near.any(), (picks[i], int(s), float(d[s]))
    _, steps = lat.observe()
    assert list(steps) == [n] * len(cfgs)
    lat.close()


def test_differentiation_full_size():
    """The differentiation workload at full size: 64 lattices of 256 x 256 at
    T_c from the ordered state (as 64 one-replica configurations, so that the
    gradients come back per lattice).  A 200-step adjoint (checkpoint every
    100) against the oracle's FP64 adjoint on two sampled lattices; the full
    2000-step adjoint with the states integrated backward against the stored
    recompute (beyond a few hundred steps at T_c the FP32 and FP64
    trajectories part, so the oracle is compared on the shorter window)."""
    from paper_2409_06412_gb300 import XY_ADJOINT_BACKWARD, XY_ADJOINT_RECOMPUTE
    cfgs = [Config(Lx=256, Ly=256, n_replicas=1, seed=1, init_mode=XY_INIT_ORDERED, knots=((0,), (TC,)),
                   n_total=10 ** 9) for _ in range(64)]
    lat = Lattice(cfgs)
    lat.step(10)
    snap = lat.save()
    picks = [5, 42]
    th0 = [lat.lattice_view(lat.theta, c).cpu().numpy().ravel().astype(np.float64) for c in picks]
    om_full = lat.omega_full().cpu().numpy().reshape(64, -1)
    om0 = [om_full[c].astype(np.float64) for c in picks]
    n = 200
    obj, grads = lat.adjoint(n, checkpoint_every=100, w_E=1.0, w_M=1.0)

    def ref(i):
        c = picks[i]
        return oracle.adjoint_lattice(256, 256, c, 0, 1, {}, ([0], [TC]), 10, n, th0[i].copy(), om0[i].copy(), 1.0,
                                      1.0)

    with ThreadPoolExecutor(max_workers=len(picks)) as ex:
        res = list(ex.map(ref, range(len(picks))))
    for i, c in enumerate(picks):
        o_g = res[i][1] / (64 * n)
        assert_grads_close(grads[c][None], o_g[None], 1e-3, what=f"lattice {c}")
    # 2000 steps, both schedules from the same snapshot
    out = {}
    for mode in (XY_ADJOINT_BACKWARD, XY_ADJOINT_RECOMPUTE):
        lat.load(snap)
        lat.set_adjoint_mode(mode)
        out[mode] = lat.adjoint(2000, checkpoint_every=100, w_E=1.0, w_M=1.0)
    (ob, gb), (orc, grc) = out[XY_ADJOINT_BACKWARD], out[XY_ADJOINT_RECOMPUTE]
    assert ob == pytest.approx(orc, rel=1e-5)
    assert_grads_close(gb, grc, 1e-3, what="2000 steps, backward against recompute")
    lat.close()
