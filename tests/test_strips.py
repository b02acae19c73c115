"""Row-strip decomposition of one lattice (the multi-GPU plan, checked on the
CPU): the plan covers every row once and feeds each ghost row from its owner;
a lattice stepped by the oracle in strips, with halo rows exchanged every K_t
steps, equals the whole-lattice oracle run bit for bit, in one process for
several worlds and over two gloo ranks; the rows that stay exact within a
window are the ones the plan claims, and one ghost row fewer is not enough."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2409_06412_gb300 import strips as st
from tests import inputs

PARAMS = dict(oracle.PAPER_PARAMS, dt=0.05)
KNOTS = ([0, 6], [3.0, 1.0])    # a quench inside the run
FIELD = ([2, 9], [0.5, 1.5])    # and a field ramp
COUPLINGS = ([3, 8], [1.0, 0.4], [1.0, 2.5])  # and coupling profiles (1 at the start)
SEED = 5


def _whole_start(Lx, Ly, seed=SEED):
    th = oracle.init_theta(Lx, Ly, 0, 0, seed, 0)
    rng = np.random.default_rng(seed)
    om = rng.normal(0.0, 1.0, Lx * Ly)
    return th, om


def _whole_run(Lx, Ly, n, every, couplings=None):
    th, om = _whole_start(Lx, Ly)
    rec = oracle.run_lattice(Lx, Ly, 0, 0, SEED, PARAMS, KNOTS, 0, n, th, om, record_every=every, field=FIELD,
                             couplings=couplings)
    return th.reshape(Ly, Lx), om.reshape(Ly, Lx), rec


def _buffers(s: st.Strip):
    th, om = _whole_start(s.Lx, s.Ly)
    F = oracle.force(s.Lx, s.Ly, dict(PARAMS, h=PARAMS["h"] * oracle.field_scale(0, FIELD)), th)
    return [s.fill(a.reshape(s.Ly, s.Lx)) for a in (th, om, F)]


def _step_strip(s: st.Strip, bufs, k0, n, every, couplings=None):
    th, om, F = bufs
    return oracle.run_strip(s.Lx, s.Ly, s.buffer_y0, 0, 0, SEED, PARAMS, KNOTS, k0, n, th, om, F,
                            rows=(s.halo, s.halo + s.rows), record_every=every, field=FIELD, couplings=couplings)


# ---------------------------------------------------------------------------
# the plan
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("Ly,world,k_t,align", [(64, 2, 2, 8), (22, 3, 3, 1), (24, 5, 1, 1), (40, 4, 4, 2),
                                               (16, 1, 3, 1), (1024, 8, 2, 64)])
def test_plan_covers_each_row_once_and_feeds_ghosts_from_their_owners(Ly, world, k_t, align):
    Lx = 12
    plan = st.plan_strips(Lx, Ly, world, k_t, align)
    owner = np.full(Ly, -1)
    for s in plan:
        assert s.rows % align == 0 and s.rows >= k_t
        rows = s.global_rows()[s.owned]
        assert np.all(owner[rows] == -1)
        owner[rows] = s.rank
    assert np.all(owner >= 0)
    assert max(s.rows for s in plan) - min(s.rows for s in plan) <= align
    copies = st.halo_copies(plan)
    assert len(copies) == 2 * world
    filled = {s.rank: np.zeros(s.buffer_rows, bool) for s in plan}
    for c in copies:
        src, dst = plan[c.src], plan[c.dst]
        g_src = src.global_rows()[c.src_row:c.src_row + c.n_rows]
        g_dst = dst.global_rows()[c.dst_row:c.dst_row + c.n_rows]
        assert np.array_equal(g_src, g_dst)
        assert np.all(owner[g_src] == c.src)                                        # read from the owner
        own = np.zeros(src.buffer_rows, bool)
        own[src.owned] = True
        assert own[c.src_row:c.src_row + c.n_rows].all()                            # owned rows only
        assert not filled[c.dst][c.dst_row:c.dst_row + c.n_rows].any()
        filled[c.dst][c.dst_row:c.dst_row + c.n_rows] = True
    for s in plan:                                                                  # exactly the ghost rows
        ghost = np.ones(s.buffer_rows, bool)
        ghost[s.owned] = False
        assert np.array_equal(filled[s.rank], ghost)
    assert st.bytes_per_exchange(plan, 8) == 2 * world * k_t * Lx * 8


def test_plan_rejects_what_it_cannot_feed():
    with pytest.raises(ValueError):
        st.plan_strips(8, 10, 4, 3)          # strips of 2-3 rows, halo 3
    with pytest.raises(ValueError):
        st.plan_strips(8, 20, 3, 1, align=8)  # 20 rows are not units of 8
    with pytest.raises(ValueError):
        st.plan_strips(8, 16, 3, 1, align=8)  # two units for three ranks
    with pytest.raises(ValueError):
        st.plan_strips(8, 16, 2, 0)
    assert st.window_lengths(7, 3) == [3, 3, 1] and st.window_lengths(6, 2) == [2, 2, 2]
    s = st.plan_strips(8, 32, 2, 3)[0]
    assert s.recompute_fraction() == pytest.approx(2 / 16)
    with pytest.raises(ValueError):
        s.exact_rows(4)


# ---------------------------------------------------------------------------
# split runs against the whole lattice (one process, all ranks' buffers)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("couplings", [None, COUPLINGS], ids=["field", "field+couplings"])
@pytest.mark.parametrize("Lx,Ly,world,k_t,n", [(10, 12, 2, 2, 9), (8, 22, 3, 3, 10), (6, 20, 4, 1, 7),
                                               (7, 9, 1, 2, 5), (12, 16, 2, 4, 11)])
def test_split_run_equals_the_whole_lattice_bit_for_bit(Lx, Ly, world, k_t, n, couplings):
    every = 2
    th_w, om_w, rec_w = _whole_run(Lx, Ly, n, every, couplings)
    plan = st.plan_strips(Lx, Ly, world, k_t)
    copies = st.halo_copies(plan)
    bufs = [_buffers(s) for s in plan]
    recs = [[] for _ in plan]
    k = 0
    for w in st.window_lengths(n, k_t):
        for s, b in zip(plan, bufs):
            recs[s.rank].append(_step_strip(s, b, k, w, every, couplings))
        k += w
        st.apply_copies(bufs, copies)
    th = np.empty((Ly, Lx))
    om = np.empty((Ly, Lx))
    for s, b in zip(plan, bufs):
        th[s.global_rows()[s.owned]] = b[0][s.owned]
        om[s.global_rows()[s.owned]] = b[1][s.owned]
    assert np.array_equal(th, th_w) and np.array_equal(om, om_w)
    # after the exchange every buffer row is exact again, ghost rows included
    for s, b in zip(plan, bufs):
        assert np.array_equal(b[0], th_w[s.global_rows()])
    # moments: per-rank raw sums over owned rows, added across ranks
    total = sum(np.concatenate(r) for r in recs) / (Lx * Ly)
    assert total.shape == rec_w.shape
    np.testing.assert_allclose(total, rec_w, rtol=1e-12, atol=1e-13)


def test_rows_exact_within_a_window_are_the_planned_ones():
    """Ghost rows go stale one per step at each end: after j steps of a window
    omega is NaN outside exact_rows(j) and exact inside."""
    Lx, Ly, k_t = 8, 24, 4
    s = st.plan_strips(Lx, Ly, 2, k_t)[1]
    b = _buffers(s)
    th_w, om_w = _whole_start(Lx, Ly)
    for j in range(1, k_t + 1):
        _step_strip(s, b, j - 1, 1, 0)
        th_w = th_w.copy()
        oracle.run_lattice(Lx, Ly, 0, 0, SEED, PARAMS, KNOTS, j - 1, 1, th_w, om_w, field=FIELD)
        lo, hi = s.exact_rows(j)
        ok = np.zeros(s.buffer_rows, bool)
        ok[lo:hi] = True
        assert np.all(np.isnan(b[1][~ok]))
        assert np.array_equal(b[1][ok], om_w.reshape(Ly, Lx)[s.global_rows()][ok])


def test_one_ghost_row_fewer_than_the_window_is_not_enough():
    """K_t steps between exchanges over K_t - 1 ghost rows: the owned rows at
    the strip edges are no longer exact."""
    Lx, Ly, k_t = 8, 16, 3
    plan = st.plan_strips(Lx, Ly, 2, k_t - 1)
    bufs = [_buffers(s) for s in plan]
    for s, b in zip(plan, bufs):
        _step_strip(s, b, 0, k_t, 0)
    for s, b in zip(plan, bufs):
        edge = b[1][s.owned]
        assert np.isnan(edge[0]).all() and np.isnan(edge[-1]).all()


# ---------------------------------------------------------------------------
# two gloo ranks
# ---------------------------------------------------------------------------

def _rank(rank, world, port, Lx, Ly, k_t, n, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = st.plan_strips(Lx, Ly, world, k_t)
        s = plan[rank]
        bufs = _buffers(s)
        rec, k = [], 0
        for w in st.window_lengths(n, k_t):
            rec.append(_step_strip(s, bufs, k, w, 3))
            k += w
            st.exchange(s, bufs, plan)
        out[rank] = (bufs[0][s.owned].tolist(), bufs[1][s.owned].tolist(), np.concatenate(rec).tolist(),
                     np.isfinite(np.stack(bufs)).all())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("k_t", [1, 3])
def test_split_run_over_two_gloo_ranks(k_t):
    Lx, Ly, n = 12, 14, 8
    oracle.build()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, Lx, Ly, k_t, n, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    th_w, om_w, rec_w = _whole_run(Lx, Ly, n, 3)
    plan = st.plan_strips(Lx, Ly, 2, k_t)
    th, om = np.empty((Ly, Lx)), np.empty((Ly, Lx))
    for s in plan:
        t, o, _, finite = out[s.rank]
        assert finite                      # ghost rows refilled by the last exchange
        th[s.global_rows()[s.owned]] = t
        om[s.global_rows()[s.owned]] = o
    assert np.array_equal(th, th_w) and np.array_equal(om, om_w)
    total = (np.array(out[0][2]) + np.array(out[1][2])) / (Lx * Ly)
    np.testing.assert_allclose(total, rec_w, rtol=1e-12, atol=1e-13)
