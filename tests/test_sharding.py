"""Sharding of a batch over ranks: balance, global noise ids, and the FP64
moment reduction over a world of two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2409_06412_gb300.lattice import Config
from paper_2409_06412_gb300.sharding import config_ids, partition, reduce_moments


def _quench_batch():
    # 16 quench rates x 3 eta x 3 h, 64 replicas each (uneven lengths)
    taus = np.logspace(2, 5, 16)
    cfgs = []
    for tq in taus:
        for eta in (0.1, 1.0, 10.0):
            for h in (0.5, 1.0, 2.0):
                cfgs.append(Config(Lx=1024, Ly=1024, n_replicas=64, params=dict(eta=eta, h=h),
                                   n_total=int(1.5 * tq) + 1000))
    return cfgs


def test_partition_covers_every_replica_once_with_global_ids():
    cfgs = _quench_batch()
    for world in (1, 2, 3, 8):
        shards, load = partition(cfgs, world, chunk=4)
        seen = {}
        for shard in shards:
            for c in shard:
                for r in range(c.replica0, c.replica0 + c.n_replicas):
                    key = (c.cfg_id, r)
                    assert key not in seen
                    seen[key] = 1
        assert len(seen) == sum(c.n_replicas for c in cfgs)
        assert max(load) <= min(load) * 1.05 + max(float(c.Lx * c.Ly * c.n_total * 4) for c in cfgs)


def test_partition_balances_uneven_lengths():
    cfgs = _quench_batch()
    shards, load = partition(cfgs, 8, chunk=1)
    assert max(load) / min(load) < 1.01


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfgs = [Config(Lx=64, Ly=64, n_replicas=5), Config(Lx=128, Ly=128, n_replicas=3),
            Config(Lx=256, Ly=256, n_replicas=2)]
    shards, _ = partition(cfgs, world)
    mine = shards[rank]
    # stand-in per-configuration sums: a function of the (global cfg, replica) ids
    local = np.array([[c.n_replicas, c.cfg_id + 0.5, c.replica0 * 2.0, 1.0, 2.0, 3.0] for c in mine])
    table = reduce_moments(local, config_ids(mine), len(cfgs))
    out[rank] = table.tolist()
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_moment_reduction_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    a, b = np.array(out[0]), np.array(out[1])
    assert np.array_equal(a, b)
    # replica counts add up to the unsharded batch
    assert a[:, 0].tolist() == [5, 3, 2]
