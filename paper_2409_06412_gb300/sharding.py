"""Splitting a batch of configurations over ranks (one process per GPU).

The lattices of a batch are independent, so the path shards with no
data-path collective: each rank steps its share, and only the FP64 moment
sums (six numbers per configuration) are added across ranks at the end.
Replica ids and configuration ids are kept global (``Config.cfg_id``,
``Config.replica0``), so the sharded run reproduces the unsharded one bit for
bit.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from .lattice import Config


def cost(c: Config, steps: int | None = None) -> float:
    """Site-updates of one replica of a configuration over its run."""
    n = c.n_total if steps is None else min(steps, c.n_total)
    return float(c.Lx) * c.Ly * max(n, 0)


def partition(configs: list[Config], world: int, steps: int | None = None, chunk: int = 1):
    """Assign replicas (in blocks of ``chunk``) to ranks, heaviest first,
    each to the least loaded rank (longest-processing-time rule).  Returns
    per rank a list of Configs carrying global ``cfg_id`` / ``replica0`` and
    the per-rank load."""
    items = []
    for ci, c in enumerate(configs):
        for r0 in range(0, c.n_replicas, chunk):
            nr = min(chunk, c.n_replicas - r0)
            items.append((cost(c, steps) * nr, ci, r0, nr))
    items.sort(key=lambda t: (-t[0], t[1], t[2]))
    load = [0.0] * world
    owned = [[] for _ in range(world)]
    for w, ci, r0, nr in items:
        rank = min(range(world), key=lambda k: (load[k], k))
        load[rank] += w
        owned[rank].append((ci, r0, nr))
    shards = []
    for rank in range(world):
        out = []
        for ci, r0, nr in sorted(owned[rank]):
            c = configs[ci]
            gid = c.cfg_id if c.cfg_id >= 0 else ci
            out.append(replace(c, n_replicas=nr, cfg_id=gid, replica0=c.replica0 + r0))
        shards.append(out)
    return shards, load


def config_ids(shard: list[Config]) -> list[int]:
    return [c.cfg_id for c in shard]


def reduce_moments(local_moments: np.ndarray, local_ids: list[int], n_global: int, group=None) -> np.ndarray:
    """Sum per-configuration FP64 moments (rows of 6) over ranks:
    scatter the local rows into a global (n_global, 6) table and all-reduce
    it (gloo on CPU, NCCL on GPU)."""
    import torch
    import torch.distributed as dist
    table = np.zeros((n_global, 6), dtype=np.float64)
    for row, gid in zip(local_moments, local_ids):
        table[gid] += row
    if dist.is_available() and dist.is_initialized():
        backend = dist.get_backend(group)
        dev = "cuda" if backend == "nccl" else "cpu"
        t = torch.from_numpy(table).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        table = t.cpu().numpy()
    return table
