"""Resident stepper on thread-block clusters: a lattice split over 2..16
blocks that exchange their bands' edge rows through distributed shared memory
must give the same bits as the plain one-launch-per-step path, and records
that agree with it.

The block and cluster size of a resident shape come from the autotuner's
cache (XY_TUNE_CACHE, read once per process), so each pinned choice runs in a
child process with a cache file that holds it.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import textwrap

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import json, sys
    import numpy as np
    import torch
    sys.path.insert(0, sys.argv[1])
    sys.path.insert(0, sys.argv[1] + "/tests")
    from inputs import PAPER, angles
    from paper_2409_06412_gb300 import Config, Lattice, XY_INIT_USER, XY_PATH_PLAIN
    Lx, Ly, n_rep, stag = (int(a) for a in sys.argv[2:6])
    p = dict(PAPER)
    p["staggered"] = float(stag)
    th = angles(n_rep, Lx, Ly, seed=21).reshape(-1)
    lats = []
    for path in (None, XY_PATH_PLAIN):
        cfg = Config(Lx=Lx, Ly=Ly, n_replicas=n_rep, seed=5, init_mode=XY_INIT_USER, params=p,
                     knots=((0, 60), (2.5, 1.2)), n_total=10**6)
        lat = Lattice([cfg], theta=torch.from_numpy(th).cuda(), omega=torch.zeros(th.size).cuda())
        if path is not None:
            lat.set_path(path)
        lats.append(lat)
    recs = [lat.step(45, record_every=3) for lat in lats]
    for lat in lats:
        lat.step(38)
    torch.cuda.synchronize()
    a, b = lats
    ra, rb = (r.cpu().numpy() for r in recs)
    out = {
        "theta_equal": bool(torch.equal(a.theta, b.theta)),
        "omega_equal": bool(torch.equal(a.omega, b.omega)),
        "rec_same_slots": bool(np.array_equal(np.isnan(ra), np.isnan(rb))),
        "rec_count": int(np.sum(~np.isnan(ra[..., 0]))),
        "rec_max_diff": float(np.nanmax(np.abs(ra - rb))),
    }
    print("RESULT " + json.dumps(out))
""")


def gpu_key_name() -> str:
    return torch.cuda.get_device_name(0).replace(" ", "_").replace("|", "_")


@pytest.mark.gpu
@pytest.mark.parametrize("Lx,Ly,n_rep,threads,csize,stag", [
    (64, 64, 1, 512, 8, 0),     # one row per band, exports across blocks
    (64, 64, 1, 64, 16, 1),     # four blocks of 4 one-row bands, staggered M
    (64, 64, 2, 128, 4, 0),     # two rows per band
    (32, 48, 3, 64, 2, 0),      # three rows per band, narrow rows (8 lanes)
    (128, 32, 1, 256, 4, 1),    # full-warp rows, two rows per band
])
def test_cluster_resident_matches_plain(tmp_path, Lx, Ly, n_rep, threads, csize, stag):
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{gpu_key_name()}|resident|{Lx}|{Ly}|{n_rep} {threads} {csize}\n")
    env = dict(os.environ, XY_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(Lx), str(Ly), str(n_rep), str(stag)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["theta_equal"] and res["omega_equal"], res
    # records: the same site terms, summed in a different order
    assert res["rec_same_slots"] and res["rec_count"] == n_rep * 15, res
    assert res["rec_max_diff"] < 1e-5, res


SHARED = textwrap.dedent(r"""
    import sys
    import torch
    sys.path.insert(0, sys.argv[1])
    from paper_2409_06412_gb300 import Config, Lattice, XY_PATH_PLAIN
    big = Lattice([Config(Lx=128, Ly=128, n_replicas=1, seed=3, init_mode=0, n_total=10**6)])
    big.step(40)
    ref = Lattice([Config(Lx=128, Ly=128, n_replicas=1, seed=3, init_mode=0, n_total=10**6)])
    ref.set_path(XY_PATH_PLAIN)
    ref.step(40)
    # a second object whose shape runs on the same kernel instance with less shared memory
    small = Lattice([Config(Lx=64, Ly=64, n_replicas=1, seed=4, init_mode=0, n_total=10**6)])
    small.step(40)
    big.step(40)   # must still launch with its own (larger) shared memory
    ref.step(40)
    torch.cuda.synchronize()
    print("RESULT", int(torch.equal(big.theta, ref.theta) and torch.equal(big.omega, ref.omega)))
""")


@pytest.mark.gpu
def test_resident_shapes_sharing_a_kernel_keep_their_shared_memory(tmp_path):
    """Two objects whose resident shapes use the same kernel instance (512
    threads, several rows per band) with different shared memory: preparing
    the smaller one after the larger must not take the larger one's shared
    memory away (the opt-in is an attribute of the kernel, not of a shape)."""
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{gpu_key_name()}|resident|128|128|1 512 1\n{gpu_key_name()}|resident|64|64|1 512 1\n")
    env = dict(os.environ, XY_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", SHARED, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1] == "RESULT 1"
