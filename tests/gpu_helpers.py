"""Helpers of the GPU parity tests: build matching GPU lattices and oracle runs
from one seeded specification (tests/inputs.py)."""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from paper_2409_06412_gb300 import Config, Lattice, XY_INIT_USER

PI = math.pi


def gpu_config(spec: dict) -> Config:
    p = dict(spec["params"])
    return Config(Lx=spec["Lx"], Ly=spec["Ly"], n_replicas=spec["n_rep"], seed=spec["seed"],
                  init_mode=spec.get("init_mode", XY_INIT_USER), params=p, knots=spec["knots"],
                  n_total=spec["n_total"])


def make_pair(specs, thetas, omegas=None, path=None):
    """GPU lattice with user-initialised state, and oracle state arrays (float64
    copies of the same float32 values).  thetas[c]: (n_rep, N) float32."""
    th = np.concatenate([t.reshape(-1) for t in thetas]).astype(np.float32)
    if omegas is None:
        om = np.zeros_like(th)
    else:
        om = np.concatenate([w.reshape(-1) for w in omegas]).astype(np.float32)
    cfgs = []
    for s in specs:
        s = dict(s)
        s["init_mode"] = XY_INIT_USER
        cfgs.append(gpu_config(s))
    lat = Lattice(cfgs, theta=torch.from_numpy(th).cuda(), omega=torch.from_numpy(om).cuda())
    if path is not None:
        lat.set_path(path)
    o_th = [t.astype(np.float64).reshape(s["n_rep"], -1).copy() for t, s in zip(thetas, specs)]
    if omegas is None:
        o_om = [np.zeros_like(t) for t in o_th]
    else:
        o_om = [w.astype(np.float64).reshape(s["n_rep"], -1).copy() for w, s in zip(omegas, specs)]
    return lat, o_th, o_om


def circ_diff(a, b):
    """|a - b| modulo pi, in [0, pi/2]."""
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % PI
    return np.minimum(d, PI - d)


def split_state(lat: Lattice, t: torch.Tensor):
    """Per configuration (n_rep, N) float64 arrays of a flat state tensor."""
    a = t.detach().cpu().numpy().astype(np.float64)
    out, off = [], 0
    for c in lat.configs:
        n = c.sites
        out.append(a[off:off + n].reshape(c.n_replicas, -1))
        off += n
    return out


def theta_parity(gpu_th, o_th, tol=1e-4):
    """Max circular |dtheta|; returns (max, list of violating (cfg, rep, site))."""
    worst, bad = 0.0, []
    for c, (g, o) in enumerate(zip(gpu_th, o_th)):
        d = circ_diff(g, o)
        worst = max(worst, float(d.max()))
        for r, s in zip(*np.nonzero(d > tol)):
            bad.append((c, int(r), int(s)))
    return worst, bad
