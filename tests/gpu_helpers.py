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


def stepwise_parity(lat, specs, o_th, o_om, n_steps, tol=1e-4, reach=(16, 4), factor=30.0, cap=1e-3):
    """Step the GPU lattice and the oracle one step at a time and classify the
    final angle differences.

    A site passes if its circular |dtheta| <= tol.  Two kinds of site may
    exceed tol, and both are returned with evidence:
      * near a cusp event: after some step the two sides held angles on
        opposite ends of the wrap cut at +-pi/2 (raw difference > pi/2, circular
        difference small), where the periodically continued field potential
        has its kink; sites within `reach` = (dx, dy) periodic lattice steps of
        such an event are reported as cusp-explained;
      * ill-conditioned: a second oracle run that stores its state in binary32
        after every step (the rounding any FP32 state must suffer) departs
        from the FP64 oracle by `sens` at that site; a site with
        |dtheta| <= factor * sens and <= cap is limited by the conditioning of
        the trajectory (unstable anti-aligned bonds amplify the rounding),
        not by the kernel.  The factor covers the ratio of the kernel's
        per-step arithmetic error (hardware sine/cosine ~3.6e-7, Box-Muller
        ~1e-6 per Gaussian) to the bare binary32 rounding of the state.
    Everything else is `unexplained` and fails the tests."""
    step_now = [0] * len(specs)
    r_th = [t.astype(np.float32).astype(np.float64) for t in o_th]
    r_om = [w.astype(np.float32).astype(np.float64) for w in o_om]
    r_step = [0] * len(specs)
    events = []
    for k in range(n_steps):
        lat.step(1)
        oracle.run_batch(specs, o_th, o_om, step_now, 1)
        oracle.run_batch(specs, r_th, r_om, r_step, 1)
        for c in range(len(specs)):
            r_th[c][:] = r_th[c].astype(np.float32)
            r_om[c][:] = r_om[c].astype(np.float32)
        g = split_state(lat, lat.theta)
        for c, s_ in enumerate(specs):
            raw = np.abs(g[c] - o_th[c])
            circ = circ_diff(g[c], o_th[c])
            for r, site in zip(*np.nonzero((raw > PI / 2) & (circ < 1e-3))):
                events.append((c, int(r), int(site), k))
    g = split_state(lat, lat.theta)
    unexplained, cusp, ill, worst_all = [], [], [], 0.0
    n_sites, n_ok = 0, 0
    for c, s_ in enumerate(specs):
        Lx, Ly = s_["Lx"], s_["Ly"]
        d = circ_diff(g[c], o_th[c])
        sens = circ_diff(r_th[c], o_th[c])
        worst_all = max(worst_all, float(d.max()))
        n_sites += d.size
        n_ok += int((d <= tol).sum())
        for r, site in zip(*np.nonzero(d > tol)):
            x, y = site % Lx, site // Lx
            near = False
            for (ec, er, es, _) in events:
                if ec != c or er != r:
                    continue
                ex, ey = es % Lx, es // Lx
                dx = min(abs(x - ex), Lx - abs(x - ex))
                dy = min(abs(y - ey), Ly - abs(y - ey))
                if dx <= reach[0] and dy <= reach[1]:
                    near = True
                    break
            rec = (c, int(r), int(site), float(d[r, site]), float(sens[r, site]))
            if near:
                cusp.append(rec)
            elif d[r, site] <= factor * sens[r, site] and d[r, site] <= cap:
                ill.append(rec)
            else:
                unexplained.append(rec)
    return dict(worst_all=worst_all, unexplained=unexplained, cusp=cusp, ill=ill, events=events,
                step_now=step_now, frac_within_tol=n_ok / n_sites, n_sites=n_sites)
