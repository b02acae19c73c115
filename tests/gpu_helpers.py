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
                  n_total=spec["n_total"], field=spec.get("field"),
                  couplings=spec.get("couplings"))


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


# ---------------------------------------------------------------------------
# FP32 error model of one step of the CUDA kernels, for the first-order bound
# of the parity tests.
#
# A stepping kernel advances (theta_k, v_k) to (theta_{k+1}, v_{k+1}) in
# binary32 with round-to-nearest (unit roundoff U = 2^-24) and the fast
# hardware sine, cosine, log2 and reciprocal square root.  Against the exact
# step from the same binary32 state it makes a local error bounded, site by
# site and step by step, by
#   |d theta_{k+1}| <= A + U |theta_{k+1}| + C [the angle was wrapped]
#   |d v_{k+1}|     <= 2 dg_k + U g_max + 5.1 U |omega_k|
#   dg_k = dt/2 dF + dt/2 F_max U + c_k (EG(r_k) + 5.5 U |n_k|) + U g_max
# (plus dg_0 + 3.1 U |omega_0| for the priming of v_0).  The FP64 oracle
# propagates these along its own trajectory through the linearised dynamics
# (oracle.theta_sensitivity): to first order the kernel's angle after n steps
# lies within sum |lambda| w of the oracle's, w the bounds above.
#
# Where the constants come from (xy_device.cuh):
#   sin q theta, cos q theta: q theta exact (q = 2); hardware error <= ESC;
#   sin p theta: p theta rounded (<= U p pi/2); hardware error <= ESP;
#   neighbour sums s_l + s_r: <= 2 ESC + 2U; bond terms a = s cx - c sx
#     (|a| <= 2): <= 8 ESC + 8U;
#   F = -qJ_par a_x - qJ_perp a_y + hp sin p theta, each constant rounded once
#     (relative U), three roundings of the sums: dF below;
#   the noise c n: the Box-Muller map's absolute error EG(r) = ER1 / r +
#     (ERR + ETRIG + 2U) r at pair radius r (ER1 / r: the absolute error of
#     the hardware log2 near 1, 2^-22 on [1/2, 2], seen through r = sqrt(-2 ln u);
#     ERR: the relative error of the radius elsewhere; ETRIG: the error of
#     the hardware sine and cosine of the angle); c = amp sqrt(T) from an FP32
#     schedule (relative <= 4.5U) and one more product;
#   g = dt/2 F + c n, omega = (v + g) / (1 + a), v' = (1 - a) omega + g with
#     the constants rounded once and one rounding per operation;
#   theta' = theta + dt v' (one rounding, dt rounded: A = dt U (|omega| + |g|)max)
#     and the wrap, which subtracts the binary32 pi at most twice:
#     C = 2 |pi - fl(pi)| + U pi.
# ESC, ESP, ER1, ERR and ETRIG are checked by exhaustive sweeps of the
# hardware functions over every argument the kernels can form
# (tests/test_gpu_fp32_model.py).
# ---------------------------------------------------------------------------

U32 = 2.0 ** -24
ESC = 2.0 ** -21.2    # hardware sin / cos of q theta, |theta| <= pi/2 (just past |q theta| = pi)
ESP = 2.0 ** -20.5    # hardware sin of fl(p theta), |p theta| <= 2.5 pi / 2
ER1 = math.log(2.0) * 2.0 ** -22   # radius error from the absolute error of log2 near 1, times r
ERR = 4.5e-7          # relative error of the radius away from u = 1
ETRIG = 4.5e-7        # error of the hardware sine / cosine of the Box-Muller angle
R_MAX = math.sqrt(-2.0 * math.log(2.0 ** -24))  # largest radius: u0 = 2^-24
PI_F32_ERR = abs(float(np.float32(math.pi)) - math.pi)


def box_muller_error(r: np.ndarray) -> np.ndarray:
    """Bound on |g~ - g| of one unit Gaussian of a pair with radius r."""
    r = np.maximum(np.asarray(r, dtype=np.float64), 1e-12)
    return ER1 / r + (ERR + ETRIG + 2 * U32) * r


def _force_error(prm: dict, smax: float = 1.0, amax: float = 1.0, bmax: float = 1.0) -> tuple[float, float]:
    U = U32
    # the largest couplings of profiles J_par a(k), J_perp b(k)
    qJx, qJy = abs(prm["q"] * prm["J_par"]) * amax, abs(prm["q"] * prm["J_perp"]) * bmax
    hp = abs(prm["h"] * prm["p"]) * smax  # the largest field of a schedule h s(k)
    F_max = 2 * qJx + 2 * qJy + hp
    d_bond = 8 * ESC + 8 * U
    dF = (qJx * (1 + U) * d_bond + 2 * qJx * U + qJy * (1 + U) * d_bond + 2 * qJy * U
          + hp * (ESP + U * abs(prm["p"]) * math.pi / 2 + 2 * U) + U * (2 * qJy + hp) + U * F_max)
    return dF, F_max


def local_error_weights(spec: dict, cfg: int, rep: int, k0: int, n: int, theta: np.ndarray, omega: np.ndarray):
    """Per-site bounds (wt, wv), each (n, N), of the kernel's local error along
    the oracle trajectory theta, omega ((n + 1, N) each, steps k0 .. k0 + n)."""
    prm = inputs_params(spec)
    U = U32
    N = theta.shape[1]
    hdt, dt = 0.5 * prm["dt"], prm["dt"]
    field = spec.get("field")
    smax = max([1.0] if field is None else [abs(x) for x in field[1]])
    cpl = spec.get("couplings")
    amax = max([1.0] if cpl is None else [abs(x) for x in cpl[1]])
    bmax = max([1.0] if cpl is None else [abs(x) for x in cpl[2]])
    dF, F_max = _force_error(prm, smax, amax, bmax)
    if field is not None:
        dF += abs(prm["h"] * prm["p"]) * smax * 2 * U  # h p s(k): the scale and the product rounded
    if cpl is not None:  # -q J a(k), -q J b(k): the scales and the products rounded, times |bond sums| <= 2
        dF += 2 * 2 * U * (abs(prm["q"] * prm["J_par"]) * amax + abs(prm["q"] * prm["J_perp"]) * bmax)
    amps = np.array([0.5 * math.sqrt(2.0 * prm["eta"] * max(oracle.temperature(k0 + j, spec["knots"]), 0.0) * dt)
                     for j in range(n + 1)])
    g_max = hdt * F_max + amps.max() * R_MAX
    om_max = float(np.abs(omega).max()) if omega.size else 0.0
    wv = np.empty((n, N))
    for j in range(n):
        z = oracle.gauss(spec["seed"], cfg, rep, N, k0 + j)
        r = np.repeat(np.hypot(z[0::2], z[1::2]), 2)  # sites 4q, 4q+1 and 4q+2, 4q+3 share a radius
        dg = hdt * dF + hdt * F_max * U + amps[j] * (box_muller_error(r) + 5.5 * U * np.abs(z)) + U * g_max
        wv[j] = 2 * dg + U * g_max + 5.1 * U * np.abs(omega[j])
        if j == 0:  # the priming v_0 = (1 + a) omega_0 - g_0: one more perturbation of the same velocity
            wv[j] += dg + 3.1 * U * np.abs(omega[0])
    A = dt * U * (om_max + g_max)
    C = 2 * PI_F32_ERR + U * math.pi
    wrapped = np.abs(np.diff(theta, axis=0)) > math.pi / 2   # a drift is < 0.1 rad: a jump of ~pi is the wrap
    wt = A + U * np.abs(theta[1:]) + C * wrapped
    return wt, wv


def first_order_bound(spec: dict, cfg: int, rep: int, k0: int, n: int, theta0, omega0, sites):
    """(bound, rms) per site: the first-order bound of the kernel's angle error
    after n steps, and the spread if the local errors were independent and
    uniform within their bounds."""
    Lx, Ly = spec["Lx"], spec["Ly"]
    _, tth, tom = oracle.theta_sensitivity(Lx, Ly, cfg, rep, spec["seed"], spec["params"], spec["knots"], k0, n,
                                           theta0, omega0, [], trajectory=True, field=spec.get("field"),
                                           couplings=spec.get("couplings"))
    wt, wv = local_error_weights(spec, cfg, rep, k0, n, tth, tom)
    out = oracle.theta_sensitivity(Lx, Ly, cfg, rep, spec["seed"], spec["params"], spec["knots"], k0, n, theta0,
                                   omega0, sites, wt=wt, wv=wv, field=spec.get("field"),
                                   couplings=spec.get("couplings"))
    return out[:, 0], out[:, 1] / math.sqrt(3.0)


def inputs_params(spec: dict) -> dict:
    full = dict(oracle.PAPER_PARAMS)
    full.update(spec["params"])
    return full


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


def stepwise_parity(lat, specs, o_th, o_om, n_steps, tol=1e-4, reach=(16, 4)):
    """Step the GPU lattice and the oracle one step at a time and classify the
    final angle differences.

    A site passes if its circular |dtheta| <= tol.  Two kinds of site may
    exceed tol, and both are returned with evidence:
      * near a cusp event: after some step the two sides held angles on
        opposite ends of the wrap cut at +-pi/2 (raw difference > pi/2, circular
        difference small), where the periodically continued field potential
        has its kink; sites within `reach` = (dx, dy) periodic lattice steps of
        such an event are reported as cusp-explained;
      * FP32-conditioned: the difference stays within the first-order bound
        of the kernel's binary32 arithmetic at that site: the local error of
        every step (local_error_weights, derived from the operations of a
        step and the swept error of the hardware functions) propagated by the
        oracle's linearised dynamics along its own trajectory
        (oracle.theta_sensitivity).  Unstable anti-aligned bonds amplify
        rounding along random-start trajectories; this bound says by how much.
    Everything else is `unexplained` and fails the tests.  The result also
    carries the largest ratio |dtheta| / bound over the FP32-conditioned
    sites, and the largest |dtheta| / rms, rms being the spread the same local
    errors would give if they were independent and uniform within their
    bounds (a scale, not a criterion)."""
    step_now = [0] * len(specs)
    th_start = [t.copy() for t in o_th]
    om_start = [w.copy() for w in o_om]
    events = []
    for k in range(n_steps):
        lat.step(1)
        oracle.run_batch(specs, o_th, o_om, step_now, 1)
        g = split_state(lat, lat.theta)
        for c, s_ in enumerate(specs):
            raw = np.abs(g[c] - o_th[c])
            circ = circ_diff(g[c], o_th[c])
            for r, site in zip(*np.nonzero((raw > PI / 2) & (circ < 1e-3))):
                events.append((c, int(r), int(site), k))
    g = split_state(lat, lat.theta)
    unexplained, cusp, ill, worst_all = [], [], [], 0.0
    n_sites, n_ok = 0, 0
    worst_ratio, worst_z = 0.0, 0.0
    for c, s_ in enumerate(specs):
        Lx, Ly = s_["Lx"], s_["Ly"]
        d = circ_diff(g[c], o_th[c])
        worst_all = max(worst_all, float(d.max()))
        n_sites += d.size
        n_ok += int((d <= tol).sum())
        pending = {}
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
            if near:
                cusp.append((c, int(r), int(site), float(d[r, site])))
            else:
                pending.setdefault(int(r), []).append(int(site))
        if not pending:
            continue
        for r, sites in pending.items():
            bound, rms = first_order_bound(s_, c, r, 0, step_now[c], th_start[c][r], om_start[c][r], sites)
            for site, bnd, sd in zip(sites, bound, rms):
                rec = (c, r, site, float(d[r, site]), float(bnd), float(sd))
                if d[r, site] <= bnd:
                    ill.append(rec)
                    worst_ratio = max(worst_ratio, float(d[r, site] / bnd))
                    worst_z = max(worst_z, float(d[r, site] / sd))
                else:
                    unexplained.append(rec)
    return dict(worst_all=worst_all, unexplained=unexplained, cusp=cusp, ill=ill, events=events,
                step_now=step_now, frac_within_tol=n_ok / n_sites, n_sites=n_sites, worst_ratio=worst_ratio,
                worst_z=worst_z)


def parity_report(res) -> str:
    """One line of what a stepwise parity run excused and why."""
    return (f"worst {res['worst_all']:.3g}; within 1e-4: {res['frac_within_tol']:.6f} of {res['n_sites']} sites; "
            f"cusp events {len(res['events'])}, cusp-explained sites {len(res['cusp'])}; FP32-conditioned sites "
            f"{len(res['ill'])} (largest |dtheta| / first-order bound {res['worst_ratio']:.3g}, "
            f"/ rms of the same local errors {res['worst_z']:.3g}); unexplained {len(res['unexplained'])}")

def assert_grads_close(got, want, rel, what=""):
    """Every gradient component within `rel` of its own reference value
    (arrays of shape (n_cfg, 4): d/d(J_par, J_perp, h, eta))."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    err = np.abs(got - want)
    bad = err > rel * np.abs(want)
    assert not bad.any(), (f"{what}: components beyond {rel} relative at {np.argwhere(bad).tolist()}: "
                           f"got {got.tolist()}, want {want.tolist()}, relative {(err / np.abs(want)).tolist()}")
