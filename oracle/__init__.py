"""FP64 CPU oracle of the Si(001) dimer-angle Langevin dynamics (arXiv 2409.06412).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library under ``paper_2409_06412_gb300`` never does, and this
package imports nothing from it: the two share no code.

The arithmetic lives in ``xy_oracle.c`` (plain C, doubles, one loop per
equation of the paper); this module compiles it with gcc and marshals numpy
arrays through ctypes.  Multi-lattice runs are spread over host threads with
one lattice per call (ctypes releases the GIL), which changes no arithmetic.

Parameter vector order: (J_par, J_perp, h, p, q, eta, dt, staggered).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xy_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libxy_oracle.so")
_lib = None
_lock = threading.Lock()

PARAM_NAMES = ("J_par", "J_perp", "h", "p", "q", "eta", "dt", "staggered")
PAPER_PARAMS = dict(J_par=10.0, J_perp=0.1, h=1.0, p=2.5, q=2.0, eta=1.0, dt=0.01, staggered=0.0)
T_C = 0.1969 * 10.0  # Fig. 4 caption: (beta_c J_par)^-1 = 0.1969 at J_par = 10


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libxy_oracle.so`` (gcc, -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    P = ctypes.POINTER
    d, i32, i64, u64, u32 = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
    vp = ctypes.c_void_p
    L.xyo_philox_batch.argtypes = [i64, vp, vp, vp]
    L.xyo_gauss_batch.argtypes = [u64, i32, i32, i64, i64, i32, vp]
    L.xyo_wrap_batch.argtypes = [i64, vp, vp]
    L.xyo_uniform.argtypes = [u32]
    L.xyo_uniform.restype = d
    L.xyo_temperature.argtypes = [i64, i32, vp, vp]
    L.xyo_temperature.restype = d
    L.xyo_init_theta.argtypes = [i32, i32, i32, i32, u64, i32, vp]
    L.xyo_force.argtypes = [i32, i32, vp, vp, vp]
    L.xyo_observe.argtypes = [i32, i32, vp, vp, vp, P(d), P(d)]
    L.xyo_field_scale.argtypes = [i64, i32, vp, vp]
    L.xyo_field_scale.restype = d
    L.xyo_run_lattice.argtypes = [i32, i32, i32, i32, u64, vp, i32, vp, vp, vp, i64, i64, vp, vp, i32, vp]
    L.xyo_run_lattice.restype = i64
    L.xyo_run_strip.argtypes = [i32, i32, i32, i32, i32, i32, u64, vp, i32, vp, vp, vp, i64, i64,
                                vp, vp, vp, i32, i32, i32, vp]
    L.xyo_run_strip.restype = i64
    L.xyo_harmonic_msd.argtypes = [i64, i64, d, d, d, d, u64, vp]
    L.xyo_ccl.argtypes = [i32, i32, vp, vp]
    L.xyo_ccl.restype = i64
    L.xyo_adjoint_lattice.argtypes = [i32, i32, i32, i32, u64, vp, i32, vp, vp, vp, i64, i64, vp, vp,
                                      d, d, P(d), vp, vp, vp]
    L.xyo_theta_sensitivity.argtypes = [i32, i32, i32, i32, u64, vp, i32, vp, vp, vp, i64, i64, vp, vp,
                                        i32, vp, vp, vp, vp, vp, vp, vp, vp]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def param_vector(params: dict) -> np.ndarray:
    full = dict(PAPER_PARAMS)
    full.update(params or {})
    return np.array([float(full[k]) for k in PARAM_NAMES], dtype=np.float64)


def _knots(knots):
    """Schedule arguments of the C oracle as (n_knots, steps, values): knots
    ((steps), (T)) for the piecewise-linear schedule, or {"power": (T_c,
    k_cross, tau_Q, gamma, eps_i, eps_f)} for the nonlinear quench, which the C
    side takes as n_knots = -1 (see xyo_temperature)."""
    if isinstance(knots, dict):
        Ts = np.ascontiguousarray(np.asarray(knots["power"], dtype=np.float64))
        assert Ts.shape == (6,)
        return -1, np.zeros(1, dtype=np.int64), Ts
    ks = np.ascontiguousarray(np.asarray(knots[0], dtype=np.int64))
    Ts = np.ascontiguousarray(np.asarray(knots[1], dtype=np.float64))
    assert ks.shape == Ts.shape and ks.ndim == 1 and ks.size >= 1
    return ks.size, ks, Ts


def _field(field):
    """A profile of the C oracle as (n, steps, scales): ((steps), (scales)),
    or None for a constant 1."""
    if field is None:
        return 0, np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.float64)
    ks = np.ascontiguousarray(np.asarray(field[0], dtype=np.int64))
    ss = np.ascontiguousarray(np.asarray(field[1], dtype=np.float64))
    assert ks.shape == ss.shape and ks.ndim == 1
    return ks.size, ks, ss


class _Sched(ctypes.Structure):
    """xyo_sched: the field profile s(k) of h and the coupling profiles a(k),
    b(k) of J_par and J_perp (one knot grid for both)."""
    _fields_ = [("nf", ctypes.c_int), ("fks", ctypes.c_void_p), ("fss", ctypes.c_void_p),
                ("nc", ctypes.c_int), ("cks", ctypes.c_void_p), ("cpar", ctypes.c_void_p),
                ("cperp", ctypes.c_void_p)]


def _sched(field=None, couplings=None):
    """(struct, arrays it points into): field ((steps), (scales)) of h;
    couplings ((steps), (scales of J_par), (scales of J_perp))."""
    nf, fks, fss = _field(field)
    if couplings is None:
        nc, cks, ca, cb = 0, np.zeros(1, np.int64), np.zeros(1), np.zeros(1)
    else:
        cks = np.ascontiguousarray(np.asarray(couplings[0], dtype=np.int64))
        ca = np.ascontiguousarray(np.asarray(couplings[1], dtype=np.float64))
        cb = np.ascontiguousarray(np.asarray(couplings[2], dtype=np.float64))
        assert cks.shape == ca.shape == cb.shape and cks.ndim == 1
        nc = cks.size
    keep = (fks, fss, cks, ca, cb)
    st = _Sched(nf, fks.ctypes.data, fss.ctypes.data, nc, cks.ctypes.data, ca.ctypes.data, cb.ctypes.data)
    return st, keep


# ---------------------------------------------------------------- primitives

def philox(ctrs: np.ndarray, key) -> np.ndarray:
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctrs)
    lib().xyo_philox_batch(ctrs.shape[0], _ptr(ctrs), _ptr(k), _ptr(out))
    return out


def uniform(words: np.ndarray) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint32)
    return np.array([lib().xyo_uniform(int(w)) for w in words.ravel()]).reshape(words.shape)


def gauss(seed: int, cfg: int, rep: int, n_sites: int, k: int, tag: int = 0) -> np.ndarray:
    out = np.empty(n_sites, dtype=np.float64)
    lib().xyo_gauss_batch(seed, cfg, rep, n_sites, k, tag, _ptr(out))
    return out


def wrap(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    lib().xyo_wrap_batch(x.size, _ptr(x), _ptr(out))
    return out


def temperature(k: int, knots) -> float:
    nk, ks, Ts = _knots(knots)
    return lib().xyo_temperature(k, nk, _ptr(ks), _ptr(Ts))


def field_scale(k: int, field) -> float:
    nf, fks, fss = _field(field)
    return lib().xyo_field_scale(k, nf, _ptr(fks), _ptr(fss))


def init_theta(Lx, Ly, cfg, rep, seed, mode) -> np.ndarray:
    th = np.zeros(Lx * Ly, dtype=np.float64)
    lib().xyo_init_theta(Lx, Ly, cfg, rep, seed, mode, _ptr(th))
    return th


def force(Lx, Ly, params, theta) -> np.ndarray:
    prm = param_vector(params)
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    F = np.empty_like(th)
    lib().xyo_force(Lx, Ly, _ptr(prm), _ptr(th), _ptr(F))
    return F


def observe(Lx, Ly, params, theta, omega):
    prm = param_vector(params)
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    om = np.ascontiguousarray(omega, dtype=np.float64).ravel()
    M, E = ctypes.c_double(), ctypes.c_double()
    lib().xyo_observe(Lx, Ly, _ptr(prm), _ptr(th), _ptr(om), ctypes.byref(M), ctypes.byref(E))
    return M.value, E.value


def run_lattice(Lx, Ly, cfg, rep, seed, params, knots, k0, n, theta, omega, record_every=0, field=None,
                couplings=None):
    """Advance one lattice in place; returns the (n_rec, 2) array of (M_k, E_k)."""
    prm = param_vector(params)
    nk, ks, Ts = _knots(knots)
    sc, _keep = _sched(field, couplings)
    assert theta.dtype == np.float64 and omega.dtype == np.float64
    assert theta.flags.c_contiguous and omega.flags.c_contiguous
    nrec_max = (n // record_every + 1) if record_every > 0 else 0
    rec = np.zeros((max(nrec_max, 1), 2), dtype=np.float64)
    nrec = lib().xyo_run_lattice(Lx, Ly, cfg, rep, seed, _ptr(prm), nk, _ptr(ks), _ptr(Ts), ctypes.byref(sc),
                                 k0, n, _ptr(theta), _ptr(omega), record_every, _ptr(rec))
    return rec[:nrec].copy()


def run_strip(Lx, Ly, y0, cfg, rep, seed, params, knots, k0, n, theta, omega, F, rows=None, record_every=0,
              field=None, couplings=None):
    """Advance one row strip of an Lx x Ly lattice in place (see
    xyo_run_strip): theta, omega, F are (R, Lx) float64 buffers whose local
    row i is global row (y0 + i) mod Ly, F holding F(theta) on entry.  Rows
    that lose a neighbour become NaN, one per step at either end.  With
    ``record_every``, returns the (n_rec, 2) raw sums over the local rows
    ``rows`` = (r0, r1) of sigma sin(q theta) and of the site energy."""
    prm = param_vector(params)
    nk, ks, Ts = _knots(knots)
    sc, _keep = _sched(field, couplings)
    for a in (theta, omega, F):
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == theta.shape
    R = theta.shape[0]
    assert theta.size == R * Lx
    r0, r1 = (0, 0) if rows is None else rows
    nrec_max = (n // record_every + 1) if record_every > 0 else 0
    rec = np.zeros((max(nrec_max, 1), 2), dtype=np.float64)
    nrec = lib().xyo_run_strip(Lx, Ly, y0, R, cfg, rep, seed, _ptr(prm), nk, _ptr(ks), _ptr(Ts), ctypes.byref(sc),
                               k0, n, _ptr(theta), _ptr(omega), _ptr(F), r0, r1, record_every, _ptr(rec))
    return rec[:nrec].copy()


def harmonic_msd(n_paths, n_steps, dt, eta, T, w2, seed=1) -> np.ndarray:
    out = np.empty(n_steps + 1, dtype=np.float64)
    lib().xyo_harmonic_msd(n_paths, n_steps, dt, eta, T, w2, seed, _ptr(out))
    return out


def ccl(Lx, Ly, theta32) -> tuple[np.ndarray, np.ndarray]:
    """Labels (int32, min site index per component) and the sparse size
    histogram as an (n_sizes, 2) int64 array of (size, count), ascending."""
    th = np.ascontiguousarray(theta32, dtype=np.float32).ravel()
    lab = np.empty(Lx * Ly, dtype=np.int32)
    lib().xyo_ccl(Lx, Ly, _ptr(th), _ptr(lab))
    _, sizes = np.unique(lab, return_counts=True)
    vals, counts = np.unique(sizes, return_counts=True)
    hist = np.stack([vals.astype(np.int64), counts.astype(np.int64)], axis=1) if vals.size else np.zeros((0, 2), np.int64)
    return lab, hist


def adjoint_lattice(Lx, Ly, cfg, rep, seed, params, knots, k0, n, theta0, omega0, wE, wM, field=None,
                    couplings=None):
    """Objective sum_{k=k0+1}^{k0+n}(w_E E_k + w_M |M_k|) of one lattice, its
    gradient w.r.t. (J_par, J_perp, h, eta), and the final state."""
    prm = param_vector(params)
    nk, ks, Ts = _knots(knots)
    sc, _keep = _sched(field, couplings)
    th0 = np.ascontiguousarray(theta0, dtype=np.float64).ravel()
    om0 = np.ascontiguousarray(omega0, dtype=np.float64).ravel()
    grad = np.zeros(4, dtype=np.float64)
    obj = ctypes.c_double()
    th1 = np.empty_like(th0)
    om1 = np.empty_like(om0)
    lib().xyo_adjoint_lattice(Lx, Ly, cfg, rep, seed, _ptr(prm), nk, _ptr(ks), _ptr(Ts), ctypes.byref(sc), k0, n,
                              _ptr(th0), _ptr(om0), wE, wM, ctypes.byref(obj), _ptr(grad),
                              _ptr(th1), _ptr(om1))
    return obj.value, grad, th1, om1


def theta_sensitivity(Lx, Ly, cfg, rep, seed, params, knots, k0, n, theta0, omega0, targets, wt=None, wv=None,
                      trajectory=False, fields=False, field=None, couplings=None):
    """First-order sensitivity of the final angles theta_t(k0 + n), t in
    ``targets``, to perturbations along the FP64 trajectory from the full-step
    state (theta0, omega0) (see xyo_theta_sensitivity): an (n_targets, 2)
    array of [sum |l| w, sqrt(sum l^2 w^2)] over the angles (weights wt, shape
    (n, N): steps 1..n) and the half-step velocities (weights wv, shape
    (n, N): steps 0..n-1); weights default to 1.  With ``trajectory``, also
    the (n + 1, N) arrays theta_j, omega_j; with ``fields``, also the (n, N)
    fields lt, lv of the first target."""
    prm = param_vector(params)
    nk, ks, Ts = _knots(knots)
    sc, _keep = _sched(field, couplings)
    th0 = np.ascontiguousarray(theta0, dtype=np.float64).ravel()
    om0 = np.ascontiguousarray(omega0, dtype=np.float64).ravel()
    tg = np.ascontiguousarray(np.asarray(targets, dtype=np.int64).ravel())
    N = Lx * Ly
    out = np.zeros((tg.size, 2), dtype=np.float64)
    w_t = None if wt is None else np.ascontiguousarray(wt, dtype=np.float64).reshape(n, N)
    w_v = None if wv is None else np.ascontiguousarray(wv, dtype=np.float64).reshape(n, N)
    tth = np.zeros((n + 1, N)) if trajectory else None
    tom = np.zeros((n + 1, N)) if trajectory else None
    lt = np.zeros((n, N)) if fields else None
    lv = np.zeros((n, N)) if fields else None
    p = lambda a: None if a is None else _ptr(a)
    lib().xyo_theta_sensitivity(Lx, Ly, cfg, rep, seed, _ptr(prm), nk, _ptr(ks), _ptr(Ts), ctypes.byref(sc),
                                k0, n, _ptr(th0), _ptr(om0),
                                int(tg.size), _ptr(tg), p(w_t), p(w_v), _ptr(out), p(tth), p(tom), p(lt), p(lv))
    res = (out,)
    if trajectory:
        res += (tth, tom)
    if fields:
        res += (lt, lv)
    return res if len(res) > 1 else out


# ---------------------------------------------------------------- batches

def _workers():
    return max(1, os.cpu_count() or 1)


def run_batch(configs, thetas, omegas, step_now, n, record_every=0, t0=0, threads=None):
    """Advance a batch of lattices described like the library's configurations.

    configs: list of dicts with keys Lx, Ly, n_rep, seed, params, knots, n_total
    (and optionally field: ((steps), (scales)) of h_k = h s(k); couplings:
    ((steps), (scales of J_par), (scales of J_perp))).
    thetas/omegas: per config, float64 arrays (n_rep, Ly*Lx) updated in place
    (omega is the full-step angular velocity).  step_now: per config step
    counters (list, updated).  Returns (rec, moments) with rec[c] of shape
    (n_rep, n_rec_c, 2) and moments (n_cfg, 6) = sums over replicas and records
    at steps >= t0 of (1, M^2, M^4, E, E^2, |M|).
    """
    jobs = []
    n_eff = []
    for c, cf in enumerate(configs):
        k0 = int(step_now[c])
        ne = max(0, min(int(n), int(cf["n_total"]) - k0))
        n_eff.append(ne)
        for r in range(cf["n_rep"]):
            jobs.append((c, r, k0, ne))

    def work(job):
        c, r, k0, ne = job
        cf = configs[c]
        return run_lattice(cf["Lx"], cf["Ly"], c, r, cf["seed"], cf["params"], cf["knots"], k0, ne,
                           thetas[c][r], omegas[c][r], record_every, cf.get("field"), cf.get("couplings"))

    with ThreadPoolExecutor(max_workers=threads or _workers()) as ex:
        results = list(ex.map(work, jobs))

    recs, moments = [], np.zeros((len(configs), 6), dtype=np.float64)
    it = iter(results)
    for c, cf in enumerate(configs):
        k0 = int(step_now[c])
        per = [next(it) for _ in range(cf["n_rep"])]
        nr = per[0].shape[0] if per else 0
        recs.append(np.stack(per) if per else np.zeros((0, 0, 2)))
        if record_every > 0 and nr > 0:
            first = -(-k0 // record_every) * record_every
            ks = first + record_every * np.arange(nr)
            for r in range(cf["n_rep"]):
                for j in range(nr):
                    if ks[j] >= t0:
                        M, E = per[r][j]
                        moments[c] += (1.0, M * M, M ** 4, E, E * E, abs(M))
        step_now[c] = k0 + n_eff[c]
    return recs, moments
