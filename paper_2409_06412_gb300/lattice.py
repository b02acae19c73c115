"""Python view of a lattice object: torch tensors own the device memory and
the stream; every step of the method runs in the CUDA library."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L

PAPER_PARAMS = dict(J_par=10.0, J_perp=0.1, h=1.0, p=2.5, q=2.0, eta=1.0, dt=0.01, staggered_M=0)


@dataclass
class Config:
    """One configuration: n_replicas periodic Lx x Ly lattices sharing
    parameters and a temperature schedule: knots ((steps), (T)) of a
    piecewise-linear schedule, or {"power": (T_c, k_cross, tau_Q, gamma,
    eps_i, eps_f)} for the nonlinear quench of xy_set_power_quench."""
    Lx: int
    Ly: int
    n_replicas: int = 1
    seed: int = 1
    init_mode: int = L.XY_INIT_UNIFORM
    params: dict = field(default_factory=dict)
    knots: tuple = ((0,), (1.969,))
    n_total: int = 10**12
    cfg_id: int = -1      # configuration id in the noise counter (-1: position in the list)
    replica0: int = 0     # replica id of replica 0 in the noise counter
    field: tuple | None = None  # ((steps), (scales)): field schedule h_k = h s(k) (xy_set_field_schedule)
    # ((steps), (scales of J_par), (scales of J_perp)): coupling profiles of the
    # anisotropic quench, J_par a(k) and J_perp b(k) (xy_set_coupling_schedule)
    couplings: tuple | None = None

    @property
    def sites(self) -> int:
        return self.Lx * self.Ly * self.n_replicas


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


class Lattice:
    def __init__(self, configs, device="cuda", stream: torch.cuda.Stream | None = None,
                 theta: torch.Tensor | None = None, omega: torch.Tensor | None = None):
        self.configs = [c if isinstance(c, Config) else Config(**c) for c in configs]
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        total = sum(c.sites for c in self.configs)
        self.total_sites = total
        self.n_lattices = sum(c.n_replicas for c in self.configs)
        self.theta = theta if theta is not None else torch.zeros(total, dtype=torch.float32, device=self.device)
        self.omega = omega if omega is not None else torch.zeros(total, dtype=torch.float32, device=self.device)
        assert self.theta.numel() == total and self.omega.numel() == total
        assert self.theta.dtype == torch.float32 and self.theta.is_contiguous()
        descs = (L.ConfigDesc * len(self.configs))()
        for i, c in enumerate(self.configs):
            descs[i] = L.ConfigDesc(c.Lx, c.Ly, c.n_replicas, c.init_mode, c.seed, c.cfg_id, c.replica0)
        handle = ctypes.c_void_p()
        L.call("xy_lattice_create", descs, len(self.configs), _ptr(self.theta), _ptr(self.omega),
               ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
        self._h = handle
        # lattice index -> (config, replica) and site offsets
        self.b_cfg, self.offsets = [], []
        off = 0
        for ci, c in enumerate(self.configs):
            for r in range(c.n_replicas):
                self.b_cfg.append(ci)
                self.offsets.append(off)
                off += c.Lx * c.Ly
        for ci, c in enumerate(self.configs):
            self.set_params(ci, **c.params)
            if isinstance(c.knots, dict):
                self.set_power_quench(ci, *c.knots["power"], n_total=c.n_total)
            else:
                self.set_schedule(ci, c.knots[0], c.knots[1], c.n_total)
            if c.field is not None:
                self.set_field_schedule(ci, c.field[0], c.field[1])
            if c.couplings is not None:
                self.set_coupling_schedule(ci, *c.couplings)

    # ------------------------------------------------------------ setup
    def set_params(self, c: int, **kw):
        p = dict(PAPER_PARAMS)
        p.update({k: v for k, v in kw.items() if k != "staggered"})
        if "staggered" in kw:
            p["staggered_M"] = int(kw["staggered"])
        prm = L.Params(float(p["J_par"]), float(p["J_perp"]), float(p["h"]), float(p["p"]), float(p["q"]),
                       float(p["eta"]), float(p["dt"]), int(p["staggered_M"]), 0)
        L.call("xy_set_params", self._h, c, ctypes.byref(prm))

    def set_schedule(self, c: int, steps, temps, n_total: int):
        ks = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
        Ts = np.ascontiguousarray(np.asarray(temps, dtype=np.float64))
        L.call("xy_set_schedule", self._h, c, ks.ctypes.data_as(ctypes.c_void_p),
               Ts.ctypes.data_as(ctypes.c_void_p), int(ks.size), int(n_total))

    def set_power_quench(self, c: int, T_c: float, k_cross: int, tau_Q: float, gamma: float, eps_i: float,
                         eps_f: float, n_total: int):
        L.call("xy_set_power_quench", self._h, c, float(T_c), int(k_cross), float(tau_Q), float(gamma),
               float(eps_i), float(eps_f), int(n_total))

    def set_field_schedule(self, c: int, steps, scales):
        """Field of step k = h s(k), s piecewise linear through (steps, scales);
        empty lists remove the schedule."""
        ks = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
        ss = np.ascontiguousarray(np.asarray(scales, dtype=np.float64))
        L.call("xy_set_field_schedule", self._h, c, ks.ctypes.data_as(ctypes.c_void_p),
               ss.ctypes.data_as(ctypes.c_void_p), int(ks.size))

    def set_coupling_schedule(self, c: int, steps, par_scales, perp_scales):
        """Coupling profiles of the anisotropic quench: J_par(k) = J_par a(k),
        J_perp(k) = J_perp b(k), piecewise linear through the knots (empty:
        remove)."""
        ks = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
        a = np.ascontiguousarray(np.asarray(par_scales, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(perp_scales, dtype=np.float64))
        assert ks.shape == a.shape == b.shape and ks.ndim == 1
        L.call("xy_set_coupling_schedule", self._h, c, ks.ctypes.data_as(ctypes.c_void_p),
               a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p), int(ks.size))

    def set_path(self, path: int):
        L.call("xy_set_path", self._h, path)

    def autotune(self):
        L.call("xy_autotune", self._h)

    def set_autotune(self, on: bool):
        L.call("xy_set_autotune", self._h, int(bool(on)))

    # ------------------------------------------------------------ stepping
    def step(self, n: int, record_every: int = 0, t0: int = 0, rec: torch.Tensor | np.ndarray | None = None):
        """Advance n steps.  With record_every > 0 returns the records as a
        (B, R, 2) float64 tensor of (M, E) (device unless ``rec`` is given)."""
        if record_every > 0:
            R = n // record_every + 1
            if rec is None:
                rec = torch.full((self.n_lattices, R, 2), float("nan"), dtype=torch.float64, device=self.device)
            ptr = ctypes.c_void_p(rec.data_ptr() if isinstance(rec, torch.Tensor) else rec.ctypes.data)
        else:
            ptr = None
        L.call("xy_step_n", self._h, int(n), int(record_every), ptr, int(t0))
        return rec

    def observe(self):
        mom = np.zeros((len(self.configs), 6), dtype=np.float64)
        steps = np.zeros(len(self.configs), dtype=np.int64)
        L.call("xy_observe", self._h, mom.ctypes.data_as(ctypes.c_void_p), steps.ctypes.data_as(ctypes.c_void_p))
        return mom, steps

    def reset_moments(self):
        L.call("xy_reset_moments", self._h)

    def synchronize(self):
        L.call("xy_synchronize", self._h)

    def omega_full(self, b_first: int = 0, b_count: int | None = None) -> torch.Tensor:
        b_count = self.n_lattices - b_first if b_count is None else b_count
        n = sum(self.configs[self.b_cfg[b]].Lx * self.configs[self.b_cfg[b]].Ly
                for b in range(b_first, b_first + b_count))
        out = torch.empty(n, dtype=torch.float32, device=self.device)
        L.call("xy_omega_full", self._h, b_first, b_count, _ptr(out))
        return out

    def lattice_view(self, t: torch.Tensor, b: int) -> torch.Tensor:
        c = self.configs[self.b_cfg[b]]
        return t[self.offsets[b]:self.offsets[b] + c.Lx * c.Ly].view(c.Ly, c.Lx)

    def label_domains(self, b_first: int = 0, b_count: int | None = None, hist_cap: int = 4096):
        b_count = self.n_lattices - b_first if b_count is None else b_count
        c = self.configs[self.b_cfg[b_first]]
        N = c.Lx * c.Ly
        labels = torch.empty((b_count, N), dtype=torch.int32, device=self.device)
        hist = torch.empty((b_count, hist_cap, 2), dtype=torch.int64, device=self.device)
        n_sizes = torch.empty(b_count, dtype=torch.int64, device=self.device)
        L.call("xy_label_domains", self._h, b_first, b_count, _ptr(labels), _ptr(hist), hist_cap, _ptr(n_sizes))
        return labels, hist, n_sizes

    def structure_factor(self, b_first: int = 0, b_count: int | None = None, K: int = 16, rotor: float = 1.0):
        """S_par, S_perp of lattices [b_first, b_first + b_count) for k < K
        (App. C, Eq. S-as-lattice-FT): two (b_count, K) float64 device tensors."""
        b_count = self.n_lattices - b_first if b_count is None else b_count
        S_par = torch.empty((b_count, K), dtype=torch.float64, device=self.device)
        S_perp = torch.empty((b_count, K), dtype=torch.float64, device=self.device)
        L.call("xy_structure_factor", self._h, int(b_first), int(b_count), int(K), float(rotor), _ptr(S_par),
               _ptr(S_perp))
        return S_par, S_perp

    def set_temporal_blocking(self, kt: int):
        """0: the autotuner chooses one or two steps per launch per lattice
        shape; 1: one step per launch; 2: two steps wherever the shape allows."""
        L.call("xy_set_temporal_blocking", self._h, int(kt))

    def set_adjoint_mode(self, mode: int):
        """XY_ADJOINT_AUTO, XY_ADJOINT_RECOMPUTE or XY_ADJOINT_BACKWARD: how the
        reverse sweep gets the states of a checkpoint segment."""
        L.call("xy_set_adjoint_mode", self._h, int(mode))

    def adjoint(self, n: int, checkpoint_every: int = 100, w_E: float = 1.0, w_M: float = 0.0):
        obj = ctypes.c_double()
        grads = np.zeros((len(self.configs), 4), dtype=np.float64)
        L.call("xy_adjoint_step_n", self._h, int(n), int(checkpoint_every), float(w_E), float(w_M),
               ctypes.byref(obj), grads.ctypes.data_as(ctypes.c_void_p))
        return obj.value, grads

    def save(self) -> bytes:
        size = ctypes.c_size_t(0)
        L.call("xy_save", self._h, None, ctypes.byref(size))
        buf = ctypes.create_string_buffer(size.value)
        L.call("xy_save", self._h, buf, ctypes.byref(size))
        return buf.raw

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        L.call("xy_load", self._h, buf, len(blob))

    def set_kernel_timing(self, on: bool):
        L.call("xy_set_kernel_timing", self._h, int(bool(on)))

    def kernel_timing(self):
        """(ms, launches) per timing class (resident, strip, plain stepper launches;
        adjoint forward, recompute and reverse spans; two-step band launches;
        domain labelling spans) since timing was switched on."""
        ms = np.zeros(L.XY_KCLASS_COUNT, dtype=np.float64)
        n = np.zeros(L.XY_KCLASS_COUNT, dtype=np.int64)
        L.call("xy_kernel_timing", self._h, ms.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p))
        return ms, n

    def kernel_launches(self) -> int:
        return int(L.load().xy_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            L.load().xy_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_noise(seed, cfg, rep, k, tag, n_quads, device="cuda"):
    """Raw Philox words (n_quads, 4) uint32 (as int32 storage) and unit Gaussians (4 n_quads,)."""
    words = torch.empty((n_quads, 4), dtype=torch.int32, device=device)
    gauss = torch.empty(4 * n_quads, dtype=torch.float32, device=device)
    st = torch.cuda.current_stream(device)
    L.call("xy_debug_noise", int(seed), int(cfg), int(rep), int(k), int(tag), int(n_quads), _ptr(words),
           _ptr(gauss), ctypes.c_void_p(st.cuda_stream))
    return words, gauss


def debug_philox(counters: torch.Tensor, key0: int, key1: int) -> torch.Tensor:
    out = torch.empty_like(counters)
    st = torch.cuda.current_stream(counters.device)
    L.call("xy_debug_philox", _ptr(counters), int(key0), int(key1), int(counters.shape[0]), _ptr(out),
           ctypes.c_void_p(st.cuda_stream))
    return out
