#!/usr/bin/env python
"""Benchmark of the BBK Langevin stepper on the static-criticality workload.

Workload (one bench "step" = one sampling interval ds = 100 dt of App. B:
100 BBK time steps of the whole batch, then one observable record per lattice
and FP64 moment accumulation):
  L in {128, 256, 512, 1024} periodic lattices, 32 temperatures uniform in
  [0.9, 1.1] T_c, 16 replicas each (2048 lattices, 7.13e8 sites), ordered
  start, J_par = 10, J_perp = 0.1, h = 1, p = 2.5, q = 2, eta = 1, dt = 0.01.
Metric: site-updates per second (whole job), with the HBM roofline of the
dominant kernel, the plain per-configuration launch path, the adjoint/forward
cost on the differentiation workload (L = 256 x 64 replicas, 2000 steps,
checkpoint every 100), domain labelling throughput and the FP64 CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own copy of the batch (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TC = 1.969
LS_FULL = (128, 256, 512, 1024)
LS = LS_FULL
N_TEMPS, N_REP = 32, 16
INNER = 100           # BBK steps per bench step: one sampling interval ds = 100 dt, then one record
CPU_ROUND = 10        # BBK steps per round of the oracle's bounded sample
REF_INNER = 4         # BBK steps per step of the reference arm (the oracle on the host cores)
N_TOTAL = 10 ** 5     # run length of every configuration
T0 = N_TOTAL // 5     # moments discard the first fifth
METRIC = "site-updates/s/GPU and % HBM roofline, batched vs plain; adjoint/forward cost"
WORKLOAD = "static criticality: L in {128,256,512,1024}, 32 T in [0.9,1.1] T_c, 16 replicas, ordered start"
BYTES_PER_SU = 16.0   # theta and omega (FP32) read and written once per site-update


def temps():
    return [TC * (0.9 + 0.2 * i / (N_TEMPS - 1)) for i in range(N_TEMPS)]


KZ = False
DYNZ = False
REC_EVERY = INNER     # record interval of the timed steps


def set_workload(name):
    """'static' (the full batch), 'static-L512' (its L = 512 part only: 512
    lattices, 1.3e8 sites, 1 GB of state, for profiler captures) or
    'dynamic-z' (L up to 2048 x 256 replicas, a record every 10 steps) or
    'kibble-zurek' (the 9216-lattice quench batch, 155 GB on the device; with
    --warmup 10 the timed steps pass k = 1150, where the tau_Q = 100 ramps end
    and those lattices retire)."""
    global LS, WORKLOAD, KZ, DYNZ, REC_EVERY
    if name == "static-L512":
        LS = (512,)
        WORKLOAD = "static criticality, L = 512 part: 32 T in [0.9,1.1] T_c, 16 replicas, ordered start"
    elif name == "dynamic-z":
        DYNZ = True
        REC_EVERY = 10
        WORKLOAD = ("dynamic exponent z: L in {256, 512, 1024, 2048} x 256 replicas, ordered start at T_c, "
                    "M and E recorded every 10 steps")
    elif name == "kibble-zurek":
        KZ = True
        WORKLOAD = ("Kibble-Zurek: L = 1024, 16 log-spaced tau_Q in [1e2, 1e5] x eta {0.1, 1, 10} x "
                    "h {0.5, 1, 2} x 64 replicas (9216 lattices); 1e3 steps at 1.5 T_c, then a linear ramp "
                    "to 0 over 1.5 tau_Q; uniform random start")
    else:
        LS = LS_FULL


def static_configs(seed):
    from paper_2409_06412_gb300 import XY_INIT_ORDERED, Config
    return [Config(Lx=L, Ly=L, n_replicas=N_REP, seed=seed, init_mode=XY_INIT_ORDERED, knots=((0,), (T,)),
                   n_total=N_TOTAL) for L in LS for T in temps()]


def kz_configs(seed):
    import numpy as np

    from paper_2409_06412_gb300 import XY_INIT_UNIFORM, Config
    out = []
    for tq in np.round(np.logspace(2, 5, 16)).astype(int):
        ramp = int(round(1.5 * tq))
        for eta in (0.1, 1.0, 10.0):
            for h in (0.5, 1.0, 2.0):
                out.append(Config(Lx=1024, Ly=1024, n_replicas=64, seed=seed, init_mode=XY_INIT_UNIFORM,
                                  params=dict(eta=eta, h=h), knots=((0, 1000, 1000 + ramp), (1.5 * TC, 1.5 * TC, 0.0)),
                                  n_total=1000 + ramp))
    return out


def dynz_configs(seed):
    from paper_2409_06412_gb300 import XY_INIT_ORDERED, Config
    return [Config(Lx=L, Ly=L, n_replicas=256, seed=seed, init_mode=XY_INIT_ORDERED, knots=((0,), (TC,)),
                   n_total=N_TOTAL) for L in (256, 512, 1024, 2048)]


def workload_configs(seed):
    if KZ:
        return kz_configs(seed)
    return dynz_configs(seed) if DYNZ else static_configs(seed)


# ------------------------------------------------------------------ clocks

CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        text = open(self.f.name).read()
        os.unlink(self.f.name)
        return parse_clock_samples(text)


def parse_clock_samples(text):
    """Summary of `nvidia-smi --query-gpu=<CLOCK_Q> --format=csv,noheader,nounits`
    rows: median and maximum SM clock and the throttle reasons seen Active in
    any sample (malformed rows are skipped)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        if not line.strip():
            continue
        r = [x.strip() for x in line.split(",")]
        try:
            sm.append(float(r[1]))
            mx.append(float(r[2]))
        except (ValueError, IndexError):
            continue
        for i, nm in enumerate(names):
            if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel):
    """Per-site DRAM bytes of `kernel` from the committed ncu summary, if the
    summary was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = open(os.path.join(ROOT, "paper_2409_06412_gb300", "csrc", "xy_step.cu"), "rb").read()
    src += open(os.path.join(ROOT, "paper_2409_06412_gb300", "csrc", "xy_device.cuh"), "rb").read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("source") == digest:
            return float(f["dram_bytes_per_site"])
    return None


def time_labels(lat, b0, n, calls=5):
    """Seconds per domain-labelling call of lattices [b0, b0 + n) (the
    library call through its Python binding, outputs on the device), median
    of `calls` after two warm-up calls that also size the working memory;
    and the device time of its passes per call (CUDA events on the object's
    stream from the first pass to the last, the library's labelling timing
    class, over the same calls)."""
    import torch

    from paper_2409_06412_gb300._lib import XY_KCLASS_LABELS
    for _ in range(2):
        lat.label_domains(b0, n)
    lat.set_kernel_timing(True)
    ts = []
    for _ in range(calls):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, n_sizes = lat.label_domains(b0, n)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    ms, nl = lat.kernel_timing()
    lat.set_kernel_timing(False)
    return sorted(ts)[len(ts) // 2], n_sizes, ms[XY_KCLASS_LABELS] / 1e3 / max(1, nl[XY_KCLASS_LABELS])


def cuda_time(fn, stream):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def oracle_sample(workers):
    """A bounded sample of the workload for the FP64 oracle: per host thread,
    one lattice of each L (the workload's equal lattice counts per L), ordered
    state at T_c, distinct (configuration, replica) noise ids.  Tasks run
    largest first on `workers` threads, so every thread gets one lattice of
    each size and the threads stay evenly loaded."""
    import numpy as np

    import oracle
    oracle.build()
    tasks = []
    for i, L in reversed(list(enumerate(LS))):
        for w in range(workers):
            c, r = 32 * i + w % 32, (w // 32) % N_REP
            th = oracle.init_theta(L, L, c, r, 1, 1)
            tasks.append([L, c, r, th, np.zeros_like(th), 0])
    return tasks


def oracle_round(ex, tasks, n):
    """n BBK steps of every sampled lattice; returns the site-updates done."""
    import oracle

    def run(t):
        L, c, r, th, om, k = t
        oracle.run_lattice(L, L, c, r, 1, {}, ([0], [TC]), k, n, th, om)
        t[5] += n
        return L * L * n

    return sum(ex.map(run, tasks))


def cpu_baseline(budget_s=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload
    (oracle_sample), 10-step rounds until the budget is spent."""
    from concurrent.futures import ThreadPoolExecutor
    workers = os.cpu_count() or 1
    tasks = oracle_sample(workers)
    su, rounds = 0, 0
    with ThreadPoolExecutor(max_workers=workers) as ex:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            su += oracle_round(ex, tasks, CPU_ROUND)
            rounds += 1
        dt = time.perf_counter() - t0
    return {"value": su / dt, "unit": "site-updates/s", "cores": workers, "kind": "oracle",
            "sample": f"{workers} lattices per L in {list(LS)} at T_c (one of each per host thread), "
                      f"{rounds * CPU_ROUND} steps each ({su:.3g} site-updates, {dt:.1f} s)"}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2409_06412_gb300 import XY_ADJOINT_RECOMPUTE, XY_PATH_BATCHED, XY_PATH_PLAIN, Config, Lattice, build
    from paper_2409_06412_gb300 import _lib as LL

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    cfgs = workload_configs(seed=1 + rank)
    lat = Lattice(cfgs, stream=stream)
    S = sum(c.sites for c in cfgs)
    R = INNER // REC_EVERY + 1

    def done_su(before, after):
        """Site-updates between two step-counter readings (lattices that
        retire mid-window count their own steps only), split by stepper:
        (lattices with L >= 256: strip; the rest: cluster-resident)."""
        strip = sum(c.sites * int(a - b) for c, a, b in zip(cfgs, after, before) if c.Lx >= 256)
        res = sum(c.sites * int(a - b) for c, a, b in zip(cfgs, after, before) if c.Lx < 256)
        return strip, res

    def bench_step():
        lat.step(INNER, record_every=REC_EVERY, t0=T0)

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    steps0 = lat.observe()[1]
    clocks = ClockSampler(local)
    l0 = lat.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        bench_step()
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = lat.kernel_launches() - l0
    if world > 1:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    mom, steps = lat.observe()
    su_timed = sum(done_su(steps0, steps))
    su_step = su_timed / args.steps
    value = world * su_timed / elapsed

    extra = {}
    if rank == 0:
        # dominant kernel, timed live with events on its stream (the strip
        # stepper carries every lattice with L >= 256)
        s_before = lat.observe()[1]
        lat.set_kernel_timing(True)
        for _ in range(3):
            bench_step()
        ms, nl = lat.kernel_timing()
        lat.set_kernel_timing(False)
        su_strip, su_res = done_su(s_before, lat.observe()[1])
        hbm, peak_kind = peaks()
        # the strip stepper runs one launch per lattice shape per BBK step:
        # the site-updates it did (from the step counters) and its summed
        # launch time give bytes per launch over the average launch duration
        n_bbk = 3 * INNER
        strip_s = ms[1] / 1e3 / n_bbk                      # strip time per BBK step
        n_launch = max(1, int(nl[1]))
        achieved = BYTES_PER_SU * su_strip / (ms[1] / 1e3) / 1e9
        traffic = ncu_traffic("strip_step_kernel")
        extra["roofline"] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                             "frac": round(achieved / hbm, 4), "peak_kind": f"{peak_kind} copy bandwidth",
                             "kernel": "strip_step_kernel",
                             "traffic": (round(traffic * su_strip / n_launch) if traffic else None),
                             "algorithmic_bytes_per_launch": int(BYTES_PER_SU * su_strip / n_launch),
                             "launch_ms": round(ms[1] / n_launch, 4),
                             "launches_per_bbk_step": max(1, round(nl[1] / n_bbk))}
        # The event-timed launches run one after another on the library's
        # stream; in the captured graphs of the timed region the lattice
        # shapes' slices run concurrently, so a whole BBK step there takes less
        # than the serial launches add up to.  Both are reported: frac is the
        # kernel's own (serial launches), step_frac the whole step's at 16 B/su.
        graph_ms_bbk = elapsed / (args.steps * INNER) * 1e3
        extra["roofline"]["serial_ms_per_bbk_step"] = round((ms[0] + ms[1]) / n_bbk, 4)
        extra["roofline"]["graph_ms_per_bbk_step"] = round(graph_ms_bbk, 4)
        extra["roofline"]["step_frac"] = round(value / world * BYTES_PER_SU / 1e9 / hbm, 4)
        extra["roofline"]["gap"] = ("serial_ms_per_bbk_step exceeds graph_ms_per_bbk_step because the graphs run the "
                                    "lattice shapes' slices concurrently, the timing mode one launch at a time")
        extra["kernel_ms_per_bbk_step"] = {"resident": round(ms[0] / n_bbk, 4), "strip": round(strip_s * 1e3, 4)}
        extra["resident_su_per_s"] = su_res / (ms[0] / 1e3) if nl[0] else None

    if args.workload == "static":
        # end to end through the public API with host buffers: each step loads
        # its input state from pinned host memory (xy_load), advances INNER BBK
        # steps and returns its records to pinned host memory.  Serial: one
        # lattice object, upload then stepping.  Double-buffered (the value
        # reported): two lattice objects on two streams take the steps in
        # turn, so one step's upload overlaps the other object's stepping, as a
        # caller streaming batches would run it; every step's copies lie inside
        # the timed region.
        blob = lat.save()
        pinned = torch.empty(len(blob), dtype=torch.uint8).pin_memory()
        pinned.numpy()[:] = np.frombuffer(blob, dtype=np.uint8)
        lib = LL.load()
        import ctypes

        def load(lt):
            LL.check(lib.xy_load(lt._h, ctypes.c_void_p(pinned.data_ptr()), len(blob)), "xy_load")

        rec_host = [torch.empty((lat.n_lattices, R, 2), dtype=torch.float64).pin_memory() for _ in range(2)]

        def e2e_step():
            load(lat)
            lat.step(INNER, record_every=INNER, t0=T0, rec=rec_host[0])

        e2e_step()
        n_e2e = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        te_serial = time.perf_counter() - t0
        # where a serial step's time goes: the upload (xy_load, synchronous)
        # and the stepping with the records' read-back, each host-timed
        t_load, t_adv = [], []
        for _ in range(2):
            torch.cuda.synchronize()
            ta = time.perf_counter()
            load(lat)
            tb = time.perf_counter()
            lat.step(INNER, record_every=INNER, t0=T0, rec=rec_host[0])
            torch.cuda.synchronize()
            t_load.append(tb - ta)
            t_adv.append(time.perf_counter() - tb)

        s2 = torch.cuda.Stream()
        lat2 = Lattice(static_configs(seed=1 + rank), stream=s2)
        pair = [(lat, stream), (lat2, s2)]
        rec_dev = [torch.empty((lat.n_lattices, R, 2), dtype=torch.float64, device="cuda") for _ in range(2)]

        def e2e_pipelined(n):
            load(pair[0][0])
            for j in range(n):
                lt, st = pair[j % 2]
                lt.step(INNER, record_every=INNER, t0=T0, rec=rec_dev[j % 2])
                with torch.cuda.stream(st):
                    rec_host[j % 2].copy_(rec_dev[j % 2], non_blocking=True)
                if j + 1 < n:
                    load(pair[(j + 1) % 2][0])  # the next step's input, while this one steps
                st.synchronize()  # this step's records are on the host

        e2e_pipelined(2)
        torch.cuda.synchronize()
        n_pipe = max(4, min(args.steps, 10))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_pipelined(n_pipe)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        if world > 1:  # whole job: every rank's steps over the slowest rank's time
            tt = torch.tensor([te, te_serial], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te, te_serial = float(tt[0]), float(tt[1])
        extra["e2e"] = {"value": world * n_pipe * su_step / te, "unit": "site-updates/s",
                        "h2d_bytes_per_step": len(blob), "d2h_bytes_per_step": int(rec_host[0].numel() * 8),
                        "mode": "double-buffered: two lattice objects, each step's upload overlaps the other's stepping",
                        "serial_value": world * n_e2e * su_step / te_serial,
                        "serial_upload_ms": round(min(t_load) * 1e3, 2), "serial_step_ms": round(min(t_adv) * 1e3, 2)}
        lat2.close()
        del lat2, rec_dev

    if rank == 0 and KZ:
        # domain labels of the frozen state of the tau_Q = 100 ramps (the
        # first 64 lattices, retired at k = 1150 when the window passes it)
        tl, n_sizes, td = time_labels(lat, 0, 64)
        extra["ccl"] = {"value": 64 * 1024 * 1024 / tl, "unit": "labelled sites/s", "lattices": 64, "L": 1024,
                        "step": int(lat.observe()[1][0]), "distinct_domain_sizes_max": int(n_sizes.max()),
                        "timing": "median of 5 calls after 2 warm-up calls, host clock around the synchronised call",
                        "device_value": 64 * 1024 * 1024 / td,
                        "device_timing": "CUDA events around the passes of each call, mean over the same 5 calls"}

    if rank == 0 and args.workload == "static":
        # plain per-configuration launch path on the same batch
        lat.set_path(XY_PATH_PLAIN)
        bench_step()
        n_plain = 2
        tp = cuda_time(lambda: [bench_step() for _ in range(n_plain)], stream)
        lat.set_path(XY_PATH_BATCHED)
        plain = n_plain * su_step / tp
        extra["plain"] = {"value": plain, "unit": "site-updates/s", "batched_over_plain": value / world / plain}

        # domain labelling throughput on the 512 L = 1024 lattices (first 64)
        b0 = 3 * N_TEMPS * N_REP
        tl, n_sizes, td = time_labels(lat, b0, 64)
        extra["ccl"] = {"value": 64 * 1024 * 1024 / tl, "unit": "labelled sites/s", "lattices": 64, "L": 1024,
                        "distinct_domain_sizes_max": int(n_sizes.max()),
                        "timing": "median of 5 calls after 2 warm-up calls, host clock around the synchronised call",
                        "device_value": 64 * 1024 * 1024 / td,
                        "device_timing": "CUDA events around the passes of each call, mean over the same 5 calls"}

        # correlation lengths of the same 64 lattices: structure factors for k < 16 (timed), then over
        # the half zone for the fit, whose window follows each direction's length (xi_perp is below a
        # site here: J_perp = J_par / 100)
        from paper_2409_06412_gb300 import corrlen
        lat.structure_factor(b0, 64, 16)
        t_sf = cuda_time(lambda: lat.structure_factor(b0, 64, 16), stream)
        K_fit = 512
        t_sf_fit = cuda_time(lambda: lat.structure_factor(b0, 64, K_fit), stream)
        s_par, s_perp = lat.structure_factor(b0, 64, K_fit)
        _, xi_par, w_par = corrlen.fit_lorentzian(s_par.cpu().numpy().mean(axis=0), 1024, return_window=True)
        _, xi_perp, w_perp = corrlen.fit_lorentzian(s_perp.cpu().numpy().mean(axis=0), 1024, return_window=True)
        extra["structure_factor"] = {"value": 64 * 1024 * 1024 / t_sf, "unit": "sites/s", "lattices": 64, "L": 1024,
                                     "K": 16, "xi_par": xi_par, "xi_perp": xi_perp, "K_fit": K_fit,
                                     "fit_windows": [list(w_par), list(w_perp)], "fit_form": "lattice",
                                     "s_half_zone": t_sf_fit}

        # plain method, 64 x 64 single lattice, 1e4 steps: resident kernel vs plain launches
        c1 = Lattice([Config(Lx=64, Ly=64, n_replicas=1, seed=1, init_mode=0, knots=((0,), (TC,)),
                             n_total=10 ** 9)], stream=stream)
        c1.step(100)
        t_b = cuda_time(lambda: c1.step(10 ** 4), stream)
        c1.set_path(XY_PATH_PLAIN)
        c1.step(100)
        t_p = cuda_time(lambda: c1.step(10 ** 4), stream)
        extra["plain_method_64x64"] = {"batched_su_per_s": 4096 * 1e4 / t_b, "plain_su_per_s": 4096 * 1e4 / t_p,
                                       "ratio": t_p / t_b}
        c1.close()

        # adjoint / forward on the differentiation workload
        del pinned
        lat.close()
        torch.cuda.empty_cache()
        c5 = Lattice([Config(Lx=256, Ly=256, n_replicas=64, seed=1, init_mode=1, knots=((0,), (TC,)),
                             n_total=10 ** 9)], stream=stream)
        c5.step(10)
        snap = c5.save()
        c5.adjoint(200, checkpoint_every=100, w_E=1.0, w_M=1.0)  # untimed: first-call tuning
        c5.load(snap)
        c5.step(2000)  # untimed: graphs of this window length
        c5.load(snap)
        t_f = cuda_time(lambda: c5.step(2000), stream)
        c5.load(snap)
        # the forward pass that evaluates the same objective: M and E every step
        t_fo = cuda_time(lambda: c5.step(2000, record_every=1), stream)
        c5.load(snap)
        t0 = time.perf_counter()
        obj, grads = c5.adjoint(2000, checkpoint_every=100, w_E=1.0, w_M=1.0)
        t_a = time.perf_counter() - t0
        # the same call with every segment recomputed forward and stored
        c5.set_adjoint_mode(XY_ADJOINT_RECOMPUTE)
        c5.load(snap)
        c5.adjoint(200, checkpoint_every=100, w_E=1.0, w_M=1.0)  # untimed: first-call tuning of this mode
        c5.load(snap)
        t0 = time.perf_counter()
        obj_r, grads_r = c5.adjoint(2000, checkpoint_every=100, w_E=1.0, w_M=1.0)
        t_r = time.perf_counter() - t0
        extra["adjoint"] = {"forward_s": t_f, "adjoint_s": t_a, "adjoint_over_forward": t_a / t_f,
                            "forward_with_objective_s": t_fo, "adjoint_over_forward_with_objective": t_a / t_fo,
                            "schedule": "states integrated backward from each checkpoint",
                            "objective": obj, "grads": grads[0].tolist(),
                            "recompute_s": t_r, "recompute_over_forward": t_r / t_f,
                            "recompute_grads": grads_r[0].tolist(),
                            "workload": "L=256 x 64 replicas, 2000 steps at T_c, checkpoint every 100"}
        c5.close()
        if world == 1:
            extra["cpu_baseline"] = cpu_baseline()

    if rank == 0:
        ok = mom[:, 0] > 0
        U = (mom[ok, 2] / mom[ok, 0]) / (mom[ok, 1] / mom[ok, 0]) ** 2
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattices": sum(c.n_replicas for c in cfgs), "sites": S,
                       "bbk_steps_per_step": INNER, "record_every": REC_EVERY, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (state of every step >> 129 MB), no flush"},
            "gpu_launches": int(launches), "clocks": clk,
            "binder_U_range": [float(U.min()), float(U.max())] if U.size else None,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The FP64 oracle as it stands on the host cores, on the same metric:
    each step is REF_INNER BBK steps of a bounded sample of the workload
    (oracle_sample: per host thread one lattice of each L at T_c)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    workers = os.cpu_count() or 1
    tasks = oracle_sample(workers)
    with ThreadPoolExecutor(max_workers=workers) as ex:
        for _ in range(args.warmup):
            oracle_round(ex, tasks, REF_INNER)
        su = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            su += oracle_round(ex, tasks, REF_INNER)
        dt = time.perf_counter() - t0
    value = su / dt
    sample = (f"{workers} lattices per L in {list(LS)} at T_c (one of each per host thread), "
              f"{REF_INNER} BBK steps per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_case(name):
    """Small single-GPU cases for profiler captures (a few hundred MB on the
    device, a few hundred launches): no JSON line, exit 0 when done."""
    import torch
    from paper_2409_06412_gb300 import Config, Lattice
    if name == "adjoint-small":
        # the differentiation shape (64 lattices of 256^2) over 200 steps, checkpoint every 100
        lat = Lattice([Config(Lx=256, Ly=256, n_replicas=64, seed=1, init_mode=1, knots=((0,), (TC,)),
                              n_total=10 ** 9)])
        lat.step(10)
        lat.adjoint(200, checkpoint_every=100, w_E=1.0, w_M=1.0)
    elif name == "adjoint-short":
        # the differentiation shape over 20 steps, checkpoint every 10: the
        # same per-step launches as above in a launch list short enough to
        # capture whole
        lat = Lattice([Config(Lx=256, Ly=256, n_replicas=64, seed=1, init_mode=1, knots=((0,), (TC,)),
                              n_total=10 ** 9)])
        lat.step(10)
        lat.adjoint(20, checkpoint_every=10, w_E=1.0, w_M=1.0)
    elif name == "plain64":
        # the plain-method lattice: 64 x 64, one replica, 300 steps
        lat = Lattice([Config(Lx=64, Ly=64, n_replicas=1, seed=1, init_mode=0, knots=((0,), (TC,)),
                              n_total=10 ** 9)])
        lat.step(100)
        lat.step(200)
    elif name == "ccl":
        # domain labels of 64 lattices of 1024^2 after 200 steps from a random start
        lat = Lattice([Config(Lx=1024, Ly=1024, n_replicas=64, seed=1, init_mode=0, knots=((0,), (TC,)),
                              n_total=10 ** 6)])
        lat.step(200)
        lat.label_domains(0, 64)
        lat.label_domains(0, 64)
    elif name in ("strip1024", "band2-1024"):
        # 128 lattices of 1024^2 (1.07 GB of state in both halves of the double
        # buffer), 32 steps with one or two steps per launch (32-row bands for
        # two); four concurrent slices of 32 lattices, each launch several waves
        lat = Lattice([Config(Lx=1024, Ly=1024, n_replicas=128, seed=1, init_mode=1, knots=((0,), (TC,)),
                              n_total=10 ** 6)])
        lat.set_autotune(False)
        lat.set_temporal_blocking(2 if name == "band2-1024" else 1)
        lat.step(32)
    elif name == "sf":
        # structure factors of 64 lattices of 1024^2 for k < 16
        lat = Lattice([Config(Lx=1024, Ly=1024, n_replicas=64, seed=1, init_mode=0, knots=((0,), (TC,)),
                              n_total=10 ** 6)])
        lat.step(2)
        lat.structure_factor(0, 64, 16)
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["static", "static-L512", "dynamic-z", "kibble-zurek"], default="static")
    ap.add_argument("--profile-case", choices=["adjoint-small", "adjoint-short", "plain64", "sf", "ccl", "strip1024",
                                               "band2-1024"], default=None,
                    help="run one small case for a profiler capture instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    set_workload(args.workload)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
