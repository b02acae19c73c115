"""Host logic of bench.py: workload recipes, the oracle's bounded sample and
the reference arm's JSON line (the oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def bench():
    sys.path.insert(0, ROOT)
    import importlib

    import bench as b
    b = importlib.reload(b)
    yield b
    importlib.reload(b)


def test_workload_recipes(bench):
    bench.set_workload("static")
    cfgs = bench.workload_configs(1)
    assert len(cfgs) == 128 and sum(c.n_replicas for c in cfgs) == 2048
    assert sum(c.sites for c in cfgs) == 713031680
    ts = sorted({c.knots[1][0] for c in cfgs})
    assert len(ts) == 32 and ts[0] == pytest.approx(0.9 * bench.TC) and ts[-1] == pytest.approx(1.1 * bench.TC)
    bench.set_workload("dynamic-z")
    cfgs = bench.workload_configs(1)
    assert [c.Lx for c in cfgs] == [256, 512, 1024, 2048] and all(c.n_replicas == 256 for c in cfgs)
    assert bench.REC_EVERY == 10
    bench.set_workload("kibble-zurek")
    cfgs = bench.workload_configs(1)
    assert sum(c.n_replicas for c in cfgs) == 9216 and all(c.Lx == c.Ly == 1024 for c in cfgs)
    lengths = sorted({c.n_total for c in cfgs})
    assert len(lengths) == 16 and lengths[0] == 1000 + 150 and lengths[-1] == 1000 + 150000
    for c in cfgs:  # equilibrate at 1.5 T_c for 1e3 steps, then ramp to 0 over 1.5 tau_Q
        ks, Ts = c.knots
        assert ks[0] == 0 and ks[1] == 1000 and ks[2] == c.n_total
        assert Ts[0] == Ts[1] == pytest.approx(1.5 * bench.TC) and Ts[2] == 0.0
    assert {(c.params["eta"], c.params["h"]) for c in cfgs} == {(e, h) for e in (0.1, 1.0, 10.0)
                                                                  for h in (0.5, 1.0, 2.0)}


def test_oracle_sample_balances_threads(bench):
    bench.set_workload("static")
    tasks = bench.oracle_sample(3)
    # one lattice of each L per thread, largest first, distinct noise ids
    assert [t[0] for t in tasks] == [1024] * 3 + [512] * 3 + [256] * 3 + [128] * 3
    assert len({(t[1], t[2]) for t in tasks}) == len(tasks)


def test_reference_arm_prints_its_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "site-updates/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True


def test_clock_samples_summary(bench):
    rows = "\n".join([
        "0, 2070, 2070, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1395.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "",
    ])
    c = bench.parse_clock_samples(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clock_samples("0, 1500, 2070, 900, 0x28, Not Active, Active, Active, Not Active")
    assert hot["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.parse_clock_samples("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_ncu_traffic_only_for_the_profiled_source(bench, tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2409_06412_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "xy_step.cu").write_text("kernel v1\n")
    (csrc / "xy_device.cuh").write_text("header\n")
    import hashlib
    digest = hashlib.sha256(b"kernel v1\nheader\n").hexdigest()[:16]
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        f"kernel=strip_step_kernel source={digest} dram_bytes_per_site=15.94 workload=x\n"
        "kernel=strip_step_kernel source=0000000000000000 dram_bytes_per_site=99.0 workload=y\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("strip_step_kernel") == 15.94
    assert bench.ncu_traffic("other_kernel") is None
    (csrc / "xy_step.cu").write_text("kernel v2\n")  # changed since the capture
    assert bench.ncu_traffic("strip_step_kernel") is None
