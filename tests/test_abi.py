"""The C-ABI library builds, loads and exports every symbol the header
declares; host-side argument checks work without a GPU (no kernel runs)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2409_06412_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(xy_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_and_binding_agree():
    declared = _declared_symbols()
    assert declared, "no declarations found"
    assert declared == set(_lib.SIGNATURES), declared ^ set(_lib.SIGNATURES)


def test_binding_constants_match_the_header():
    """Every integer #define XY_... of the header that the binding also
    defines has the same value there."""
    src = open(os.path.join(ROOT, "include", "xy_lattice.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(XY_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src)}
    shared = {k for k in defs if hasattr(_lib, k)}
    assert {"XY_KCLASS_LABELS", "XY_KCLASS_COUNT", "XY_INIT_ORDERED", "XY_ETIMEOUT"} <= shared
    for k in shared:
        assert getattr(_lib, k) == defs[k], k


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (xy_[a-z_0-9]+)", out))
    missing = _declared_symbols() - exported
    assert not missing, missing
    for name in _declared_symbols():
        assert hasattr(lib, name)


def test_build_targets_sm103a_only():
    # every translation unit and the link take exactly this one -gencode
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("arch" in f or "gencode" in f for f in build.FLAGS)


def test_host_side_argument_checks(lib):
    h = ctypes.c_void_p()
    rc = lib.xy_lattice_create(None, 1, None, None, None, ctypes.byref(h))
    assert rc == _lib.XY_EINVAL
    assert b"configuration" in lib.xy_last_error() or lib.xy_last_error()
    assert lib.xy_set_params(None, 0, None) == _lib.XY_EINVAL
    assert lib.xy_step_n(None, 1, 0, None, 0) == _lib.XY_EINVAL
    assert lib.xy_observe(None, None, None) == _lib.XY_EINVAL
    assert lib.xy_kernel_launches(None) == -1
    assert lib.xy_debug_noise(1, 70000, 0, 0, 0, 1, None, None, None) == _lib.XY_EINVAL
    lib.xy_lattice_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "absent.so"))
    finally:
        _lib._lib = saved


def _slice_parts(lib, n_lat, fixed, budget):
    arr = (ctypes.c_int64 * max(1, len(n_lat)))(*n_lat)
    out = (ctypes.c_int * max(1, len(n_lat)))()
    assert lib.xy_debug_slice_parts(arr, len(n_lat), fixed, budget, out) == _lib.XY_OK
    return list(out)[:len(n_lat)]


def _slice_cuts(lib, lattice_of_task, parts):
    arr = (ctypes.c_int32 * max(1, len(lattice_of_task)))(*lattice_of_task)
    cuts = (ctypes.c_int * (parts + 1))()
    n = ctypes.c_int()
    assert lib.xy_debug_slice_cuts(arr, len(lattice_of_task), parts, cuts, ctypes.byref(n)) == _lib.XY_OK
    return list(cuts)[:n.value]


def test_slice_plan_counts(lib):
    # static-criticality batch: three strip shapes of 512 lattices beside one
    # resident group, nine branches at most
    assert _slice_parts(lib, [512, 512, 512], 1, 9) == [2, 3, 3]
    assert _slice_parts(lib, [64], 0, 9) == [4]
    assert _slice_parts(lib, [1], 0, 9) == [1]
    assert _slice_parts(lib, [3, 0], 0, 9) == [3, 1]
    # more groups than the budget: one branch each, nothing left to take
    assert _slice_parts(lib, [2] * 12, 0, 9) == [1] * 12
    # the budget binds: the groups with most slices give one up first
    assert _slice_parts(lib, [8, 8, 2], 2, 8) == [2, 2, 2]
    for n_lat, fixed, budget in [([5, 7, 1, 300], 1, 9), ([10] * 3, 0, 12), ([1000], 3, 4)]:
        p = _slice_parts(lib, n_lat, fixed, budget)
        assert all(1 <= x <= min(4, max(1, n)) for x, n in zip(p, n_lat))
        assert fixed + sum(p) <= budget or all(x == 1 for x in p)


def test_slice_cuts_fall_on_lattice_starts(lib):
    # L = 1024 of the static batch: 512 lattices of 16 blocks in three slices
    tasks = [b // 16 for b in range(8192)]
    assert _slice_cuts(lib, tasks, 3) == [0, 2736, 5456, 8192]
    assert _slice_cuts(lib, [0] * 7, 4) == [0, 7]              # one lattice: one slice
    assert _slice_cuts(lib, [0] * 10 + [1, 2, 3, 4], 2) == [0, 10, 14]
    assert _slice_cuts(lib, [0, 1] + [2] * 100, 3) == [0, 2, 102]  # no start left for a third
    assert _slice_cuts(lib, [], 2) == [0, 0]
    import random
    rng = random.Random(7)
    for _ in range(50):
        sizes = [rng.randint(1, 20) for _ in range(rng.randint(1, 40))]
        tasks = [i for i, s in enumerate(sizes) for _ in range(s)]
        parts = rng.randint(1, 4)
        c = _slice_cuts(lib, tasks, parts)
        starts = {0} | {i for i in range(1, len(tasks)) if tasks[i] != tasks[i - 1]}
        assert c[0] == 0 and c[-1] == len(tasks) and 2 <= len(c) <= parts + 1
        assert all(a < b for a, b in zip(c, c[1:]))
        assert all(x in starts for x in c[:-1])


def test_slice_plan_argument_checks(lib):
    out = (ctypes.c_int * 2)()
    assert lib.xy_debug_slice_parts(None, 1, 0, 9, out) == _lib.XY_EINVAL
    arr = (ctypes.c_int64 * 1)(-1)
    assert lib.xy_debug_slice_parts(arr, 1, 0, 9, out) == _lib.XY_EINVAL
    assert lib.xy_debug_slice_parts(arr, 0, 0, 0, out) == _lib.XY_EINVAL
    tasks = (ctypes.c_int32 * 3)(0, 2, 1)
    cuts = (ctypes.c_int * 3)()
    n = ctypes.c_int()
    assert lib.xy_debug_slice_cuts(tasks, 3, 2, cuts, ctypes.byref(n)) == _lib.XY_EINVAL
    assert lib.xy_debug_slice_cuts(tasks, 3, 0, cuts, ctypes.byref(n)) == _lib.XY_EINVAL
