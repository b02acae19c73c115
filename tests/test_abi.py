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


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (xy_[a-z_0-9]+)", out))
    missing = _declared_symbols() - exported
    assert not missing, missing
    for name in _declared_symbols():
        assert hasattr(lib, name)


def test_library_targets_sm103a_only():
    out = subprocess.run(["cuobjdump", "--list-elf", build.LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert arches == {"103a"}, arches


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
