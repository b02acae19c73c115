"""ctypes binding of the C ABI in ``include/xy_lattice.h`` (argument marshalling only).

Loading fails loudly when the CUDA library has not been built: there is no
CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

XY_OK, XY_EINVAL, XY_ENOMEM, XY_ECUDA, XY_ETIMEOUT, XY_ENAN = 0, -1, -2, -3, -4, -5
XY_INIT_UNIFORM, XY_INIT_ORDERED, XY_INIT_USER = 0, 1, 2
XY_PATH_BATCHED, XY_PATH_PLAIN = 0, 1
XY_ADJOINT_AUTO, XY_ADJOINT_RECOMPUTE, XY_ADJOINT_BACKWARD = 0, 1, 2
XY_MAX_KNOTS = 16
XY_STATIC_CCL_MAX_SITES, XY_STATIC_CCL_MAX_LATTICES = 2097152, 65536
(XY_KCLASS_RESIDENT, XY_KCLASS_STRIP, XY_KCLASS_PLAIN, XY_KCLASS_ADJ_FWD, XY_KCLASS_ADJ_RECOMP, XY_KCLASS_ADJ_REV,
 XY_KCLASS_STRIP2, XY_KCLASS_LABELS) = range(8)
XY_KCLASS_COUNT = 8

ERROR_NAMES = {XY_EINVAL: "XY_EINVAL", XY_ENOMEM: "XY_ENOMEM", XY_ECUDA: "XY_ECUDA",
               XY_ETIMEOUT: "XY_ETIMEOUT", XY_ENAN: "XY_ENAN"}

# every symbol the header declares, with (restype, argtypes)
_c = ctypes
_vp, _i32, _i64, _u32, _u64, _d, _sz = _c.c_void_p, _c.c_int, _c.c_int64, _c.c_uint32, _c.c_uint64, _c.c_double, _c.c_size_t


class ConfigDesc(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("n_replicas", ctypes.c_int32),
                ("init_mode", ctypes.c_int32), ("seed", ctypes.c_uint64), ("cfg_id", ctypes.c_int32),
                ("replica0", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("J_par", _d), ("J_perp", _d), ("h", _d), ("p", _d), ("q", _d), ("eta", _d), ("dt", _d),
                ("staggered_M", ctypes.c_int32), ("reserved", ctypes.c_int32)]


SIGNATURES = {
    "xy_lattice_create": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "xy_set_params": (_i32, [_vp, _i32, _vp]),
    "xy_set_schedule": (_i32, [_vp, _i32, _vp, _vp, _i32, _i64]),
    "xy_step_n": (_i32, [_vp, _i64, _i32, _vp, _i64]),
    "xy_observe": (_i32, [_vp, _vp, _vp]),
    "xy_reset_moments": (_i32, [_vp]),
    "xy_omega_full": (_i32, [_vp, _i32, _i32, _vp]),
    "xy_label_domains": (_i32, [_vp, _i32, _i32, _vp, _vp, _i64, _vp]),
    "xy_adjoint_step_n": (_i32, [_vp, _i64, _i32, _d, _d, _vp, _vp]),
    "xy_set_field_schedule": (_i32, [_vp, _i32, _vp, _vp, _i32]),
    "xy_set_coupling_schedule": (_i32, [_vp, _i32, _vp, _vp, _vp, _i32]),
    "xy_set_temporal_blocking": (_i32, [_vp, _i32]),
    "xy_set_adjoint_mode": (_i32, [_vp, _i32]),
    "xy_label_domains_static": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _i64, _vp, _vp]),
    "xy_structure_factor": (_i32, [_vp, _i32, _i32, _i32, _d, _vp, _vp]),
    "xy_autocorr_time": (_i32, [_vp, _i64, _i64, _i32, _i32, _i64, _i64, _d, _vp, _vp]),
    "xy_set_power_quench": (_i32, [_vp, _i32, _d, _i64, _d, _d, _d, _d, _i64]),
    "xy_set_path": (_i32, [_vp, _i32]),
    "xy_autotune": (_i32, [_vp]),
    "xy_set_autotune": (_i32, [_vp, _i32]),
    "xy_save": (_i32, [_vp, _vp, _vp]),
    "xy_load": (_i32, [_vp, _vp, _sz]),
    "xy_synchronize": (_i32, [_vp]),
    "xy_kernel_launches": (_i64, [_vp]),
    "xy_set_kernel_timing": (_i32, [_vp, _i32]),
    "xy_kernel_timing": (_i32, [_vp, _vp, _vp]),
    "xy_lattice_destroy": (None, [_vp]),
    "xy_last_error": (_c.c_char_p, []),
    "xy_debug_noise": (_i32, [_u64, _i32, _i32, _i64, _i32, _i64, _vp, _vp, _vp]),
    "xy_debug_philox": (_i32, [_vp, _u32, _u32, _i64, _vp, _vp]),
    "xy_debug_gauss4": (_i32, [_vp, _i64, ctypes.c_float, _vp, _vp]),
    "xy_debug_set_union_limit": (_i32, [_i32]),
    "xy_debug_slice_parts": (_i32, [_vp, _i32, _i32, _i32, _vp]),
    "xy_debug_slice_cuts": (_i32, [_vp, _i32, _i32, _vp, _vp]),
}

_lib = None


class XYError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the built library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"the CUDA library {p} is not built; run paper_2409_06412_gb300.build.build() "
                           "(nvcc, sm_103a) first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, fn: str):
    if code != XY_OK:
        msg = load().xy_last_error()
        raise XYError(code, fn, msg.decode() if msg else "")
    return code


def call(fn: str, *args):
    return check(getattr(load(), fn)(*args), fn)
