"""The hardware-function constants of the FP32 error model (tests/gpu_helpers.py)
checked by exhaustive sweeps on the GPU, so that the first-order bound of the
parity tests rests on measured, not assumed, error bounds:

- the fast sine and cosine at every argument the steppers form from a stored
  angle (q theta and fl(p theta) for every binary32 |theta| <= pi/2);
- the library's Box-Muller map (xy_debug_gauss4, the code the steppers run)
  at every uniform the generator can produce: every radius with the angle
  near 0, and every angle at the largest radius, against the FP64 map of the
  same uniforms (App. A.1 noise, one unit Gaussian per site and step).
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest
import torch

from paper_2409_06412_gb300 import _lib, build
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_hardware_sine_cosine_errors_within_the_model():
    src = os.path.join(os.path.dirname(__file__), "cuda", "intrinsic_error.cu")
    so = os.path.join(tempfile.mkdtemp(), "intrinsic_error.so")
    subprocess.check_call([build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-fmad=false", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.intrinsic_error.argtypes = [ctypes.c_uint32, ctypes.c_void_p]
    err = np.zeros(4, dtype=np.float32)
    half_pi_bits = int(np.float32(math.pi / 2).view(np.uint32))  # the wrap's binary32 pi/2
    assert lib.intrinsic_error(half_pi_bits + 1, err.ctypes.data) == 0
    print(f"max |error| over all binary32 |theta| <= pi/2: sin 2t {err[0]:.3g}, cos 2t {err[1]:.3g}, "
          f"sin 2.5t {err[2]:.3g}, cos 2.5t {err[3]:.3g} (model: ESC {gh.ESC:.3g}, ESP {gh.ESP:.3g})")
    assert err[0] <= gh.ESC and err[1] <= gh.ESC
    assert err[2] <= gh.ESP


def _gauss4(words: np.ndarray) -> np.ndarray:
    w = torch.from_numpy(words.view(np.int32)).cuda()
    out = torch.empty(words.size, dtype=torch.float32, device="cuda")
    _lib.call("xy_debug_gauss4", ctypes.c_void_p(w.data_ptr()), words.shape[0], ctypes.c_float(1.0),
              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64).reshape(-1, 4)


def test_box_muller_error_within_the_model():
    m = np.arange(1 << 23, dtype=np.uint64)
    u = (m.astype(np.float64) + 0.5) * 2.0 ** -23           # every uniform of the generator
    # every radius: u0 over all 2^23 values, u1 = 1/2 - 2^-24 (angle near 0 after the shift by -pi)
    m_half = (1 << 22) - 1
    u1 = (m_half + 0.5) * 2.0 ** -23
    words = np.zeros((m.size, 4), dtype=np.uint32)
    words[:, 0] = (m << 9).astype(np.uint32)
    words[:, 1] = m_half << 9
    g = _gauss4(words)
    r = np.sqrt(-2.0 * np.log(u))
    err_r = np.abs(g[:, 0] - r * np.cos(2 * np.pi * u1))
    excess_r = err_r - (gh.ER1 / r + gh.ERR * r)
    # every angle at the largest radius (u0 = 2^-24)
    words[:, 0] = 0
    words[:, 1] = (m << 9).astype(np.uint32)
    g = _gauss4(words)
    err_a = np.maximum(np.abs(g[:, 0] - gh.R_MAX * np.cos(2 * np.pi * u)), np.abs(g[:, 1] - gh.R_MAX * np.sin(2 * np.pi * u)))
    # R_MAX |co~ - cos| <= |g~ - R_MAX cos| + |r~ - R_MAX| |co~|: the angle's share of the error per unit radius
    e_trig = (err_a.max() + err_r[0]) / gh.R_MAX
    worst = int(np.argmax(excess_r))
    print(f"Box-Muller: radius error at most {err_r.max():.3g} (at u0 = {u[np.argmax(err_r)]:.8f}); largest "
          f"excess over ER1/r + ERR r {excess_r[worst]:.3g} at u0 = {u[worst]:.8f} (r = {r[worst]:.3g}); angle error "
          f"per unit radius {e_trig:.3g} (ETRIG {gh.ETRIG:.3g})")
    assert excess_r.max() <= 0.0
    assert e_trig <= gh.ETRIG
