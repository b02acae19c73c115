"""Error analysis and adaptive sampling of recorded observables
(arXiv 2409.06412, App. B).

``autocorr_time`` runs on the GPU over the records that ``Lattice.step``
returns (one series per lattice); ``suggest_record_every`` turns the
integrated autocorrelation time into the next sampling interval,
ds ~ tau_C / 10 with ds >= 100 dt (100 steps), as the paper adapts it during
a run.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

COMPONENTS = {"M": 0, "E": 1}
TRANSFORMS = {"f": 0, "f2": 1, "f4": 2, "abs": 3}


def autocorr_time(rec: torch.Tensor, observable: str = "M", transform: str = "f", skip: int = 0,
                  n: int | None = None, c_window: float = 6.0) -> torch.Tensor:
    """rec: (B, R, 2) float64 device records of (M, E).  Returns a (B, 4)
    float64 device tensor of (mean, variance, tau_C in records, error of the
    mean) of g(f) over records skip .. skip + n - 1.  c_window <= 0 integrates
    to half the series (the paper's window taken literally)."""
    if rec.dtype != torch.float64 or rec.dim() != 3 or rec.shape[2] != 2 or not rec.is_cuda:
        raise ValueError("rec must be a (B, R, 2) float64 CUDA tensor")
    rec = rec.contiguous()
    B, R, _ = rec.shape
    n = R - skip if n is None else n
    out = torch.empty((B, 4), dtype=torch.float64, device=rec.device)
    stream = torch.cuda.current_stream(rec.device).cuda_stream
    L.call("xy_autocorr_time", ctypes.c_void_p(rec.data_ptr()), int(B), int(R), COMPONENTS[observable],
           TRANSFORMS[transform], int(skip), int(n), float(c_window), ctypes.c_void_p(out.data_ptr()),
           ctypes.c_void_p(stream))
    return out


def suggest_record_every(tau_records: float, record_every: int, min_steps: int = 100) -> int:
    """Next sampling interval in steps: tau_C / 10 with tau_C = tau_records *
    record_every steps, at least min_steps (ds >~ 100 dt)."""
    return max(int(min_steps), int(round(tau_records * record_every / 10.0)))
