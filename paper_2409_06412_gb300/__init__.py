"""GB300 (sm_103a) Langevin stepper for the Si(001) dimer-angle XY model
(arXiv 2409.06412): BBK dynamics, FP64 observables, domain labelling and a
pathwise adjoint, behind the C ABI of ``include/xy_lattice.h``."""
from . import _lib
from ._lib import (XY_ADJOINT_AUTO, XY_ADJOINT_BACKWARD, XY_ADJOINT_RECOMPUTE, XY_INIT_ORDERED, XY_INIT_UNIFORM,
                   XY_INIT_USER, XY_PATH_BATCHED, XY_PATH_PLAIN, XYError, load)
from .lattice import PAPER_PARAMS, Config, Lattice, debug_noise, debug_philox

__all__ = ["Config", "Lattice", "PAPER_PARAMS", "XYError", "load", "debug_noise", "debug_philox",
           "XY_INIT_UNIFORM", "XY_INIT_ORDERED", "XY_INIT_USER", "XY_PATH_BATCHED", "XY_PATH_PLAIN",
           "XY_ADJOINT_AUTO", "XY_ADJOINT_RECOMPUTE", "XY_ADJOINT_BACKWARD", "_lib"]
