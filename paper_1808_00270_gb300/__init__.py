"""GB300-native integrator for discretized generalized Langevin dynamics (GLD).

Jung, Hanke & Schmid, "Generalized Langevin dynamics: Construction and
numerical integration of non-Markovian particle-based models",
arXiv:1808.00270.  The compute path is the CUDA library built from ``csrc/``
(C ABI in ``include/gld.h``); ``binding`` marshals arguments to it.
"""
from .binding import (GLD, Batch, Server, GLDError, ARR_CONV, ARR_DISP, ARR_FC, ARR_FD, ARR_FR, ARR_HIST, ARR_POS,
                      ARR_VEL, gauss3_dev, hist_conv_dev, philox_dev)

__all__ = ["GLD", "Batch", "Server", "GLDError", "ARR_POS", "ARR_VEL", "ARR_FC", "ARR_FD", "ARR_FR", "ARR_DISP", "ARR_HIST",
           "ARR_CONV", "philox_dev", "gauss3_dev", "hist_conv_dev"]
