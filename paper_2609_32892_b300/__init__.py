"""B300-native fused lattice-Boltzmann LES step with the Tau-orthogonal SGS
forcing: a C-ABI CUDA library (liblbm.so, include/lbm.h) and its Python
binding.  PyTorch supplies device memory and streams only."""

from .binding import *  # noqa: F401,F403
from .sim import LbmSim  # noqa: F401
