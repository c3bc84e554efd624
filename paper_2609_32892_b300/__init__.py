"""B300-native fused lattice-Boltzmann LES step with the Tau-orthogonal SGS
forcing: a C-ABI CUDA library (liblbm.so, include/lbm.h) and its Python
binding.  PyTorch supplies device memory and streams only.

The library is loaded on first use of the binding (so that `build` can run
before it exists); a missing or stale liblbm.so raises at that point.  There is
no fallback implementation."""

import importlib


def __getattr__(name):
    if name in ("build",):
        return importlib.import_module(f"{__name__}.build")
    if name in ("binding", "sim"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("LbmSim", "nq_of"):
        return getattr(importlib.import_module(f"{__name__}.sim"), name)
    binding = importlib.import_module(f"{__name__}.binding")
    try:
        return getattr(binding, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
