"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds no arithmetic of the method itself (no streaming, collision,
forcing, filtering, quantity of interest, pattern or regression step).  It only
produces the *inputs* that both implementations consume:

* initial macroscopic fields (density 1, seeded velocity perturbations, the
  laminar channel parabola),
* synthetic time-series-model coefficients (regression matrix, residual mean and
  covariance, reference scales) of the shapes the paper's LRS model has,
* lattice-unit parameter sets for the paper's two flows,
* the workload descriptions used by the tests and the benchmark.

Every generator is seeded (numpy PCG64) so both sides see identical inputs.
"""

from .units import kolmogorov_lattice, channel_lattice  # noqa: F401
from .fields import uniform_noise_u0, channel_u0, initial_velocity  # noqa: F401
from .lrs_inputs import synthetic_lrs  # noqa: F401
from .workloads import WORKLOADS, serving_requests, workload  # noqa: F401
