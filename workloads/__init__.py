"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds only input generation: media (slowness kappa, attenuation
gamma), point sources and the solver settings of each workload.  It contains
none of the method's arithmetic (no operator, transfer, smoother or Krylov
code), so both the CPU oracle and the CUDA path can take their inputs from it
without sharing any computation.
"""
from .media import (  # noqa: F401
    omega_for_ppw,
    homogeneous_kappa,
    layered_kappa_2d,
    geophysical_kappa_3d,
    absorbing_gamma,
    point_source,
    random_interior_nodes,
)
from .configs import (  # noqa: F401
    SERVE_LEVELS, ServeRequest, Workload, config1, config2, config3, config4, config5, small_variant,
)
