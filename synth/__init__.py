"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds workload descriptions (grid sizes, frequency, solver
settings) and generators for media, point sources and receivers.  It holds
none of the solver's arithmetic: no PML profile, no stencil, no domain
decomposition.  Both ``oracle/`` and the product package import it; it
imports neither.
"""

from .configs import CONFIGS, Workload, workload, scaled_workload, adjoint_workload_2d  # noqa: F401
from .media import medium, velocity, sources, source_nodes, receivers, fd_directions  # noqa: F401
