"""Seeded synthetic inputs for the null-space solver.

This package only builds matrices (CSR arrays) and their planted structure
(component labels, copied-column pairs).  It holds none of the solver's
arithmetic, so both the CPU oracle and the CUDA library may consume its output.
"""

from .graphs import (  # noqa: F401
    CSR,
    Workload,
    config_seed,
    solver_seed,
    laplacian_er_components,
    laplacian_cycle_components,
    laplacian_grid_components,
    incidence_cycle_components,
    rectangular_copies,
    rectangular_copies_scaled,
    batched_laplacians,
    diag_example,
    tiny_planted,
    make_config,
    CONFIGS,
)
