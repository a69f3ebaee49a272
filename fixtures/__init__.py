"""Seeded synthetic inputs for the Nyström–Schur preconditioner (no method arithmetic).

This package only *generates* problem instances: sparse SPD diffusion matrices on
structured grids, coefficient fields, the doubly bordered block diagonal (DBBD)
partition that the paper assumes is given (§2.3, eq. (perm_A): the paper uses
METIS, here a geometric nested dissection stands in for it), a fill-reducing order of
each interior block, right-hand sides and Gaussian sketch blocks.

Both the CUDA path and the CPU oracle consume these inputs; neither is imported here.
Nothing in this package computes any step of the preconditioner itself.
"""

from .seeds import substream_seed, rng_for, MASTER_SEED
from .grids import grid_coords, diffusion_matrix
from .fields import gaussian_field, gaussian_grid_field, lognormal_field, lognormal_grid_field
from .partition import nd_partition, interior_nd_order, interface_partition
from .configs import (CONFIGS, Problem, make_problem, make_rhs, make_sketch, make_probe,
                      sample_rows,
                      batched_problem_specs, problem_from_spec)

__all__ = [
    "substream_seed", "rng_for", "MASTER_SEED", "grid_coords", "diffusion_matrix",
    "gaussian_field", "gaussian_grid_field", "lognormal_field", "lognormal_grid_field",
    "nd_partition", "interior_nd_order", "interface_partition",
    "CONFIGS", "Problem", "make_problem", "make_rhs", "make_sketch", "make_probe",
    "sample_rows",
    "batched_problem_specs", "problem_from_spec",
]
