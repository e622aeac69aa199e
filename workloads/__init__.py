"""Seeded synthetic sparse matrices shaped like the paper's workloads.

This module only draws random structure and values and assembles CSC arrays.
It contains none of the SpGEMM arithmetic: both the CPU oracle side and the
CUDA side take their inputs from here, and nothing here depends on either.

Every generator is deterministic in its seed (numpy PCG64 ``default_rng``).
The paper's datasets (Table 5: protein-similarity networks, Friendster) are
not available; the generators below stand in for them:

* ``er_exact``      -- every column has exactly ``d`` distinct rows drawn
                       uniformly without replacement, stored in draw order
                       (unsorted), as in the small Erdos-Renyi workloads.
* ``rmat``          -- R-MAT edge draws (per-level independent quadrant draws,
                       no noise, no vertex permutation), symmetrised as
                       X + X^T with duplicates summed (social-graph stand-in).
* ``lognormal_symmetric`` -- Chung-Lu style symmetric matrix with lognormal
                       column degrees (protein-similarity stand-in).
* ``er_binomial`` / ``multi_problem_set`` -- G(n, p) columns with Binomial
                       counts, for the many-uneven-problems workload.
"""
from .csc import CSC, from_coo, transpose, shuffle_within_columns, column_slice
from .generators import (
    CONFIG_SEED_BASE,
    config_seed,
    er_exact,
    rmat,
    lognormal_symmetric,
    er_binomial,
    multi_problem_set,
    values_on_pattern,
    config1,
    config2,
    config3,
    config4,
    config5,
)

__all__ = [
    "CSC", "from_coo", "transpose", "shuffle_within_columns", "column_slice",
    "CONFIG_SEED_BASE", "config_seed", "er_exact", "rmat", "lognormal_symmetric",
    "er_binomial", "multi_problem_set", "values_on_pattern",
    "config1", "config2", "config3", "config4", "config5",
]
