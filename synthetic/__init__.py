"""Seeded synthetic input generators (Philox4x32-10). Holds none of the method's arithmetic."""
from .philox import philox4x32_10, u53  # noqa: F401
from .workloads import (  # noqa: F401
    BATCHED, LARGE, MEDIUM, TINY, Workload, coulomb_v, eps_occ, eps_unocc, omega_grid, z_block, z_rows,
)
