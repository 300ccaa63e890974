"""Seeded synthetic molecules (atom centres and radii) for tests and benchmarks.

This module only draws random inputs; it holds none of the meshing arithmetic.
Both the CPU oracle and the CUDA path receive its arrays, so neither depends
on the other.  Recipes (radius mix, densities, sizes) follow the workloads of
TMSmesh 2.0's benchmark (Table 1: single molecules from tens of atoms up to a
1.08M-atom virus envelope); the paper's PQR files themselves are not used.
"""
from .molecules import (RADII, RADII_WEIGHTS, draw_radii, chain, globular,
                        icosahedral_rotations, assembly, batch_specs, config)

__all__ = ["RADII", "RADII_WEIGHTS", "draw_radii", "chain", "globular",
           "icosahedral_rotations", "assembly", "batch_specs", "config"]
