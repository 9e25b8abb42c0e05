"""Seeded synthetic inputs shaped like the paper's workloads.

This package only builds meshes, permeability fields and boundary data. It holds none of the solver's
arithmetic: both the FP64 oracle (through the tests) and the CUDA library consume what it returns.
"""
from .grids import (Mesh, cartesian_mesh, lognormal_field, channelized_field, problem_config,
                    CONFIGS)

__all__ = ["Mesh", "cartesian_mesh", "lognormal_field", "channelized_field", "problem_config", "CONFIGS"]
