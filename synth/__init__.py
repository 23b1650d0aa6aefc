"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package holds input generators only: synthetic capsule hands, object
SDF grids, candidate initialisations and the workload recipes that combine
them.  It contains none of the grasp-search arithmetic (no forward
kinematics, no SDF interpolation, no contact model, no loss), so the oracle
and the CUDA path can both consume its output without sharing method code.
"""

from .hands import make_hand, interior_hand, HAND_KINDS
from .objects import (sphere_grid, box_grid, superquadric_grid, polyhedron_grid,
                      linear_grid, random_superquadric, random_polyhedron, realize)
from .candidates import sample_candidates, uniform_quaternions, quat_to_rotvec, unit_directions
from .workloads import (default_params, tiny_sphere_workload, batched_superquadric_workload,
                        polyhedra_workload, sweep_workload, serving_stream, Workload)

__all__ = [
    "make_hand", "interior_hand", "unit_directions", "HAND_KINDS", "sphere_grid", "box_grid", "superquadric_grid",
    "polyhedron_grid", "linear_grid", "random_superquadric", "random_polyhedron", "realize",
    "sample_candidates", "uniform_quaternions", "quat_to_rotvec", "default_params",
    "tiny_sphere_workload", "batched_superquadric_workload", "polyhedra_workload",
    "sweep_workload", "serving_stream", "Workload",
]
