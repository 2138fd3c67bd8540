"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the finite element method itself: no basis
functions, no quadrature, no DoF numbering, no coefficient laws.  It only
draws random numbers and evaluates input fields (signed distances, initial
level sets, convection fields, initial temperatures) at coordinates the
caller supplies, and it builds the adaptive leaf list that both sides take as
their mesh input.  Both sides call the same functions on their own node
coordinates, so the inputs they see are bit-identical.

Random numbers come from splitmix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used as a
counter-based generator: output i of stream ``seed`` is mix(seed + (i+1)*gamma).
"""
from .rng import splitmix64, uniform_pm1, uniform_01
from .fields import (sphere_distance, wavy_plane_distance, deformed_sphere_distance,
                     initial_level_set, convection_field, heat_initial_temperature,
                     heat_target_temperature, kq_field, wavy_plane_phases, interface_temperature,
                     meltpool_state)
from .octree import refine_band_leaves, is_two_to_one_balanced
from .workloads import (TI64, EVAPORATION, HELMHOLTZ_SPHERE, OSEEN_INTERFACE, HEAT_LASER, HEAT_ADJOINT,
                        REINIT_OCTREE, MELTPOOL_STEP, Workload, scaled)

__all__ = [
    "splitmix64", "uniform_pm1", "uniform_01", "sphere_distance", "wavy_plane_distance",
    "deformed_sphere_distance", "initial_level_set", "convection_field",
    "heat_initial_temperature", "heat_target_temperature", "kq_field", "wavy_plane_phases",
    "interface_temperature", "meltpool_state", "EVAPORATION", "MELTPOOL_STEP",
    "refine_band_leaves", "is_two_to_one_balanced", "TI64", "HELMHOLTZ_SPHERE",
    "OSEEN_INTERFACE", "HEAT_LASER", "HEAT_ADJOINT", "REINIT_OCTREE", "Workload", "scaled",
]
