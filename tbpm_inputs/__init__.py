"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package generates Hamiltonians, on-site disorder and random-phase states.
It holds none of the propagation method's arithmetic, so that the oracle and
the CUDA library stay independent of each other and meet only here.
"""
from .rng import splitmix64, uniform01
from .states import random_phase_state, random_phase_block, site_state
from .lattice import (CSR, anderson_onsite, graphene_csr, bilayer_csr, random_hermitian_csr,
                      gershgorin_bound, T_GRAPHENE, T_PERP_AB, A_LATTICE, Current, graphene_current,
                      bilayer_current, graphene_positions, graphene_geometry, graphene_area_per_orbital)
from .batch import Instance, batch_instances

__all__ = [
    "splitmix64", "uniform01", "random_phase_state", "random_phase_block", "site_state",
    "CSR", "anderson_onsite", "graphene_csr", "bilayer_csr", "random_hermitian_csr",
    "gershgorin_bound", "T_GRAPHENE", "T_PERP_AB", "Instance", "batch_instances", "A_LATTICE", "Current",
    "graphene_current", "bilayer_current", "graphene_positions", "graphene_geometry",
    "graphene_area_per_orbital",
]
