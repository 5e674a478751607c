"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package only *generates* inputs: closed triangle meshes snapped to the
2^-20 grid, lattice populations and per-link weights.  It holds none of the
embedding arithmetic (no predicates, no voxelization, no link lengths), so both
the CUDA path and the CPU oracle can consume it without sharing method code.
"""
from .meshes import (  # noqa: F401
    GRID_BITS,
    snap,
    icosphere,
    radial_star,
    axis_box,
    tetrahedron,
    octahedron,
    corner_face_tetrahedra,
    bump,
    signed_volume,
)
from .workloads import (  # noqa: F401
    Workload,
    WORKLOADS,
    workload,
    batch_meshes,
    populations,
    link_weights,
    D3Q27_DIRS,
    D3Q19_WEIGHTS,
)
