"""Seeded synthetic workloads for the monodomain solver.

This package only *describes* problems (grid sizes, spacing, per-element fibre
directions and conductivities, stimulus node sets and times, cell-model names
and parameters, random fields and meshes).  It contains none of the method's
arithmetic (no assembly, no stability bound, no cell-model equations, no time
stepping), so that the CUDA path and the CPU oracle can both consume the same
inputs while sharing no code.
"""
from .workloads import (  # noqa: F401
    Stimulus,
    Workload,
    grid_node_coords,
    ms_square_2d,
    tp06_slab_3d,
    aniso_sheet_2d,
    cubic_strip_2d,
    tet_slab_3d,
    lognormal_field_2d,
    batch_tissues,
    ms_adjoint_2d,
    MS_DEFAULT_PARAMS,
    S1S2_S2_TIME,
)
