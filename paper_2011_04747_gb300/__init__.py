"""GB300-native dual adaptive explicit monodomain solver (arXiv:2011.04747).

The compute path is ``libdaeti.so`` (hand-written sm_103a CUDA behind the C
ABI of ``include/daeti.h``); ``binding`` is its thin ctypes binding.  Build
with ``paper_2011_04747_gb300.build.build()``.
"""
from .binding import (  # noqa: F401
    DaetiError,
    Solver,
    load_library,
    solver_from_workload,
)
