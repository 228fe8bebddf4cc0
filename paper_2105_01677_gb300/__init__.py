"""GB300-native MPS time-step library (arXiv 2105.01677 hot path).

The product is the shared library built from ``csrc/`` (C ABI in ``include/mps.h``);
``mps`` is its thin ctypes binding.  Build with ``__graft_entry__.build()`` or
``python -m paper_2105_01677_gb300._build``.
"""
from . import _build  # noqa: F401
from .mps import (  # noqa: F401
    EXPORTS, FLUID, WALL, DUMMY, GHOST, MPSError, Simulation, lib, mps_create, mps_debug_cells,
    mps_debug_neighbors, mps_destroy, mps_get_constants, mps_params, mps_params_default,
    mps_get_profile, mps_read_state, mps_report, mps_set_profiling, mps_solve_ppe, mps_step, mps_strerror, mps_write_state)
