"""GB300 (sm_103a) multilayer shallow-water lattice Boltzmann solver for the
n-layer thin-film equation.

The solver lives in the CUDA library ``_lib/libmlswlbm.so`` behind the C ABI
of ``include/mlswlbm.h``; :mod:`.mlswlbm` is its ctypes binding.
"""
from .mlswlbm import (  # noqa: F401
    MLSW_D1Q3, MLSW_D2Q9, MLSW_MAX_LAYERS, MlswError, Solver, lib,
    mlswlbm_create, mlswlbm_destroy, mlswlbm_friction_eval, mlswlbm_get_diagnostics,
    mlswlbm_get_heights, mlswlbm_get_state, mlswlbm_set_heights, mlswlbm_set_state,
    mlswlbm_spreading_from_tensions, mlswlbm_status, mlswlbm_step, mlswlbm_strerror,
    mlswlbm_check_params,
)
