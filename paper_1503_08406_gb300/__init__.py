"""GB300-native double-MRT lattice Boltzmann solver for solid-liquid phase
change with natural convection in porous media (Liu & He, arXiv:1503.08406).

The computation lives in liblbm.so (CUDA, sm_103a; C ABI in include/lbm.h).
This package is its binding: :class:`Lattice`, :class:`Batch` and the ``lbm_*`` wrappers.
"""
from .lbm import (  # noqa: F401
    BC, Batch, LBMError, Lattice, declared_functions, lbm_create, lbm_destroy, lbm_error_string,
    lbm_params, lbm_status, lbm_step, lbm_workspace_bytes, load, make_params,
)

__all__ = ["Lattice", "Batch", "LBMError", "load", "make_params", "lbm_params", "declared_functions",
           "lbm_create", "lbm_destroy", "lbm_step", "lbm_status", "lbm_workspace_bytes",
           "lbm_error_string", "BC"]
