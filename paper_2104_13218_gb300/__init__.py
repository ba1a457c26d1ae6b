"""GB300-native stochastic Chebyshev (KPM) typicality for spin-1/2 Heisenberg models.

The compute path is libkpm.so (CUDA for sm_103a, C ABI in include/kpm.h);
this package only marshals arguments (see api.py).
"""
from ._lib import KPMError, lib, library_path  # noqa: F401
from . import analysis  # noqa: F401
from .api import (ChebyshevThermo, CModel, SectorSet, autotune, bounds,  # noqa: F401
                  bounds_workspace_size, chebyshev_thermo, fp64_peak, moments, moments_backward,
                  moments_backward_workspace_size, moments_workspace_size, realisations,
                  sector_dims, sector_set, spin_bounds, spin_moments, spin_sector_dims,
                  spin_sector_set, thermo, thermo_backward)

__all__ = ["lib", "library_path", "KPMError", "bounds", "moments", "thermo", "thermo_backward",
           "moments_backward", "chebyshev_thermo", "ChebyshevThermo", "sector_set", "sector_dims",
           "bounds_workspace_size", "moments_workspace_size", "moments_backward_workspace_size",
           "CModel", "SectorSet", "realisations", "autotune", "fp64_peak", "spin_bounds",
           "spin_moments", "spin_sector_dims", "spin_sector_set"]
