"""GB300-native explicit forward-Euler step for phase-field (Allen-Cahn, Cahn-Hilliard,
Model C) and reaction-diffusion (Gray-Scott, N coupled species) models on periodic 2D/3D
grids, plus the
semi-implicit Fourier spectral solver and the structure factor (arxiv 2109.02598).

The compute path is libpfgpu.so (hand-written CUDA for sm_103a behind the C ABI of
``include/pfgpu.h``); this package only marshals arguments to it.
"""
from ._lib import PF_TILE_BANDS, PF_TILE_STRIPS, PfError, load  # noqa: F401
from .grid import Grid, rd_coeffs  # noqa: F401
from .adjoint import (GrayScottAdjoint, PhaseFieldAdjoint, adjoint_backward,  # noqa: F401
                      adjoint_forward)
from .batch import Batch, shard_instances  # noqa: F401
from .spectral import Spectral, porod_fit, structure_factor  # noqa: F401
from .slab import SlabGrid, SlabLayout, slab_range  # noqa: F401

__all__ = ["PF_TILE_BANDS", "PF_TILE_STRIPS", "Batch", "Grid", "shard_instances", "GrayScottAdjoint", "PhaseFieldAdjoint", "PfError",
           "Spectral", "adjoint_backward", "adjoint_forward", "load", "porod_fit",
           "SlabGrid", "SlabLayout", "rd_coeffs", "slab_range", "structure_factor"]
