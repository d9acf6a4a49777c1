"""Seeded synthetic inputs for the recycling Krylov solvers.

This package builds the structured-grid operators (banded coefficients) and
right-hand-side sequences that stand in for the paper's GenIDLEST pressure
systems (Sec. 3: turbulent channel, porous medium). It holds no solver
arithmetic: it is shared by the CPU oracle and by the CUDA library's callers
and imports neither.

Layout convention (the paper's banded "diagonal" storage, Sec. 2.1, 'Data
Layout'): coefficients are a float64 array ``coef[S, N]`` with
``N = nx*ny*nz`` cells indexed ``i + nx*(j + ny*k)`` (x fastest) and band ``s``
multiplying the unknown at offset ``OFFSETS[s]``.
"""
from .grid import Grid, OFFSETS, S7, S19
from .operators import (
    convection_diffusion_7pt,
    channel_7pt,
    porous_skew_19pt,
    random_operator,
)
from .fields import smooth_noise, divergence_sequence
from .configs import make_config, ConfigProblem, CONFIG_SEED_BASE

__all__ = [
    "Grid", "OFFSETS", "S7", "S19",
    "convection_diffusion_7pt", "channel_7pt", "porous_skew_19pt", "random_operator",
    "smooth_noise", "divergence_sequence",
    "make_config", "ConfigProblem", "CONFIG_SEED_BASE",
]
