"""CPU oracle for the recycling Krylov solvers — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 implementation of what the GPU library computes, written
from the paper (Algorithms 1-4, Sec. 2.2-2.4) and checked against pins that
do not depend on it (dense LU solves, closed forms, invariants, special cases
that reduce to textbook methods; see tests/test_oracle_*.py). Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product library never does, and the two share no code. The
seeded problem generators live in the separate package ``problems``.

Parity status of each function:
* ``Stencil.apply/apply_prec/residual``: pinned (brute-force dense matrix).
* ``gmres``: pinned (dense LU, finite termination, monotone residuals).
* ``rgcrot``: pinned (k=0 equals ``gmres`` exactly; dense LU; A U = C,
  C^T C = I, V ⟂ C, augmented Arnoldi relation; exact recycling).
* ``harmonic_ritz_update``: pinned (independent dense harmonic Ritz values,
  and the selected subspace against the eigenvectors of the k smallest
  |theta| of the explicit dense pencil).
* ``bicgstab``: pinned (dense LU).
* ``rbicgstab``: pinned (empty recycle space equals ``bicgstab`` exactly;
  dense LU; r ⟂ C; solution/residual relation).
* ``Stencil.apply_f32/schwarz_f32`` (the FP32 restatements of the mixed
  precision): pinned within FP32 rounding of the pinned FP64 forms.
* Iteration counts of the paper's Tables 2-8: parity unpinned (the paper's
  matrices are not available).
"""
from ._clib import Stencil, build as build_clib
from .krylov import (
    OK, NOT_CONVERGED, BREAKDOWN,
    gmres, rgcrot, bicgstab, rbicgstab, harmonic_ritz_update, recycle_from_u, RecyclingSequence,
)
from .dense import dense_matrix

__all__ = [
    "Stencil", "build_clib", "OK", "NOT_CONVERGED", "BREAKDOWN", "gmres", "rgcrot", "bicgstab",
    "rbicgstab", "harmonic_ritz_update", "recycle_from_u", "RecyclingSequence", "dense_matrix",
]
