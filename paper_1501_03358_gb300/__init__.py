"""GB300 (sm_103a) recycling Krylov solvers for sequences of nonsymmetric
structured-grid systems: GMRES(m), rGCROT(m,k), rBiCGStab and the
rGCROT -> rBiCGStab hybrid of arXiv 1501.03358, as a C-ABI CUDA library
(librk.so, include/rk.h) with a thin Python binding.

Importing the package is cheap; ``Context``/``Problem`` load librk.so on
first use and raise if it has not been built (there is no CPU fallback)."""

__all__ = ["Context", "Problem", "solve_batch", "build"]


def build(force: bool = False) -> str:
    from .build import build as _b
    return _b(force=force)


def __getattr__(name):
    if name in ("Context", "Problem", "solve_batch"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
