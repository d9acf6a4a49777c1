"""Build and load the oracle's C loops (test infrastructure only).

Compiled with gcc -O2 -fopenmp -ffp-contract=off so that the only fused
multiply-adds are the explicit fma() calls of stencil.c.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_stencil.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile stencil.c into oracle/_build/liboracle_stencil.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            i64, p = ctypes.c_int64, ctypes.c_void_p
            for name, extra in (("oracle_apply_prec", 2), ("oracle_apply", 1), ("oracle_residual", 2)):
                fn = getattr(L, name)
                fn.restype = None
                fn.argtypes = [i64, i64, i64, p, ctypes.c_int, p] + [p] * (extra + 1)
            L.oracle_apply_prec_f32.restype = None
            L.oracle_apply_prec_f32.argtypes = [i64, i64, i64, p, ctypes.c_int, p, p, p, p]
            L.oracle_jacobi_inverse.restype = None
            L.oracle_jacobi_inverse.argtypes = [i64, p, p]
            L.oracle_apply_f32.restype = None
            L.oracle_apply_f32.argtypes = [i64, i64, i64, p, ctypes.c_int, p, p, ctypes.c_int, p, p]
            L.oracle_schwarz_jacobi_f32.restype = None
            L.oracle_schwarz_jacobi_f32.argtypes = [i64, i64, i64, p, ctypes.c_int, p, p, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, p, p]
            L.oracle_schwarz_jacobi.restype = None
            L.oracle_schwarz_jacobi.argtypes = [i64, i64, i64, p, ctypes.c_int, p, p, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, p, p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c64(a):
    a = np.asarray(a, dtype=np.float64)
    return a if a.flags["C_CONTIGUOUS"] else np.ascontiguousarray(a)


class Stencil:
    """Banded operator on a grid, evaluated by the C loops."""

    def __init__(self, grid, coef):
        self.grid = grid
        self.coef = _c64(coef)
        self.S = int(self.coef.shape[0])
        self.n = grid.n
        assert self.coef.shape == (self.S, self.n)
        self._per = np.array([1 if p else 0 for p in grid.periodic], dtype=np.uint8)
        self.dinv = np.empty(self.n)
        lib().oracle_jacobi_inverse(self.n, _ptr(self.coef), _ptr(self.dinv))

    def _dims(self):
        g = self.grid
        return g.nx, g.ny, g.nz, _ptr(self._per), self.S, _ptr(self.coef)

    def apply_prec(self, v):
        v = _c64(v)
        w = np.empty(self.n)
        lib().oracle_apply_prec(*self._dims(), _ptr(self.dinv), _ptr(v), _ptr(w))
        return w

    def apply_prec_f32(self, v):
        """The mixed-precision inner operator A32 M32^{-1} v (FP32 arithmetic)."""
        v = _c64(v)
        w = np.empty(self.n)
        lib().oracle_apply_prec_f32(*self._dims(), _ptr(self.dinv), _ptr(v), _ptr(w))
        return w

    def apply(self, x):
        x = _c64(x)
        w = np.empty(self.n)
        lib().oracle_apply(*self._dims(), _ptr(x), _ptr(w))
        return w

    def residual(self, b, x):
        b = _c64(b)
        x = _c64(x)
        r = np.empty(self.n)
        lib().oracle_residual(*self._dims(), _ptr(b), _ptr(x), _ptr(r))
        return r

    def minv(self, v):
        """M^{-1} v with M = diag(A): one rounding per element."""
        return self.dinv * v

    # the "Jacobi preconditioner" of Sec. 2.1 (see oracle_schwarz_jacobi)
    SCHWARZ_BOX = (16, 8, 8)
    SCHWARZ_OVERLAP = 1
    SCHWARZ_SWEEPS = 5
    SCHWARZ_OMEGA = 2.0 / 3.0

    def schwarz(self, r, box=None, overlap=None, sweeps=None, omega=None):
        """z = M^{-1} r for the sub-domain damped-Jacobi preconditioner
        (parameters default to the class constants)."""
        r = _c64(r)
        z = np.empty(self.n)
        bx, by, bz = self.SCHWARZ_BOX if box is None else box
        lib().oracle_schwarz_jacobi(*self._dims(), _ptr(self.dinv), bx, by, bz,
                                    self.SCHWARZ_OVERLAP if overlap is None else overlap,
                                    self.SCHWARZ_SWEEPS if sweeps is None else sweeps,
                                    self.SCHWARZ_OMEGA if omega is None else omega, _ptr(r), _ptr(z))
        return z

    def apply_f32(self, v, left=False):
        """The FP32 operator of the mixed precision: A32 v32, or with ``left``
        d32 .* (A32 v32) (oracle_apply_f32)."""
        v = _c64(v)
        y = np.empty(self.n)
        lib().oracle_apply_f32(*self._dims()[:6], _ptr(self.dinv), 3 if left else 1, _ptr(v), _ptr(y))
        return y

    def schwarz_f32(self, r):
        """z = M32^{-1} r: the sub-domain preconditioner restated in FP32
        (oracle_schwarz_jacobi_f32), the class constants as parameters."""
        r = _c64(r)
        z = np.empty(self.n)
        bx, by, bz = self.SCHWARZ_BOX
        lib().oracle_schwarz_jacobi_f32(*self._dims()[:6], _ptr(self.dinv), bx, by, bz, self.SCHWARZ_OVERLAP,
                                        self.SCHWARZ_SWEEPS, self.SCHWARZ_OMEGA, _ptr(r), _ptr(z))
        return z

    def left_schwarz_f32(self, v):
        """M32^{-1} (A32 v): the left-preconditioned FP32 product of the mixed precision."""
        return self.schwarz_f32(self.apply_f32(v))

    def right_schwarz_f32(self, v):
        """A32 (M32^{-1} v): the right-preconditioned FP32 product of the mixed precision."""
        return self.apply_f32(self.schwarz_f32(v))

    def apply_left(self, v):
        """M^{-1} (A v) (left preconditioning): the product, then one rounding per element."""
        return self.dinv * self.apply(v)

    def residual_left(self, b, x):
        """M^{-1} (b - A x)."""
        return self.dinv * self.residual(b, x)
