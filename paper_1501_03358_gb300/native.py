"""ctypes binding of librk (include/rk.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. If the shared library
is missing, importing this module raises: there is no CPU fallback."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librk.so")

RK_OK = 0
RK_E_INVALID = 1
RK_E_OOM = 2
RK_E_NOT_CONVERGED = 3
RK_E_BREAKDOWN = 4
RK_E_RECYCLE_INVARIANT = 5
RK_E_DEVICE_TIMEOUT = 6
RK_E_CUDA = 7
STATUS_NAMES = {0: "RK_OK", 1: "RK_E_INVALID", 2: "RK_E_OOM", 3: "RK_E_NOT_CONVERGED", 4: "RK_E_BREAKDOWN",
                5: "RK_E_RECYCLE_INVARIANT", 6: "RK_E_DEVICE_TIMEOUT", 7: "RK_E_CUDA"}

RK_GMRES, RK_RGCROT, RK_RBICGSTAB, RK_HYBRID = 0, 1, 2, 3
MODES = {"GMRES": RK_GMRES, "rGCROT": RK_RGCROT, "rBiCGStab": RK_RBICGSTAB, "BiCGStab": RK_RBICGSTAB,
         "hybrid": RK_HYBRID}
RK_FP64, RK_MIXED, RK_DF = 0, 1, 2
RK_PC_JACOBI, RK_PC_SUBDOMAIN = 0, 1

# Every exported symbol that include/rk.h declares.
EXPORTS = ("rk_last_error", "rk_version", "rk_context_create", "rk_context_destroy", "rk_create_problem",
           "rk_problem_destroy", "rk_set_recycle", "rk_get_recycle", "rk_solve", "rk_apply", "rk_residual",
           "rk_dots", "rk_problem_stats", "rk_profile_enable", "rk_profile_read", "rk_harmonic_ritz",
           "rk_dots_noalloc", "rk_row_gemm", "rk_solve_batch", "rk_problem_memory", "rk_problem_release",
           "rk_problem_reset", "rk_fp64_fma_rate", "rk_arnoldi_dots", "rk_problem_wait_limit",
           "rk_problem_footprint",
           "rk_recycle_bytes", "rk_export_recycle", "rk_import_recycle")


class rk_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_uint8 * 3), ("reserved", ctypes.c_uint8)]


class rk_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("m", ctypes.c_int32), ("k", ctypes.c_int32),
                ("max_matvec", ctypes.c_int32), ("hybrid_switch", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("update_recycle", ctypes.c_int32), ("hybrid_refresh", ctypes.c_int32),
                ("hybrid_fallback", ctypes.c_int32), ("precond_side", ctypes.c_int32),
                ("precond", ctypes.c_int32)]


class rk_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("mode_used", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("cycles_or_iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("recycle_dim", ctypes.c_int32),
                ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double), ("model_bytes", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rk_prof_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("fma", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


class RKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load librk.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librk.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    L = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.rk_last_error.restype = ctypes.c_char_p
    L.rk_version.restype = ctypes.c_char_p
    L.rk_context_create.argtypes = [ALLOC_FN, FREE_FN, vp, ctypes.POINTER(vp)]
    L.rk_context_destroy.argtypes = [vp]
    L.rk_context_destroy.restype = None
    L.rk_create_problem.argtypes = [vp, ctypes.POINTER(rk_grid), i32, vp, vp, ctypes.POINTER(vp)]
    L.rk_problem_destroy.argtypes = [vp]
    L.rk_problem_destroy.restype = None
    L.rk_set_recycle.argtypes = [vp, vp, vp, i32, vp]
    L.rk_get_recycle.argtypes = [vp, vp, vp, ctypes.POINTER(i32), vp]
    L.rk_solve.argtypes = [vp, vp, vp, ctypes.POINTER(rk_solve_params), ctypes.POINTER(rk_solve_info), vp]
    L.rk_apply.argtypes = [vp, vp, vp, i32, vp]
    L.rk_residual.argtypes = [vp, vp, vp, vp, vp]
    L.rk_dots.argtypes = [vp, i64, i32, vp, i64, vp, vp, vp]
    L.rk_problem_stats.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.rk_problem_reset.argtypes = [vp]
    L.rk_problem_footprint.argtypes = [vp, ctypes.POINTER(rk_solve_params), ctypes.POINTER(i64)]
    L.rk_problem_wait_limit.argtypes = [vp, i32, vp]
    L.rk_fp64_fma_rate.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    L.rk_arnoldi_dots.argtypes = [vp, i64, i32, vp, i64, vp, vp, vp, i32, vp]
    L.rk_profile_enable.argtypes = [vp, i32]
    L.rk_harmonic_ritz.argtypes = [vp, i32, vp, vp, i32, vp, vp, ctypes.POINTER(i32), i32, vp]
    L.rk_dots_noalloc.argtypes = [i64, i32, vp, i64, vp, vp, vp]
    L.rk_row_gemm.argtypes = [vp, i64, i32, vp, i64, i32, vp, i64, vp, vp, i32, vp, i64, i32, vp]
    L.rk_profile_read.argtypes = [vp, ctypes.POINTER(rk_prof_entry), i32, ctypes.POINTER(i32)]
    for name in EXPORTS:
        if name not in ("rk_context_destroy", "rk_problem_destroy", "rk_last_error", "rk_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(code: int):
    if code != RK_OK:
        raise RKError(code, load().rk_last_error().decode())
    return code


def last_error() -> str:
    return load().rk_last_error().decode()
