"""Python face of librk: problems, recycle spaces and solves on torch CUDA
tensors. Argument marshalling only — every step runs in librk's kernels.

Shapes: coefficients (S, N) float64; vectors (N,) float64; a recycle space
is a (k, N) float64 tensor whose row c is column c of U (so it is the N x k
column-major array the C ABI expects)."""
import ctypes

import torch

from . import native as N

_TORCH_ALLOC = None


def _torch_allocator():
    """ctypes callbacks that draw device memory from torch's caching allocator."""
    global _TORCH_ALLOC
    if _TORCH_ALLOC is None:
        def _alloc(size, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(size))
            except Exception:
                return None

        def _free(ptr, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        _TORCH_ALLOC = (N.ALLOC_FN(_alloc), N.FREE_FN(_free))
    return _TORCH_ALLOC


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _f64_cuda(t, shape=None):
    if not torch.is_tensor(t):
        t = torch.as_tensor(t)
    t = t.to(device="cuda", dtype=torch.float64).contiguous()
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Context:
    """A librk context on the current CUDA device (memory from torch)."""

    def __init__(self, use_torch_allocator: bool = True):
        self.lib = N.load()
        self._h = ctypes.c_void_p()
        if use_torch_allocator:
            a, f = _torch_allocator()
        else:
            a, f = N.ALLOC_FN(), N.FREE_FN()
        self._cb = (a, f)
        N.check(self.lib.rk_context_create(a, f, None, ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def dots(self, Q: torch.Tensor, w: torch.Tensor, stream=None) -> torch.Tensor:
        """out[q] = Q[q] . w for the rows of Q ((nq, N), row-contiguous)."""
        Q = _f64_cuda(Q)
        w = _f64_cuda(w)
        n = w.numel()
        nq = Q.shape[0] if Q.dim() == 2 else 0
        out = torch.empty(max(nq, 1), dtype=torch.float64, device="cuda")
        ld = Q.stride(0) if nq else n
        N.check(self.lib.rk_dots(self._h, n, nq, _dptr(Q), ld, _dptr(w), _dptr(out), _stream_ptr(stream)))
        return out[:nq]

    def arnoldi_dots(self, Q, p, w, precision="fp64", stream=None):
        """[Q^T p, Q^T w, p^T p, p^T w, w^T w] for Q (nq, N) row-contiguous and
        p, w (N,), by the fused inner-product kernel of one Arnoldi step that
        solves of ``precision`` ("fp64" or "df") run (rk_arnoldi_dots)."""
        p = _f64_cuda(p)
        w = _f64_cuda(w)
        n = p.numel()
        Q = _f64_cuda(Q) if Q is not None else None
        nq = Q.shape[0] if Q is not None else 0
        out = torch.empty(2 * nq + 3, dtype=torch.float64, device="cuda")
        N.check(self.lib.rk_arnoldi_dots(self._h, n, nq, _dptr(Q) if nq else None, Q.stride(0) if nq else n,
                                         _dptr(p), _dptr(w), _dptr(out),
                                         {"fp64": N.RK_FP64, "df": N.RK_DF}[precision], _stream_ptr(stream)))
        return out

    def row_gemm(self, A, B, s, P, engine=1, stream=None):
        """[A, diag(s) B] P for A (na, N), B (nb, N) row-contiguous (either may
        be None), s (N,) or None, P (na + nb, nc): the recycle-update product
        through rk_row_gemm (engine 1: tensor cores, 0: FP32 pipe, both on
        double-float copies of A and B; 2: FP64 on the operands as given). Returns
        (nc, N)."""
        n = (A if A is not None else B).shape[1]
        A = _f64_cuda(A) if A is not None else None
        B = _f64_cuda(B) if B is not None else None
        s = _f64_cuda(s, (n,)) if s is not None else None
        na = A.shape[0] if A is not None else 0
        nb = B.shape[0] if B is not None else 0
        P = _f64_cuda(P)
        nc = P.shape[1]
        Pc = P.t().contiguous()  # column-major (na + nb) x nc
        out = torch.empty((nc, n), dtype=torch.float64, device="cuda")
        N.check(self.lib.rk_row_gemm(self._h, n, na, _dptr(A) if A is not None else None, n, nb,
                                     _dptr(B) if B is not None else None, n, _dptr(s) if s is not None else None,
                                     _dptr(Pc), nc, _dptr(out), n, engine, _stream_ptr(stream)))
        return out

    def harmonic_ritz(self, G, F, k, stream=None, precision="fp64"):
        """Device harmonic Ritz selection of the recycle update (Algorithm 3): returns (QC, PU) as
        ((n+1) x knew, n x knew) tensors (see include/rk.h). precision "fp64": the
        Schur iteration in FP64; "df": in double-float."""
        G = _f64_cuda(G)
        F = _f64_cuda(F)
        n = G.shape[1]
        # column-major (n+1) x n == row-major transpose
        Gc = G.t().contiguous()
        Fc = F.t().contiguous()
        QC = torch.zeros((k, n + 1), dtype=torch.float64, device="cuda")
        PU = torch.zeros((k, n), dtype=torch.float64, device="cuda")
        kn = ctypes.c_int32()
        N.check(self.lib.rk_harmonic_ritz(self._h, n, _dptr(Gc), _dptr(Fc), k, _dptr(QC), _dptr(PU),
                                          ctypes.byref(kn), {"fp64": N.RK_FP64, "df": N.RK_DF}[precision],
                                          _stream_ptr(stream)))
        return QC[: kn.value].t(), PU[: kn.value].t()

    def close(self):
        if self._h:
            self.lib.rk_context_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """A banded operator on a structured grid with its recycle space."""

    def __init__(self, ctx: Context, grid, coef, stream=None):
        self.ctx = ctx
        self.lib = ctx.lib
        nx, ny, nz = grid.nx, grid.ny, grid.nz
        per = grid.periodic
        self.n = nx * ny * nz
        self.grid = grid
        coef = _f64_cuda(coef)
        self.S = coef.shape[0]
        if coef.shape != (self.S, self.n):
            raise ValueError("coef must be (S, N)")
        g = N.rk_grid(nx, ny, nz, (ctypes.c_uint8 * 3)(*[1 if p else 0 for p in per]), 0)
        self._h = ctypes.c_void_p()
        N.check(self.lib.rk_create_problem(ctx.handle, ctypes.byref(g), self.S, _dptr(coef), _stream_ptr(stream),
                                           ctypes.byref(self._h)))

    def apply(self, v, precond=True, stream=None, fp32=False, df=False, left=False, subdomain=None):
        """A M^{-1} v (precond), A v, M^{-1} A v (left), or with fp32 / df the
        FP32 / double-float operator (with the preconditioner) of the "mixed"
        / "df" precisions (fp32 with left: d32 .* (A32 v)). subdomain="minv":
        M^{-1} v, "left": M^{-1} A v with the sub-domain preconditioner
        ("minv_df", "left_df": its double-float variant with the double-float
        operator; "minv32", "left32": its FP32 variant with the FP32 operator)."""
        v = _f64_cuda(v, (self.n,))
        y = torch.empty_like(v)
        if subdomain is not None:
            mode = {"minv": 5, "left": 6, "minv_df": 7, "left_df": 8, "minv32": 9, "left32": 10}[subdomain]
        elif fp32 and left:
            mode = 11
        else:
            mode = 2 if fp32 else (3 if df else (4 if left else (1 if precond else 0)))
        N.check(self.lib.rk_apply(self._h, _dptr(v), _dptr(y), mode, _stream_ptr(stream)))
        return y

    def residual(self, b, x, stream=None):
        b = _f64_cuda(b, (self.n,))
        x = _f64_cuda(x, (self.n,))
        r = torch.empty_like(b)
        N.check(self.lib.rk_residual(self._h, _dptr(b), _dptr(x), _dptr(r), _stream_ptr(stream)))
        return r

    def set_recycle(self, U, C=None, stream=None):
        if U is None or (torch.is_tensor(U) and U.numel() == 0):
            N.check(self.lib.rk_set_recycle(self._h, None, None, 0, _stream_ptr(stream)))
            return
        U = _f64_cuda(U)
        k = U.shape[0]
        if U.shape != (k, self.n):
            raise ValueError("U must be (k, N)")
        Cp = None
        if C is not None:
            C = _f64_cuda(C, (k, self.n))
            Cp = _dptr(C)
        N.check(self.lib.rk_set_recycle(self._h, _dptr(U), Cp, k, _stream_ptr(stream)))

    def stats(self):
        s, k, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        N.check(self.lib.rk_problem_stats(self._h, ctypes.byref(s), ctypes.byref(k), ctypes.byref(n)))
        return dict(solves=s.value, recycle_dim=k.value, n=n.value)

    def reset(self):
        """Start a new time-step sequence: drop the recycle space and restart
        the hybrid's solve counter (rk_problem_reset)."""
        N.check(self.lib.rk_problem_reset(self._h))

    def profile(self, on: bool = True):
        """Enable (and reset) or disable per-kernel-class timing of solves."""
        N.check(self.lib.rk_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{class: {"launches", "ms", "bytes", "fma"}} accumulated since profile(True)."""
        arr = (N.rk_prof_entry * 16)()
        cnt = ctypes.c_int32()
        N.check(self.lib.rk_profile_read(self._h, arr, 16, ctypes.byref(cnt)))
        return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes, fma=arr[i].fma)
                for i in range(min(cnt.value, 16))}

    def get_recycle(self, stream=None):
        k = self.stats()["recycle_dim"]
        U = torch.empty((max(k, 1), self.n), dtype=torch.float64, device="cuda")
        C = torch.empty_like(U)
        kk = ctypes.c_int32(max(k, 1))
        N.check(self.lib.rk_get_recycle(self._h, _dptr(U), _dptr(C), ctypes.byref(kk), _stream_ptr(stream)))
        return U[: kk.value], C[: kk.value]

    def solve(self, b, x0=None, tol=1e-8, m=40, k=20, mode="rGCROT", max_matvec=2000, hybrid_switch=5,
              update_recycle=True, out=None, stream=None, check_status=False, precision="fp64", hybrid_refresh=0,
              hybrid_fallback=0, precond_side="right", precond="jacobi"):
        """Solve A x = b; returns (x, info dict). x0 defaults to 0."""
        b, out = self._bx(b, x0, out)
        prm = _params(tol, m, k, mode, max_matvec, hybrid_switch, update_recycle, precision, hybrid_refresh,
                      hybrid_fallback, precond_side, precond)
        info = N.rk_solve_info()
        rc = self.lib.rk_solve(self._h, _dptr(b), _dptr(out), ctypes.byref(prm), ctypes.byref(info),
                               _stream_ptr(stream))
        if rc not in (N.RK_OK, N.RK_E_NOT_CONVERGED, N.RK_E_BREAKDOWN) or (check_status and rc != N.RK_OK):
            N.check(rc)
        d = info.as_dict()
        d["status_name"] = N.STATUS_NAMES.get(rc, rc)
        return out, d

    def _bx(self, b, x0, out):
        b = _f64_cuda(b, (self.n,))
        if out is None:
            out = torch.zeros_like(b) if x0 is None else _f64_cuda(x0, (self.n,)).clone()
        elif x0 is not None:
            out.copy_(_f64_cuda(x0, (self.n,)))
        return b, out

    def footprint(self, tol=1e-8, m=40, k=20, mode="rGCROT", max_matvec=2000, hybrid_switch=5,
                  update_recycle=True, precision="fp64", hybrid_refresh=0, hybrid_fallback=0,
                  precond_side="right", precond="jacobi", **_):
        """Device bytes this problem will hold during and after a solve with
        these parameters (rk_problem_footprint): for admission under a memory
        budget before the first solve."""
        prm = _params(tol, m, k, mode, max_matvec, hybrid_switch, update_recycle, precision, hybrid_refresh,
                      hybrid_fallback, precond_side, precond)
        v = ctypes.c_int64()
        N.check(self.lib.rk_problem_footprint(self._h, ctypes.byref(prm), ctypes.byref(v)))
        return int(v.value)

    def memory(self) -> int:
        """Device bytes held by this problem."""
        v = ctypes.c_int64()
        N.check(self.lib.rk_problem_memory(self._h, ctypes.byref(v)))
        return int(v.value)

    def export_recycle(self, stream=None) -> torch.Tensor:
        """The stored recycle space as an opaque uint8 device tensor (exact)."""
        nb = ctypes.c_int64()
        N.check(self.lib.rk_recycle_bytes(self._h, ctypes.byref(nb)))
        buf = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
        N.check(self.lib.rk_export_recycle(self._h, _dptr(buf), ctypes.c_int64(buf.numel()), _stream_ptr(stream)))
        return buf

    def import_recycle(self, blob: torch.Tensor, stream=None):
        """Restore a space saved by export_recycle (bit-exact)."""
        blob = blob.to(device="cuda", dtype=torch.uint8).contiguous()
        N.check(self.lib.rk_import_recycle(self._h, _dptr(blob), ctypes.c_int64(blob.numel()), _stream_ptr(stream)))

    def release(self, stream=None):
        """Free the basis / recycle / workspace memory (the recycle space is
        dropped; save it with get_recycle first to restore it later)."""
        N.check(self.lib.rk_problem_release(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rk_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params(tol, m, k, mode, max_matvec, hybrid_switch, update_recycle, precision, hybrid_refresh=0,
            hybrid_fallback=0, precond_side="right", precond="jacobi"):
    prec = {"fp64": N.RK_FP64, "mixed": N.RK_MIXED, "df": N.RK_DF}[precision]
    side = {"right": 0, "left": 1}[precond_side]
    pc = {"jacobi": N.RK_PC_JACOBI, "subdomain": N.RK_PC_SUBDOMAIN}[precond]
    prm = N.rk_solve_params(float(tol), int(m), int(k), int(max_matvec), int(hybrid_switch), N.MODES[mode],
                            prec, 1 if update_recycle else 0, int(hybrid_refresh), int(hybrid_fallback), side, pc)
    if mode == "BiCGStab":
        prm.k = 0
    return prm


def solve_batch(problems, bs, outs=None, params=None, nthreads=0, stream=None, check_status=False, **kw):
    """Solve one right-hand side on each of several distinct problems
    concurrently (rk_solve_batch). ``params``: one dict of solve() keyword
    arguments per problem, or None to use ``kw`` for all. Returns (outs,
    infos); outs[i] holds x0 on entry if given (zeros otherwise). A failing
    solve is reported in its info ("status", "status_name") and does not
    raise unless ``check_status``; invalid batch arguments raise."""
    n = len(problems)
    if len(bs) != n:
        raise ValueError("one right-hand side per problem")
    outs = [None] * n if outs is None else list(outs)
    bl, xl = [], []
    for i, p in enumerate(problems):
        b, x = p._bx(bs[i], None, outs[i])
        bl.append(b)
        xl.append(x)
    plist = params if params is not None else [kw] * n
    defaults = dict(tol=1e-8, m=40, k=20, mode="rGCROT", max_matvec=2000, hybrid_switch=5, update_recycle=True,
                    precision="fp64", hybrid_refresh=0, hybrid_fallback=0, precond_side="right", precond="jacobi")
    prm = (N.rk_solve_params * n)()
    for i in range(n):
        d = dict(defaults, **plist[i])
        prm[i] = _params(d["tol"], d["m"], d["k"], d["mode"], d["max_matvec"], d["hybrid_switch"],
                         d["update_recycle"], d["precision"], d["hybrid_refresh"], d["hybrid_fallback"],
                         d["precond_side"], d["precond"])
    infos = (N.rk_solve_info * n)()
    H = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
    B = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bl])
    X = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xl])
    lib = problems[0].lib if n else N.load()
    rc = lib.rk_solve_batch(H, B, X, ctypes.c_int32(n), prm, infos, ctypes.c_int32(nthreads), _stream_ptr(stream))
    per_problem = rc != N.RK_OK and any(infos[i].status == rc for i in range(n))
    if (rc != N.RK_OK and not per_problem) or (check_status and rc != N.RK_OK):
        N.check(rc)  # a batch-level error (bad arguments), or any failure when asked
    out_infos = []
    for i in range(n):
        d = infos[i].as_dict()
        d["status_name"] = N.STATUS_NAMES.get(infos[i].status, infos[i].status)
        out_infos.append(d)
    return xl, out_infos
