"""Oracle Krylov solvers: plain, slow, FP64, step by step (test infrastructure).

Each solver follows one of the paper's algorithms in its order and notation,
with N-length products evaluated by the C loops of stencil.c (through
``Stencil``) and NumPy dot products / axpys, and the small dense problems by
NumPy/SciPy LAPACK. Readings of the paper that this module takes:

* Preconditioning is point Jacobi M = diag(A) applied from the right for
  every solver, so every residual below is the true residual b - A x.
* Convergence is tested relative to ||b||; GMRES(m) and rGCROT stop a cycle
  at the first step whose least-squares residual estimate |g_{j+1}| meets the
  tolerance (the in-cycle estimate of the note under Algorithm 1) and then
  recompute the true residual b - A x; another cycle runs if that is still above.
* Matrix-vector products are counted in the recurrences only (the Arnoldi
  product, and BiCGStab's two products); b - A x and the A U that forms C are not.
* Algorithm 3, the U-part of the solution update: x <- x + U z with z = -B y,
  the sign that the derivation of eq. (xm_UV_rm) gives (x_m = x_0 + V_m y + U z);
  the listing's 'x - U(R^{-1} z)' contradicts it, and with U stored as U R^{-1}
  (so that A U = C) no R appears.
* The recycle-space update uses harmonic Ritz vectors (the GCRO-DR
  selection named in the title of Algorithm 3), after every cycle; see
  ``harmonic_ritz_update``.
* The projection of the initial residual onto C (xi = C^T r, r <- r - C xi, x <- x + U xi) is
  applied at the top of every cycle, not only the first. In exact arithmetic
  the true residual at the end of a cycle is already orthogonal to the updated C (it is
  W_hat times a vector orthogonal to range(G)), so the iterates are
  unchanged; in floating point its C-component is amplified by every update
  (by about 30x per cycle on the 5^3 convection-diffusion problem), which
  breaks v_1 ⟂ C (eq. V_perp_C) within a few cycles.
* BiCGStab's shadow residual is r~ = r_0 (the note under Algorithm 2), taken
  after the projection of the initial residual in Algorithm 4.
"""
import numpy as np
import scipy.linalg as sla

from ._clib import Stencil

OK = 0
NOT_CONVERGED = 1
BREAKDOWN = 2


def _info(status, matvecs, cycles, restarts, relres_true, relres_est, hist, kdim=0):
    return dict(status=status, matvecs=matvecs, cycles=cycles, restarts=restarts,
                relres_true=relres_true, relres_est=relres_est, history=hist, recycle_dim=kdim)


def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0, a
    r = np.hypot(a, b)
    return a / r, b / r, r


class _Prec:
    """The preconditioner M of a solve: "jacobi" = diag(A) (point Jacobi,
    Sec. 2.1 reading R5) or "schwarz" = the sub-domain damped-Jacobi
    preconditioner of Sec. 2.1 (Stencil.schwarz). left(v) = M^{-1} A v,
    right(v) = A M^{-1} v."""

    def __init__(self, op, kind="jacobi"):
        if kind not in ("jacobi", "schwarz"):
            raise ValueError(kind)
        self.op, self.kind = op, kind

    def minv(self, v):
        return self.op.minv(v) if self.kind == "jacobi" else self.op.schwarz(v)

    def left(self, v):
        return self.op.apply_left(v) if self.kind == "jacobi" else self.op.schwarz(self.op.apply(v))

    def right(self, v):
        return self.op.apply_prec(v) if self.kind == "jacobi" else self.op.apply(self.op.schwarz(v))

    def resid_left(self, b, x):
        return self.op.residual_left(b, x) if self.kind == "jacobi" else self.op.schwarz(self.op.residual(b, x))


def _stop_test(left, op, b, x, rho, tolp, toltrue):
    """The stop test of GMRES and rGCROT (Sec. 4: the L2 norm of the
    residual, ||b - A x|| <= tol ||b||). Right preconditioning: the cycle's
    residual is the true one. Left: the cycles work on
    M^{-1}(b - A x) with the target tolp; the true residual decides, and when
    the preconditioned target is met but the true residual is not, the target
    is scaled down by the observed shortfall. Returns (converged, tolp,
    ||b - A x|| or None)."""
    if not left:
        return rho <= tolp, tolp, None
    rt = float(np.linalg.norm(op.residual(b, x)))
    if rt <= toltrue:
        return True, tolp, rt
    if rho <= tolp:
        tolp = rho * (toltrue / rt)
    return False, tolp, rt


class _LS:
    """Progressive Givens QR of the (j+1) x j Hessenberg matrix and rotated rhs
    (Algorithms 1 and 3: y = argmin || e_1 rho - H y ||)."""

    def __init__(self, m, rho):
        self.R = np.zeros((m + 1, m))
        self.g = np.zeros(m + 1)
        self.g[0] = rho
        self.cs = np.zeros(m)
        self.sn = np.zeros(m)

    def add_column(self, j, h):
        """h = H[0:j+2, j]; returns |g_{j+1}| (the residual-norm estimate)."""
        h = h.copy()
        for i in range(j):
            t = self.cs[i] * h[i] + self.sn[i] * h[i + 1]
            h[i + 1] = -self.sn[i] * h[i] + self.cs[i] * h[i + 1]
            h[i] = t
        c, s, r = _givens(h[j], h[j + 1])
        self.cs[j], self.sn[j] = c, s
        h[j], h[j + 1] = r, 0.0
        self.R[: j + 2, j] = h[: j + 2]
        self.g[j + 1] = -s * self.g[j]
        self.g[j] = c * self.g[j]
        return abs(self.g[j + 1])

    def solve(self, jj):
        return sla.solve_triangular(self.R[:jj, :jj], self.g[:jj], lower=False)


def _op(grid_or_op, coef=None):
    if isinstance(grid_or_op, Stencil):
        return grid_or_op
    return Stencil(grid_or_op, coef)


# --------------------------------------------------------------------------- GMRES(m)
def gmres(op, b, x0=None, tol=1e-8, m=30, max_matvec=2000, keep_cycle=False, left=False, prec="jacobi"):
    """GMRES(m), Algorithm 1, right-preconditioned by M = diag(A).

    Arnoldi with modified Gram-Schmidt on A M^{-1}; solution
    update x <- x + M^{-1} V_j y; true residual b - A x after every cycle.
    With ``left``, preconditioned from the left as Sec. 2.1 states it:
    Arnoldi on M^{-1} A, x <- x + V_j y, the cycles' target on
    ||M^{-1}(b - A x)|| starting at tol ||M^{-1} b||, and the stop test on
    ||b - A x|| <= tol ||b|| (_stop_test). ``prec``: "jacobi" (point Jacobi) or "schwarz" (the
    sub-domain preconditioner of Sec. 2.1, left side only)."""
    P = _Prec(op, prec)
    if prec != "jacobi" and not left:
        raise ValueError("the sub-domain preconditioner is applied from the left for GMRES")
    n = op.n
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bnorm_true = float(np.linalg.norm(b))
    if bnorm_true == 0.0:
        return np.zeros(n), _info(OK, 0, 0, 0, 0.0, 0.0, [])
    bnorm = float(np.linalg.norm(P.minv(b))) if left else bnorm_true
    resid = P.resid_left if left else op.residual
    prod = P.left if left else op.apply_prec
    r = resid(b, x)
    rho = float(np.linalg.norm(r))
    matvecs = cycles = 0
    hist = [rho / bnorm]
    est = rho / bnorm
    last = None
    tolp, toltrue = tol * bnorm, tol * bnorm_true
    conv, tolp, rt = _stop_test(left, op, b, x, rho, tolp, toltrue)
    while not conv and matvecs < max_matvec:
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        V[0] = r / rho
        ls = _LS(m, rho)
        jj = 0
        for j in range(m):
            w = prod(V[j])
            matvecs += 1
            for l in range(j + 1):
                H[l, j] = V[l] @ w
                w = w - V[l] * H[l, j]
            H[j + 1, j] = np.linalg.norm(w)
            happy = H[j + 1, j] == 0.0
            if not happy:
                V[j + 1] = w / H[j + 1, j]
            e = ls.add_column(j, H[: j + 2, j])
            est = e / bnorm
            jj = j + 1
            if e <= tolp or happy or matvecs >= max_matvec:
                break
        y = ls.solve(jj)
        x = x + (V[:jj].T @ y if left else op.minv(V[:jj].T @ y))
        r = resid(b, x)
        rho = float(np.linalg.norm(r))
        cycles += 1
        hist.append(rho / bnorm)
        if keep_cycle:
            last = dict(V=V[: jj + 1].copy(), H=H[: jj + 1, :jj].copy(), y=y)
        conv, tolp, rt = _stop_test(left, op, b, x, rho, tolp, toltrue)
    st = OK if conv else NOT_CONVERGED
    rel = rt / bnorm_true if left else rho / bnorm
    info = _info(st, matvecs, cycles, 0, rel, est, hist)
    if keep_cycle:
        info["last_cycle"] = last
    return x, info


# --------------------------------------------------------------------------- recycle space helpers
def recycle_from_u(op, U, left=False, prec="jacobi"):
    """Forming C from U (Algorithms 3 and 4): C~ = A U, thin QR C~ = C R; return (U R^{-1}, C) so A U = C.
    With ``left``: C~ = M^{-1} A U, so M^{-1} A U = C."""
    P = _Prec(op, prec)
    Ct = np.stack([(P.left(u) if left else op.apply(u)) for u in U.T], axis=1)
    Q, R = np.linalg.qr(Ct)
    Unew = sla.solve_triangular(R, U.T, trans="T", lower=False).T  # U R^{-1}
    return Unew, Q


def harmonic_ritz_update(op, U, C, V, B, H, jj, k, return_theta=False, left=False):
    """Recycle-space update of Algorithm 3: new recycle space from harmonic Ritz vectors.

    W = [U, M^{-1} V_j] (x-space) and W_hat = [C, V_{j+1}] satisfy
    A W = W_hat G with G = [[I, B], [0, H_j]] (the augmented Arnoldi relation,
    eq. aug-arnoldi-rec). Harmonic Ritz pairs of A M^{-1} with respect to
    range(M W) solve G^T G p = theta G^T F p, F = W_hat^T M W =
    [[C^T M U, 0], [V_{j+1}^T M U, [I; 0]]]. The eigenvectors of the k
    smallest |theta| (a complex pair enters as [Re p, Im p]; a pair split by
    the cut is dropped; infinite theta never selected) form P; with
    G P = Q R' (thin QR), C <- W_hat Q and U <- W P R'^{-1}, which keeps
    A U = C and C^T C = I. With ``left`` (Arnoldi on M^{-1} A): W = [U, V_j],
    F = W_hat^T W, and the update keeps M^{-1} A U = C."""
    n = op.n
    kc = 0 if U is None else U.shape[1]
    nn = kc + jj
    G = np.zeros((nn + 1, nn))
    F = np.zeros((nn + 1, nn))
    if kc:
        G[:kc, :kc] = np.eye(kc)
        G[:kc, kc:] = B[:kc, :jj]
        MU = U if left else U * op.coef[0][:, None]
        F[:kc, :kc] = C.T @ MU
        F[kc:, :kc] = V[: jj + 1] @ MU
    G[kc:, kc:] = H[: jj + 1, :jj]
    F[kc:kc + jj, kc:] = np.eye(jj)
    A_ = G.T @ G
    B_ = G.T @ F
    ab, vr = sla.eig(A_, B_, right=True, left=False, homogeneous_eigvals=True)
    alpha, beta = ab[0], ab[1]
    with np.errstate(divide="ignore", invalid="ignore"):
        theta = alpha / beta
    mag = np.abs(theta)
    mag[~np.isfinite(mag)] = np.inf
    order = np.lexsort((np.imag(theta) < 0, np.real(theta), mag))
    kk = min(k, nn)
    cols = []
    used = set()
    for idx in order:
        if len(cols) >= kk or not np.isfinite(mag[idx]):
            break
        if idx in used:
            continue
        if abs(np.imag(theta[idx])) > 0:
            if len(cols) + 2 > kk:
                break
            v = vr[:, idx]
            cols.append(np.real(v))
            cols.append(np.imag(v))
            # the conjugate partner is the nearest remaining eigenvalue to conj(theta)
            rest = [i for i in order if i != idx and i not in used]
            partner = min(rest, key=lambda i: abs(theta[i] - np.conj(theta[idx])))
            used.add(idx)
            used.add(partner)
        else:
            cols.append(np.real(vr[:, idx]))
            used.add(idx)
    if not cols:
        return (U, C, theta) if return_theta else (U, C)
    P = np.stack(cols, axis=1)
    Q, Rp = np.linalg.qr(G @ P)
    What = np.concatenate([C, V[: jj + 1].T], axis=1) if kc else V[: jj + 1].T
    Vx = V[:jj].T if left else op.dinv[:, None] * V[:jj].T
    Wx = np.concatenate([U, Vx], axis=1) if kc else Vx
    Cn = What @ Q
    Un = Wx @ sla.solve_triangular(Rp, P.T, trans="T", lower=False).T  # W P R'^{-1}
    return (Un, Cn, theta) if return_theta else (Un, Cn)


# --------------------------------------------------------------------------- rGCROT(m,k)
def rgcrot(op, b, x0=None, tol=1e-8, m=30, k=10, U=None, C=None, update=True, max_matvec=2000,
           keep_cycle=False, left=False, prec="jacobi"):
    """rGCROT(m,k), Algorithm 3, right-preconditioned by M = diag(A).

    U, C are N x k_cur arrays (or None) with A U = C, C^T C = I; if only U is
    given, C is formed from it (recycle_from_u). Returns (x, U, C, info).
    With ``left`` (Sec. 2.1's side): Arnoldi on M^{-1} A, M^{-1} A U = C,
    x <- x + V_j y + U z, the cycles' target on ||M^{-1}(b - A x)|| starting
    at tol ||M^{-1} b||, and the stop test on ||b - A x|| <= tol ||b||
    (_stop_test).
    ``prec``: "jacobi" or "schwarz" (the latter from the left only)."""
    P = _Prec(op, prec)
    if prec != "jacobi" and not left:
        raise ValueError("the sub-domain preconditioner is applied from the left for rGCROT")
    n = op.n
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bnorm_true = float(np.linalg.norm(b))
    if U is not None and U.shape[1] == 0:
        U = C = None
    if U is not None and C is None:
        U, C = recycle_from_u(op, U, left, prec)
    kc = 0 if U is None else U.shape[1]
    if bnorm_true == 0.0:
        return np.zeros(n), U, C, _info(OK, 0, 0, 0, 0.0, 0.0, [], kc)
    bnorm = float(np.linalg.norm(P.minv(b))) if left else bnorm_true
    resid = P.resid_left if left else op.residual
    prod = P.left if left else op.apply_prec
    rhat = resid(b, x)                            # initial residual
    if kc:
        xi = C.T @ rhat                           # projection onto C
        r = rhat - C @ xi
        x = x + U @ xi
    else:
        r = rhat
    rho = float(np.linalg.norm(r))
    matvecs = cycles = 0
    hist = [rho / bnorm]
    est = rho / bnorm
    last = None
    first = True
    tolp, toltrue = tol * bnorm, tol * bnorm_true
    conv, tolp, rt = _stop_test(left, op, b, x, rho, tolp, toltrue)
    while not conv and matvecs < max_matvec:            # outer loop
        if kc and not first:
            # the projection onto C again: v_1 must be orthogonal to the (updated) C for
            # eq. V_perp_C; the true residual is only orthogonal to it
            # up to rounding, and each recycle update amplifies the drift.
            xi = C.T @ r
            r = r - C @ xi
            x = x + U @ xi
            rho = float(np.linalg.norm(r))
        first = False
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        Bm = np.zeros((max(kc, 1), m))
        V[0] = r / rho                                  # v_1 = r / ||r||
        ls = _LS(m, rho)
        jj = 0
        for j in range(m):                              # Arnoldi steps
            w = prod(V[j])                              # w = A M^{-1} v_j (left: M^{-1} A v_j)
            matvecs += 1
            for l in range(kc):                         # B column: w <- w - C C^T w
                Bm[l, j] = C[:, l] @ w
                w = w - C[:, l] * Bm[l, j]
            for l in range(j + 1):                      # modified Gram-Schmidt against V_j
                H[l, j] = V[l] @ w
                w = w - V[l] * H[l, j]
            H[j + 1, j] = np.linalg.norm(w)             # h_{j+1,j} = ||w||
            happy = H[j + 1, j] == 0.0
            if not happy:
                V[j + 1] = w / H[j + 1, j]
            e = ls.add_column(j, H[: j + 2, j])
            est = e / bnorm
            jj = j + 1
            if e <= tolp or happy or matvecs >= max_matvec:
                break
        y = ls.solve(jj)                                # least squares for y
        x = x + (V[:jj].T @ y if left else op.minv(V[:jj].T @ y))   # x <- x + M^{-1} V_j y
        if kc:
            z = -Bm[:kc, :jj] @ y                       # z = -B y
            x = x + U @ z                               # x <- x + U z
        r = resid(b, x)                                 # true residual
        rho = float(np.linalg.norm(r))
        cycles += 1
        hist.append(rho / bnorm)
        if keep_cycle:
            last = dict(V=V[: jj + 1].copy(), H=H[: jj + 1, :jj].copy(), B=Bm[:kc, :jj].copy(),
                        C=None if C is None else C.copy(), U=None if U is None else U.copy(), y=y, jj=jj)
        if update and k > 0:                            # recycle-space update
            U, C = harmonic_ritz_update(op, U, C, V, Bm, H, jj, k, left=left)
            kc = 0 if U is None else U.shape[1]
        conv, tolp, rt = _stop_test(left, op, b, x, rho, tolp, toltrue)
    st = OK if conv else NOT_CONVERGED
    rel = rt / bnorm_true if left else rho / bnorm
    info = _info(st, matvecs, cycles, 0, rel, est, hist, kc)
    if keep_cycle:
        info["last_cycle"] = last
    return x, U, C, info


# --------------------------------------------------------------------------- BiCGStab
def bicgstab(op, b, x0=None, tol=1e-8, max_matvec=2000, prec="jacobi"):
    """BiCGStab, Algorithm 2, right-preconditioned: the iterates p, s live in
    the preconditioned space and x = x_0 + M^{-1} (sum of alpha p + omega s).
    ``prec``: "jacobi" or "schwarz" (Sec. 2.1's sub-domain preconditioner)."""
    P = _Prec(op, prec)
    n = op.n
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), _info(OK, 0, 0, 0, 0.0, 0.0, [])
    r = op.residual(b, x)                               # initial residual
    rt = r.copy()                                       # r~ = r_0
    xt = np.zeros(n)
    matvecs = it = 0
    hist = [np.linalg.norm(r) / bnorm]
    status = NOT_CONVERGED
    p = v = None
    alpha = omega = rho_old = 0.0
    while np.linalg.norm(r) > tol * bnorm and matvecs < max_matvec:  # iteration
        rho = rt @ r                                    # rho = (r~, r)
        if rho == 0.0:                                  # breakdown test
            status = BREAKDOWN
            break
        if it == 0:                                     # first search direction
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = P.right(p)                                  # v = A M^{-1} p
        matvecs += 1
        alpha = rho / (rt @ v)                          # alpha
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:            # early exit on ||s||
            xt = xt + alpha * p
            r = s
            it += 1
            hist.append(np.linalg.norm(r) / bnorm)
            break
        t = P.right(s)                                  # t = A M^{-1} s
        matvecs += 1
        tt = t @ t
        if tt == 0.0:
            status = BREAKDOWN
            break
        omega = (t @ s) / tt                            # omega
        xt = xt + alpha * p + omega * s                 # x~ update
        r = s - omega * t                               # r update
        rho_old = rho                                   # keep rho
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        if omega == 0.0:
            status = BREAKDOWN
            break
    x = x + P.minv(xt)
    rtrue = op.residual(b, x)
    rel = float(np.linalg.norm(rtrue)) / bnorm
    if status != BREAKDOWN:
        status = OK if rel <= tol else NOT_CONVERGED
    return x, _info(status, matvecs, it, 0, rel, float(np.linalg.norm(r)) / bnorm, hist)


# --------------------------------------------------------------------------- rBiCGStab
def _rbicgstab_pass(op, b, x, tol, U, C, max_matvec, bnorm, callback=None, prec="jacobi"):
    """One run of Algorithm 4 from x_hat = x; returns (x, matvecs, its,
    breakdown, updated-residual norm, history)."""
    P = _Prec(op, prec)
    n = op.n
    kc = 0 if C is None else C.shape[1]
    rhat = op.residual(b, x)                            # initial residual
    if kc:
        eta1 = C.T @ rhat                               # projection onto C
        r = rhat - C @ eta1
        xi = -eta1
    else:
        r = rhat
        xi = np.zeros(0)
    rt = r.copy()                                       # shadow residual r~ = r_0
    xt = np.zeros(n)
    matvecs = it = 0
    hist = []
    brk = False
    p = v = None
    alpha = omega = rho_old = 0.0
    while np.linalg.norm(r) > tol * bnorm and matvecs < max_matvec:   # iteration
        rho = rt @ r                                    # rho = (r~, r)
        if abs(rho) <= 1e-14 * np.linalg.norm(rt) * np.linalg.norm(r):   # breakdown test
            brk = True
            break
        if it == 0:                                     # first search direction
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = P.right(p)                                  # v = A M^{-1} p
        matvecs += 1
        if kc:
            eta1 = C.T @ v                              # eta1 = C^T v
            v = v - C @ eta1
        rtv = rt @ v
        if rtv == 0.0:
            brk = True
            break
        alpha = rho / rtv                               # alpha
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:            # early exit on ||s||
            xt = xt + alpha * p                         # x~ update
            r = s
            if kc:
                xi = xi + alpha * eta1                  # postponed U coefficient
            it += 1
            hist.append(np.linalg.norm(r) / bnorm)
            break
        t = P.right(s)                                  # t = A M^{-1} s
        matvecs += 1
        if kc:
            eta2 = C.T @ t                              # eta2 = C^T t
            t = t - C @ eta2
        tt = t @ t
        if tt == 0.0:
            brk = True
            break
        omega = (t @ s) / tt                            # omega
        if kc:
            xi = xi + alpha * eta1 + omega * eta2       # postponed U coefficient
        xt = xt + alpha * p + omega * s                 # x~ update
        r = s - omega * t                               # r update
        rho_old = rho                                   # keep rho
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        if callback is not None:
            callback(r)
        if omega == 0.0:
            brk = True
            break
    if callback is not None:
        callback(r)
    x = x + P.minv(xt)                                  # x = x_hat + M^{-1} x~, then the postponed U part
    if kc:
        x = x - U @ xi
    return x, matvecs, it, brk, float(np.linalg.norm(r)), hist


def rbicgstab(op, b, x0=None, tol=1e-8, U=None, C=None, max_matvec=2000, max_restarts=3, callback=None,
              prec="jacobi"):
    """rBiCGStab with one recycle space, Algorithm 4, right-preconditioned.

    When the updated residual meets the tolerance the postponed U update is
    folded in and the true residual b - A x is checked; if it is
    above the tolerance, or on breakdown, Algorithm 4 restarts from the
    current x (at most ``max_restarts`` times)."""
    n = op.n
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    bnorm = float(np.linalg.norm(b))
    if U is not None and U.shape[1] == 0:
        U = C = None
    if U is not None and C is None:
        U, C = recycle_from_u(op, U)                    # forming C from U
    kc = 0 if U is None else U.shape[1]
    if bnorm == 0.0:
        return np.zeros(n), _info(OK, 0, 0, 0, 0.0, 0.0, [], kc)
    matvecs = its = restarts = 0
    hist = []
    status = NOT_CONVERGED
    upd = np.inf
    while True:
        x, mv, it, brk, upd, h = _rbicgstab_pass(op, b, x, tol, U, C, max_matvec - matvecs, bnorm, callback, prec)
        matvecs += mv
        its += it
        hist += h
        rel = float(np.linalg.norm(op.residual(b, x))) / bnorm
        if rel <= tol:
            status = OK
            break
        if matvecs >= max_matvec:
            status = NOT_CONVERGED
            break
        if restarts >= max_restarts:
            status = BREAKDOWN if brk else NOT_CONVERGED
            break
        restarts += 1
    return x, _info(status, matvecs, its, restarts, rel, upd / bnorm, hist, kc)


# --------------------------------------------------------------------------- sequence drivers
class RecyclingSequence:
    """Solves a sequence A x_t = b_t carrying the recycle space (U, C) across
    steps (Sec. 1, Sec. 2.3). mode: 'GMRES', 'rGCROT', 'BiCGStab',
    'rBiCGStab' or 'hybrid' (rGCROT with recycle update for the first
    ``hybrid_switch`` steps, then rBiCGStab with U, C frozen; Sec. 2.4).

    The two variants Sec. 2.4 mentions, in this reading: ``refresh`` = R > 0
    runs every R-th solve after the switch with rGCROT ("intermittent solves
    with rGCROT to update the recycle space"); ``fallback`` = F > 0 stops an
    rBiCGStab solve that breaks down or has used F matrix-vector products
    without converging, finishes it with rGCROT from its current iterate
    (within ``max_matvec`` in total) and starts a new rGCROT phase with that
    solve ("if convergence is poor ... switch back to rGCROT").

    ``left``: GMRES and rGCROT preconditioned from the left (Sec. 2.1); the
    carried pair then satisfies M^{-1} A U = C, and a solve on the other
    side (rBiCGStab is always right-preconditioned) first re-forms C from U
    for its operator (recycle_from_u)."""

    def __init__(self, op, mode="rGCROT", m=30, k=10, tol=1e-8, hybrid_switch=5, max_matvec=2000, refresh=0,
                 fallback=0, left=False, prec="jacobi"):
        self.op, self.mode, self.m, self.k, self.tol = op, mode, m, k, tol
        self.prec = prec
        self.hybrid_switch, self.max_matvec = hybrid_switch, max_matvec
        self.refresh, self.fallback, self.left = refresh, fallback, left
        self.U = self.C = None
        self.side = False  # side of the carried pair: False A U = C, True M^{-1} A U = C
        self.t = 0
        self.base = 0  # first solve of the current rGCROT phase (hybrid)

    def _side(self, left):
        if self.U is not None and self.U.shape[1] > 0 and self.side != left:
            self.U, self.C = recycle_from_u(self.op, self.U, left, self.prec)
        self.side = left

    def solve(self, b, x0=None):
        mode = self.mode
        if mode == "hybrid":
            t = self.t - self.base
            refresh = self.refresh > 0 and t >= self.hybrid_switch and \
                (t - self.hybrid_switch + 1) % self.refresh == 0
            mode = "rGCROT" if (t < self.hybrid_switch or refresh) else "rBiCGStab"
            if mode == "rBiCGStab" and self.fallback > 0:
                cap = min(self.fallback, self.max_matvec)
                self._side(False)
                x, info = rbicgstab(self.op, b, x0, self.tol, self.U, self.C, cap, prec=self.prec)
                if info["status"] != OK and info["matvecs"] < self.max_matvec:
                    used = info["matvecs"]
                    self._side(self.left)
                    x, self.U, self.C, ig = rgcrot(self.op, b, x, self.tol, self.m, self.k, self.U, self.C,
                                                   update=True, max_matvec=self.max_matvec - used, left=self.left,
                                                   prec=self.prec)
                    ig["matvecs"] += used
                    ig["restarts"] += info["restarts"]
                    info = ig
                    mode = "rGCROT"
                    self.base = self.t
                info["mode"] = mode
                self.t += 1
                return x, info
        if mode == "GMRES":
            x, info = gmres(self.op, b, x0, self.tol, self.m, self.max_matvec, left=self.left, prec=self.prec)
        elif mode == "rGCROT":
            self._side(self.left)
            x, self.U, self.C, info = rgcrot(self.op, b, x0, self.tol, self.m, self.k, self.U, self.C,
                                             update=True, max_matvec=self.max_matvec, left=self.left, prec=self.prec)
        elif mode == "BiCGStab":
            x, info = bicgstab(self.op, b, x0, self.tol, self.max_matvec, prec=self.prec)
        elif mode == "rBiCGStab":
            self._side(False)
            x, info = rbicgstab(self.op, b, x0, self.tol, self.U, self.C, self.max_matvec, prec=self.prec)
        else:
            raise ValueError(mode)
        info["mode"] = mode
        self.t += 1
        return x, info
