"""GPU path (librk through its C ABI) against the CPU oracle.

Bars (element by element on the same seeded inputs):
* structured-grid products A M^{-1} v, A v, b - A x: bit-exact (same band
  order of fused multiply-adds on both sides);
* block inner products: |d - d_ref| <= 1e-13 ||Q_q|| ||w|| (normwise);
* solves: ||b - A x|| / ||b|| <= tol; ||x - x_oracle|| <= max(1e-6, 2 kappa
  tol) ||x_oracle|| (two solutions that both meet the tolerance can differ by
  up to kappa(A) tol, so 1e-6 is only attainable when kappa tol is below it);
  matrix-vector products within +-2 of the oracle's, widened to the oracle's
  own spread when rounding-level (1e-14 relative) perturbations of b move the
  oracle's count by more than that. Restarted GMRES over many cycles is
  chaotic under rounding (GPU and oracle x agree to 1e-13 after one cycle of
  GMRES(40) on the 12^3 channel and the gap then grows about tenfold per
  cycle while both residual histories agree to six digits), so long runs are
  checked in lock step over their first five cycles and only for convergence
  and a count within 25% over the whole solve. The GPU orthogonalises by
  classical Gram-Schmidt with reorthogonalisation in double-float arithmetic,
  the oracle by modified Gram-Schmidt in FP64;
* recycle spaces: compared as subspaces (||C C^T - C' C'^T||_2), never column
  by column, plus A U = C and C^T C = I.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from problems import Grid, make_config, random_operator, porous_skew_19pt
from problems.operators import sphere_pack
from problems.fields import rng_for
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_1501_03358_gb300 import Context
    c = Context()
    yield c
    c.close()


def gpu_problem(ctx, grid, coef):
    from paper_1501_03358_gb300 import Problem
    return Problem(ctx, grid, torch.from_numpy(np.ascontiguousarray(coef)))


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


GRIDS = [
    ((37, 11, 5), (False, False, False)),
    ((32, 8, 9), (True, False, True)),
    ((33, 9, 7), (True, True, True)),
    ((1, 1, 1), (False, False, False)),
    ((2, 3, 4), (True, True, False)),
    ((64, 17, 3), (False, True, False)),
]


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", GRIDS)
def test_stencil_bit_exact(ctx, S, dims, per):
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(g.n)
    b = rng.standard_normal(g.n)
    y1 = prob.apply(t(v), precond=True).cpu().numpy()
    y2 = prob.apply(t(v), precond=False).cpu().numpy()
    r = prob.residual(t(b), t(v)).cpu().numpy()
    assert np.array_equal(y1, op.apply_prec(v))
    assert np.array_equal(y2, op.apply(v))
    assert np.array_equal(r, op.residual(b, v))


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", GRIDS[:4])
def test_fp32_operator_bit_exact(ctx, S, dims, per):
    """The mixed-precision inner operator (A11) matches the oracle's FP32
    restatement bit for bit."""
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims, 32)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    v = np.random.default_rng(5).standard_normal(g.n)
    assert np.array_equal(prob.apply(t(v), fp32=True).cpu().numpy(), op.apply_prec_f32(v))


def df_operator_bound(g, coef, v):
    """Elementwise bound for the double-float operator: every input (bands,
    1/a_pp, v) is rounded to double-float (relative 2^-48), z = v / a_pp and
    each band product lose at most a few units of 2^-48, and the lazy
    accumulation (renormalised every 8 bands) adds at most S + 1 more; the FP64
    oracle's own error is S 2^-53. (S + 8) 2^-46 sum_s |c_s| |z_s| covers all
    of these with room to spare."""
    S = coef.shape[0]
    z = np.abs(v / coef[0])
    return (S + 8) * 2.0 ** -46 * oracle.Stencil(g, np.abs(coef)).apply(z)


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", GRIDS[:4])
def test_df_operator_within_rounding_bound(ctx, S, dims, per):
    """The double-float operator of the "df" precision (bands and 1/a_pp
    rounded to double-float once, double-float products and accumulation in
    band order) against the FP64 oracle, element by element."""
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims, 48)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    v = np.random.default_rng(6).standard_normal(g.n)
    got = prob.apply(t(v), df=True).cpu().numpy()
    ref = op.apply_prec(v)
    assert np.all(np.abs(got - ref) <= df_operator_bound(g, coef, v))
    assert np.any(got != ref)  # it is not the FP64 operator


@pytest.mark.parametrize("n,nq", [(1, 1), (1000, 3), (4099, 17), (100003, 40), (262144, 61)])
def test_block_dots(ctx, n, nq):
    rng = np.random.default_rng(n + nq)
    Q = rng.standard_normal((nq, n))
    Q[0] *= 1e-3
    w = rng.standard_normal(n)
    got = ctx.dots(t(Q), t(w)).cpu().numpy()
    ref = np.array([math.fsum(Q[q] * w) for q in range(nq)])  # exactly rounded products' sum
    bound = 1e-13 * np.linalg.norm(Q, axis=1) * np.linalg.norm(w)
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("n,nq", [(1, 1), (1000, 3), (4099, 17), (100003, 40), (262144, 61), (2 ** 21, 61),
                                  (3001, 0), (777, 128)])
def test_arnoldi_dots_against_exact_sums(ctx, n, nq, precision):
    """The hot path's fused Arnoldi inner products [Q^T p, Q^T w, p^T p,
    p^T w, w^T w] (the kernel the solvers run at every step: FP64 for the
    fp64 and mixed precisions, double-float for df) against sums of the
    exactly rounded products (math.fsum), element by element, at the
    normwise bar of single dot products: |d - d_ref| <= 1e-13 ||a|| ||b||.
    Sizes from one row to 2^21 rows (the row ranges of 152 blocks), 0 to
    128 columns, a ragged tail, and columns scaled over six decades."""
    rng = np.random.default_rng(n + 7 * nq)
    Q = rng.standard_normal((nq, n)) * np.exp2(rng.integers(-10, 10, size=(nq, 1)))
    pv = rng.standard_normal(n)
    w = rng.standard_normal(n) * 1e3
    got = ctx.arnoldi_dots(t(Q) if nq else None, t(pv), t(w), precision=precision).cpu().numpy()
    pairs = [(Q[q], pv) for q in range(nq)] + [(Q[q], w) for q in range(nq)] + [(pv, pv), (pv, w), (w, w)]
    ref = np.array([math.fsum(a * b) for a, b in pairs])
    bound = np.array([1e-13 * np.linalg.norm(a) * np.linalg.norm(b) for a, b in pairs])
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


@pytest.mark.parametrize("n,nq", [(2, 1), (64, 5), (130, 62), (4096, 20), (100002, 41), (262144, 61),
                                  (2 ** 21, 62), (1000000, 33)])
def test_arnoldi_dots_tensor_core_engine(ctx, n, nq, monkeypatch):
    """The FP64 fused Arnoldi inner products on the tensor cores (exact
    digit products of 56-bit truncations per 32-row block, 128-bit integer
    running sums) against sums of exactly rounded products: within
    1e-14 ||a|| ||b|| (tighter than the FP64-pipe kernel's bar; the engine is
    selected by RK_TC_DOTS=1; below 32 rows the FP64-pipe kernel serves),
    with the FP64-pipe kernel (RK_TC_DOTS=0, the default) on the same
    operands within its own bar. Sizes from one 32-row block (a single
    block, a ragged tail) to hundreds of blocks per SM (every buffer reused
    many times); operands: column scales over six decades, a zero column, a
    column of mixed-sign values spanning 2^-40..2^40 within each block."""
    rng = np.random.default_rng(n + 11 * nq)
    Q = rng.standard_normal((nq, n)) * np.exp2(rng.integers(-10, 10, size=(nq, 1)))
    if nq >= 3:
        Q[1] = 0.0
        Q[2] = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, size=n))
    pv = rng.standard_normal(n)
    w = rng.standard_normal(n) * 1e3
    pairs = [(Q[q], pv) for q in range(nq)] + [(Q[q], w) for q in range(nq)] + [(pv, pv), (pv, w), (w, w)]
    ref = np.array([math.fsum(a * b) for a, b in pairs])
    scale = np.array([np.linalg.norm(a) * np.linalg.norm(b) for a, b in pairs])
    monkeypatch.setenv("RK_TC_DOTS", "1")
    got = ctx.arnoldi_dots(t(Q), t(pv), t(w), precision="fp64").cpu().numpy()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-14 * scale), float(np.max(err / np.maximum(scale, 1e-300)))
    if nq >= 3:
        assert got[1] == 0.0 and got[nq + 1] == 0.0
    monkeypatch.setenv("RK_TC_DOTS", "0")
    got64 = ctx.arnoldi_dots(t(Q), t(pv), t(w), precision="fp64").cpu().numpy()
    assert np.all(np.abs(got64 - ref) <= 1e-13 * scale)


@pytest.mark.parametrize("engine", [1, 0, 2, 3])
@pytest.mark.parametrize("n,na,nb,nc,scaled", [
    (1, 3, 2, 2, False), (127, 20, 41, 20, True), (129, 61, 0, 20, False), (1000, 20, 40, 20, True),
    (5003, 0, 64, 32, True), (4099, 32, 32, 7, False), (300, 1, 0, 2, False), (70000, 20, 41, 20, True),
    (70001, 20, 41, 20, True)])
def test_row_gemm_recycle_update(ctx, engine, n, na, nb, nc, scaled):
    """[A, diag(s) B] P (the recycle-update product) against an exact
    reference, element by element. FP32-pipe engine (double-float products,
    lazy accumulation over up to 128 terms): |out - X P| <= 2^-44 (|X| |P|).
    Tensor-core engine: the inputs rounded to double-float (2^-48 |X|), a
    double-float epilogue, and the fixed-point digits, which truncate each
    element below 2^-56 of its row's (X) or column's (P) largest:
    |out - X P| <= 2^-45 (|X| |P|) + 2^-52 K max_row|X| max_col|P|.
    FP64 engine: K fused multiply-adds per output and one rounded product
    s_i b_iq: |out - X P| <= (K + 2) 2^-53 (|X| |P|). Tensor-core engine on
    FP64 operands (the fp64 and mixed recycle update): s_i b_iq rounded
    once, each element truncated below 2^-56 of 2^E_r (< 2^-55 of its row's
    largest), P's seven digits to 2^-57 of 2^F_c, digit levels above 8
    dropped, one final rounding: |out - X P| <= 2^-51 (|X| |P|) +
    2^-50 K max_row|X| max_col|P|.
    Scales within a row and within a column of P span 2^8. 70000 rows
    span hundreds of tiles per block (bulk-copied tiles prefetched one
    ahead, then a ragged last tile); 70001 rows give operands the bulk copy
    cannot take (odd leading dimension: every tile loaded by the threads)."""
    rng = np.random.default_rng(n * 131 + na * 7 + nb + nc)
    A = rng.standard_normal((na, n)) * np.exp2(rng.integers(-4, 5, size=(na, 1))) if na else None
    B = rng.standard_normal((nb, n)) if nb else None
    sv = np.exp(rng.standard_normal(n)) if scaled else None
    P = rng.standard_normal((na + nb, nc)) * np.exp2(rng.integers(-4, 5, size=(na + nb, nc)))
    X = np.concatenate([m for m in (A, None if B is None else (B * sv if scaled else B)) if m is not None], axis=0)
    if scaled:
        # the B part of the reference with the row scale applied exactly
        Xl = np.concatenate([m.astype(np.longdouble) for m in (A,) if m is not None] +
                            [B.astype(np.longdouble) * sv.astype(np.longdouble)], axis=0)
    else:
        Xl = X.astype(np.longdouble)
    ref = (Xl.T @ P.astype(np.longdouble)).T
    got = ctx.row_gemm(None if A is None else t(A), None if B is None else t(B), None if sv is None else t(sv),
                       t(P), engine=engine).cpu().numpy()
    comp = (np.abs(X).T @ np.abs(P)).T
    if engine == 1:
        K = na + nb
        bound = 2.0 ** -45 * comp + 2.0 ** -52 * K * np.abs(P).max(axis=0)[:, None] * np.abs(X).max(axis=0)[None, :]
    elif engine == 2:
        bound = (na + nb + 2) * 2.0 ** -53 * comp
    elif engine == 3:
        K = na + nb
        bound = 2.0 ** -51 * comp + 2.0 ** -50 * K * np.abs(P).max(axis=0)[:, None] * np.abs(X).max(axis=0)[None, :]
    else:
        bound = 2.0 ** -44 * comp
    err = np.abs((got.astype(np.longdouble) - ref).astype(np.float64))
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))


@pytest.mark.parametrize("engine", [1, 3])
def test_row_gemm_tensor_engine_limits(ctx, engine):
    from paper_1501_03358_gb300.native import RKError
    A = t(np.ones((65, 64)))
    with pytest.raises(RKError):
        ctx.row_gemm(A, None, None, t(np.ones((65, 4))), engine=engine)
    with pytest.raises(RKError):
        ctx.row_gemm(t(np.ones((4, 64))), None, None, t(np.ones((4, 33))), engine=engine)


_KAPPA = {}


def kappa(grid, coef):
    key = (grid, coef.tobytes()[:4096], coef.shape)
    if key not in _KAPPA:
        _KAPPA[key] = float(np.linalg.cond(oracle.dense_matrix(grid, coef)))
    return _KAPPA[key]


def perturbed(b, seed):
    return b * (1.0 + 1e-14 * np.random.default_rng(seed).standard_normal(b.size))


def mv_slack(run, b, base):
    """+-2, or twice the spread of the oracle's own counts over three
    rounding-level perturbations of b when that is larger (three samples
    underestimate the spread of a chaotic count)."""
    counts = [base] + [run(perturbed(b, s))["matvecs"] for s in (1, 2, 3)]
    return max(2, 2 * (max(counts) - min(counts))), counts


def check_solve(op, b, xg, info, xo, io, tol, slack=2, kap=None):
    rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
    assert rel <= tol * 1.0000001, (rel, info)
    assert info["status"] == 0, info
    xtol = 1e-6 if kap is None else max(1e-6, 2.0 * kap * tol)
    assert np.linalg.norm(xg - xo) <= xtol * np.linalg.norm(xo), (np.linalg.norm(xg - xo) / np.linalg.norm(xo), xtol)
    assert abs(info["matvecs"] - io["matvecs"]) <= slack, (info["matvecs"], io["matvecs"], slack)


def subspace_gap(C1, C2):
    """||C1 C1^T - C2 C2^T||_2 for N x k bases: the sine of the largest
    principal angle, computed as ||(I - Q1 Q1^T) Q2||_2 (accurate for small
    angles)."""
    q1 = np.linalg.qr(C1)[0]
    q2 = np.linalg.qr(C2)[0]
    return float(np.linalg.norm(q2 - q1 @ (q1.T @ q2), 2))


@pytest.mark.parametrize("cfg_id,size,m", [(1, 12, 30), (2, 12, 40), (1, 10, 7), (1, 8, 200)])
def test_gmres_parity(ctx, cfg_id, size, m):
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    x, info = prob.solve(t(b), tol=1e-8, m=m, k=0, mode="GMRES", max_matvec=8000)
    xo, io = oracle.gmres(op, b, tol=1e-8, m=m, max_matvec=8000)
    kap = kappa(cfg.grid, cfg.coef)
    if io["cycles"] <= 5:
        check_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, 2, kap)
        return
    # lock step over the first five cycles
    x5, i5 = prob.solve(t(b), tol=1e-14, m=m, k=0, mode="GMRES", max_matvec=5 * m)
    xo5, io5 = oracle.gmres(op, b, tol=1e-14, m=m, max_matvec=5 * m)
    assert i5["matvecs"] == io5["matvecs"] == 5 * m
    assert np.linalg.norm(x5.cpu().numpy() - xo5) <= 1e-9 * np.linalg.norm(xo5)
    # the whole solve: converged, x within the kappa bound, count within 25%
    check_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, max(2, int(0.25 * io["matvecs"])), kap)


@pytest.mark.parametrize("cfg_id,size,m,k,steps", [(1, 12, 30, 10, 5), (2, 12, 40, 20, 4), (1, 9, 6, 4, 4)])
def test_rgcrot_sequence_parity(ctx, cfg_id, size, m, k, steps):
    """rGCROT(m,k) over a sequence of right-hand sides with the recycle space
    carried across steps (Algorithm 3, recycle update after every cycle)."""
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    kap = kappa(cfg.grid, cfg.coef)
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=m, k=k, tol=1e-8, max_matvec=5000)
    for s in range(steps):
        b = cfg.rhs(s)
        x, info = prob.solve(t(b), tol=1e-8, m=m, k=k, mode="rGCROT", max_matvec=5000)
        U0, C0 = seq.U, seq.C
        xo, io = seq.solve(b)
        slack = 2
        if io["cycles"] > 3:
            run = lambda bb: oracle.rgcrot(op, bb, tol=1e-8, m=m, k=k, U=U0, C=C0, max_matvec=5000)[3]
            slack, _ = mv_slack(run, b, io["matvecs"])
        check_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kap)
        U, C = prob.get_recycle()
        U, C = U.cpu().numpy().T, C.cpu().numpy().T
        assert U.shape[1] == seq.U.shape[1] == info["recycle_dim"]
        A_U = np.stack([op.apply(u) for u in U.T], axis=1)
        assert np.linalg.norm(A_U - C) <= 1e-10 * np.linalg.norm(C) * max(1.0, np.abs(cfg.coef).max())
        assert np.linalg.norm(C.T @ C - np.eye(C.shape[1])) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("cfg_id,size,m,k", [(1, 10, 12, 6), (2, 10, 20, 8), (1, 8, 30, 10)])
def test_harmonic_ritz_cycles_match_oracle(ctx, cfg_id, size, m, k, precision):
    """Recycle space after one and after two cycles (updated by harmonic Ritz
    vectors, computed on the device) spans the oracle's (SciPy eig of the
    pencil) to within rounding-level principal angles."""
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    U = C = None
    for cyc in range(2):
        prob.solve(t(b), tol=1e-14, m=m, k=k, mode="rGCROT", max_matvec=m, precision=precision)
        _, U, C, _ = oracle.rgcrot(op, b, tol=1e-14, m=m, k=k, U=U, C=C, max_matvec=m)
        Ug, Cg = prob.get_recycle()
        Cg = Cg.cpu().numpy().T
        assert Cg.shape == C.shape
        assert subspace_gap(Cg, C) <= 1e-6, (cyc, subspace_gap(Cg, C))


def test_full_size_first_cycles_lock_step(ctx):
    """At the 128^3 channel size, in the benchmark's launch configuration
    (2,097,152 rows: 1188-block inner products, the 152-block persistent
    tensor-core recycle update over 16,384 row tiles): rGCROT(40,20) with
    point Jacobi, one cycle from an empty recycle space (a GMRES(40) cycle,
    then the harmonic Ritz update) and one cycle with the 20-column space it
    built, GPU against the oracle.

    Bound for x: both sides minimise the same residual over Krylov bases that
    differ by orthogonalisation rounding (CGS2 against MGS), a relative
    perturbation of about m sqrt(N) u ~ 1e-11 (u = 2^-53), amplified by the
    condition of the small least-squares problem of one cycle (about 10 here:
    the first cycle cuts the residual by less than 10x), so 1e-9 relative
    holds with margin. The recycle spaces are compared as subspaces; the
    second cycle's x depends only on span(C) (A U = C fixes U from it), so
    its bar is 1e-9 plus the subspace gap."""
    cfg = make_config(2)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    U = C = None
    gap = 0.0
    for cyc in range(2):
        x, info = prob.solve(t(b), tol=1e-14, m=40, k=20, mode="rGCROT", max_matvec=40, precision="fp64")
        xo, U, C, io = oracle.rgcrot(op, b, tol=1e-14, m=40, k=20, U=U, C=C, max_matvec=40)
        assert info["matvecs"] == io["matvecs"] == 40
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) <= (1e-9 + 10 * gap) * np.linalg.norm(xo), cyc
        assert abs(info["relres_true"] - io["relres_true"]) <= 1e-8 * io["relres_true"], cyc
        Ug, Cg = prob.get_recycle()
        Cg = Cg.cpu().numpy().T
        assert Cg.shape == C.shape == (cfg.n, 20)
        gap = subspace_gap(Cg, C)
        assert gap <= 1e-6, (cyc, gap)


def test_recycle_set_get_roundtrip_and_forming_c(ctx):
    cfg = make_config(1, size=10)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    _, U, C, _ = oracle.rgcrot(op, cfg.rhs(0), tol=1e-10, m=10, k=6)
    kk = U.shape[1]  # 6, or 5 when the cut falls inside a conjugate pair
    # C given: stored as is (FP64 store: bit for bit)
    prob.set_recycle(t(U.T), t(C.T))
    U2, C2 = prob.get_recycle()
    assert np.array_equal(U2.cpu().numpy(), U.T) and np.array_equal(C2.cpu().numpy(), C.T)
    # after a df solve the store is double-float (to ~48 significant bits)
    prob.solve(t(cfg.rhs(1)), tol=1e-8, m=10, k=6, mode="rGCROT", update_recycle=False, precision="df")
    U2, C2 = prob.get_recycle()
    assert np.all(np.abs(U2.cpu().numpy() - U.T) <= 2.0 ** -46 * np.abs(U.T))
    assert np.all(np.abs(C2.cpu().numpy() - C.T) <= 2.0 ** -46 * np.abs(C.T))
    # and back to FP64 by the next fp64 solve (the conversion rounds once)
    prob.solve(t(cfg.rhs(1)), tol=1e-8, m=10, k=6, mode="rGCROT", update_recycle=False)
    U3, C3 = prob.get_recycle()
    assert np.array_equal(U3.cpu().numpy(), U2.cpu().numpy()) and np.array_equal(C3.cpu().numpy(), C2.cpu().numpy())
    prob.set_recycle(t(U.T), t(C.T))
    # C omitted: the library forms C = orth(A U) and rescales U so that A U = C
    Uraw = U @ np.diag([1.0, 2.0, -3.0, 0.5, 4.0, 1.5][:kk])
    prob.set_recycle(t(Uraw.T))
    U3, C3 = prob.get_recycle()
    U3, C3 = U3.cpu().numpy().T, C3.cpu().numpy().T
    # range(A U) equals range(C) only as far as the oracle's own A U = C holds
    A_Uo = np.stack([op.apply(u) for u in U.T], axis=1)
    assert subspace_gap(C3, C) <= 2.0 * np.linalg.norm(A_Uo - C, 2) + 1e-12
    A_U = np.stack([op.apply(u) for u in U3.T], axis=1)
    assert np.linalg.norm(A_U - C3) <= 1e-11 * np.linalg.norm(C3) * np.abs(cfg.coef).max()
    assert np.linalg.norm(C3.T @ C3 - np.eye(kk)) <= 1e-12
    # an inconsistent pair is refused
    from paper_1501_03358_gb300.native import RKError, RK_E_RECYCLE_INVARIANT
    with pytest.raises(RKError) as e:
        prob.set_recycle(t(U.T), t((C * 1.01).T))
    assert e.value.code == RK_E_RECYCLE_INVARIANT


@pytest.mark.parametrize("with_space", [False, True])
def test_rbicgstab_parity(ctx, with_space):
    cfg = make_config(1, size=14)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    U = C = None
    if with_space:
        _, U, C, _ = oracle.rgcrot(op, cfg.rhs(0), tol=1e-9, m=20, k=8)
        prob.set_recycle(t(U.T), t(C.T))
    b = cfg.rhs(2)
    x, info = prob.solve(t(b), tol=1e-8, k=8 if with_space else 0, mode="rBiCGStab", max_matvec=3000)
    xo, io = oracle.rbicgstab(op, b, tol=1e-8, U=U, C=C, max_matvec=3000)
    run = lambda bb: oracle.rbicgstab(op, bb, tol=1e-8, U=U, C=C, max_matvec=3000)[1]
    slack, _ = mv_slack(run, b, io["matvecs"])
    check_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kappa(cfg.grid, cfg.coef))


def test_hybrid_sequence_porous(ctx):
    """Hybrid (Sec. 2.4) on a small skewed porous problem (19 points): rGCROT
    for the first steps, then rBiCGStab with the recycle space frozen."""
    n = (14, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(77, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=4000)
    base = np.random.default_rng(5).standard_normal(grid.n)
    for s in range(4):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=4000)
        xo, io = seq.solve(b)
        assert info["mode_used"] == (1 if s < 2 else 2)
        slack = 2
        rel = np.linalg.norm(op.residual(b, x.cpu().numpy())) / np.linalg.norm(b)
        assert rel <= 1e-8 and info["status"] == 0
        xtol = max(1e-6, 2.0 * kap * 1e-8)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= xtol * np.linalg.norm(xo)
        if io["matvecs"] > 2 * slack:
            U0, C0 = (seq.U, seq.C)
            run = (lambda bb: oracle.rbicgstab(op, bb, tol=1e-8, U=U0, C=C0, max_matvec=4000)[1]) if s >= 2 else None
            if run is not None:
                slack = max(slack, mv_slack(run, b, io["matvecs"])[0])
        assert abs(info["matvecs"] - io["matvecs"]) <= slack, (s, info["matvecs"], io["matvecs"])


@pytest.mark.parametrize("refresh,fallback", [(2, 0), (0, 6), (3, 6)])
def test_hybrid_variants_match_oracle(ctx, refresh, fallback):
    """The hybrid variants of Sec. 2.4 on the small porous problem: rGCROT
    refresh solves every `refresh` solves after the switch, and the switch
    back to rGCROT when rBiCGStab has not converged after `fallback`
    products. Per solve: the same mode as the oracle's schedule (a fallback
    solve reports rGCROT), convergence on the true residual, x within the
    kappa bound of the oracle's, products within 25% (a fallback solve's
    rGCROT part starts from an rBiCGStab iterate, which moves the count)."""
    n = (14, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(77, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=4000,
                                   refresh=refresh, fallback=fallback)
    base = np.random.default_rng(5).standard_normal(grid.n)
    code = {"rGCROT": 1, "rBiCGStab": 2}
    fell_back = 0
    for s in range(6):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=4000,
                             hybrid_refresh=refresh, hybrid_fallback=fallback)
        base_before = seq.base
        xo, io = seq.solve(b)
        fell_back += int(seq.base != base_before)
        assert info["mode_used"] == code[io["mode"]], (s, info["mode_used"], io["mode"])
        xg = x.cpu().numpy()
        rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
        assert rel <= 1e-8 and info["status"] == 0, (s, info)
        assert np.linalg.norm(xg - xo) <= max(1e-6, 2.0 * kap * 1e-8) * np.linalg.norm(xo)
        assert abs(info["matvecs"] - io["matvecs"]) <= max(4, int(0.25 * io["matvecs"])), (s, info, io)
    if fallback:
        assert fell_back >= 1


# ---------------------------------------------------------------- left preconditioning (Sec. 2.1)
@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", GRIDS[:4])
def test_left_operator_bit_exact(ctx, S, dims, per):
    """M^{-1}(A v) (the product, then one rounded multiplication) bit for bit."""
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims, 9)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    v = np.random.default_rng(4).standard_normal(g.n)
    assert np.array_equal(prob.apply(t(v), left=True).cpu().numpy(), op.apply_left(v))


def check_left_solve(op, b, xg, info, xo, io, tol, slack, kap):
    """Left preconditioning: the true residual meets tol (the stop test; the
    cycles work on M^{-1}(b - A x)); relres_true is ||b - A x|| / ||b|| (to
    the rounding of forming it); x within the kappa bound of the oracle's;
    products within slack."""
    rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
    assert rel <= tol * 1.0000001 and info["status"] == 0, (rel, info)
    assert abs(rel - info["relres_true"]) <= 1e-6 * rel + 1e-15
    xtol = max(1e-6, 2.0 * kap * tol)
    assert np.linalg.norm(xg - xo) <= xtol * np.linalg.norm(xo)
    assert abs(info["matvecs"] - io["matvecs"]) <= slack, (info["matvecs"], io["matvecs"], slack)


@pytest.mark.parametrize("cfg_id,size,m", [(1, 12, 30), (2, 12, 40)])
def test_left_gmres_parity(ctx, cfg_id, size, m):
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    x, info = prob.solve(t(b), tol=1e-8, m=m, k=0, mode="GMRES", max_matvec=8000, precond_side="left")
    xo, io = oracle.gmres(op, b, tol=1e-8, m=m, max_matvec=8000, left=True)
    slack = max(2, int(0.25 * io["matvecs"])) if io["cycles"] > 5 else 2
    check_left_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kappa(cfg.grid, cfg.coef))


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("cfg_id,size,m,k,steps", [(1, 12, 30, 10, 4), (2, 12, 40, 20, 3)])
def test_left_rgcrot_sequence_parity(ctx, cfg_id, size, m, k, steps, precision):
    """Left-preconditioned rGCROT over a sequence, the recycle pair carried:
    the solve bars above, and M^{-1} A U = C, C^T C = I for the carried pair."""
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    kap = kappa(cfg.grid, cfg.coef)
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=m, k=k, tol=1e-8, max_matvec=5000, left=True)
    for s in range(steps):
        b = cfg.rhs(s)
        x, info = prob.solve(t(b), tol=1e-8, m=m, k=k, mode="rGCROT", max_matvec=5000, precond_side="left",
                             precision=precision)
        U0, C0 = seq.U, seq.C
        xo, io = seq.solve(b)
        slack = 2
        if io["cycles"] > 3:
            run = lambda bb: oracle.rgcrot(op, bb, tol=1e-8, m=m, k=k, U=U0, C=C0, max_matvec=5000, left=True)[3]
            slack, _ = mv_slack(run, b, io["matvecs"])
        check_left_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kap)
        U, C = prob.get_recycle()
        U, C = U.cpu().numpy().T, C.cpu().numpy().T
        BU = np.stack([op.apply_left(u) for u in U.T], axis=1)
        nb = np.abs(op.minv(np.ones(op.n))).max() * np.abs(cfg.coef).sum(axis=0).max()
        assert np.linalg.norm(BU - C) <= 1e-10 * np.linalg.norm(C) * max(1.0, nb)
        assert np.linalg.norm(C.T @ C - np.eye(C.shape[1])) <= 1e-11


def test_left_hybrid_converts_the_space(ctx):
    """Hybrid with left-preconditioned rGCROT for the first solves and
    right-preconditioned rBiCGStab after the switch (Sec. 2.1): the carried
    pair is re-formed for the right side at the switch (A U = C afterwards),
    and every solve meets its own criterion as the oracle's does."""
    n = (14, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(77, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=4000,
                                   left=True)
    base = np.random.default_rng(5).standard_normal(grid.n)
    for s in range(4):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=4000,
                             precond_side="left")
        xo, io = seq.solve(b)
        xg = x.cpu().numpy()
        assert info["mode_used"] == (1 if s < 2 else 2) and info["status"] == 0, (s, info)
        assert np.linalg.norm(op.residual(b, xg)) <= 1e-8 * np.linalg.norm(b) * 1.0000001
        assert np.linalg.norm(xg - xo) <= max(1e-6, 2.0 * kap * 1e-8) * np.linalg.norm(xo)
    U, C = prob.get_recycle()
    U, C = U.cpu().numpy().T, C.cpu().numpy().T
    AU = np.stack([op.apply(u) for u in U.T], axis=1)
    assert np.linalg.norm(AU - C) <= 1e-10 * np.linalg.norm(C) * np.abs(coef).max()
    qa = np.linalg.qr(U)[0]
    qb = np.linalg.qr(seq.U)[0]
    assert np.linalg.norm(qb - qa @ (qa.T @ qb), 2) <= 1e-6


def test_mixed_precision_sequence(ctx):
    """Mixed precision (A11): FP32 inner operator inside the FP64/double-float
    rGCROT recurrence with b - A x recomputed in FP64 every cycle. Every step
    reaches ||b - A x|| / ||b|| <= 1e-8 (true residual, FP64), its solution
    error against the FP64 oracle stays within the kappa bound, and the carried
    recycle space keeps A U = C (re-derived in FP64 after each solve)."""
    cfg = make_config(1, size=12)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    kap = kappa(cfg.grid, cfg.coef)
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=30, k=10, tol=1e-8, max_matvec=5000)
    for s in range(4):
        b = cfg.rhs(s)
        x, info = prob.solve(t(b), tol=1e-8, m=30, k=10, mode="rGCROT", precision="mixed", max_matvec=5000)
        xo, io = seq.solve(b)
        xg = x.cpu().numpy()
        rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
        assert info["status"] == 0 and rel <= 1e-8
        err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
        assert err <= max(1e-6, 2 * kap * 1e-8), err
        assert info["matvecs"] <= 2 * io["matvecs"] + 60
        U, C = prob.get_recycle()
        U, C = U.cpu().numpy().T, C.cpu().numpy().T
        A_U = np.stack([op.apply(u) for u in U.T], axis=1)
        assert np.linalg.norm(A_U - C) <= 1e-10 * np.linalg.norm(C) * np.abs(cfg.coef).max()


@pytest.mark.parametrize("cfg_id,size,m,k,steps", [(1, 12, 30, 10, 4), (2, 12, 40, 20, 3)])
def test_df_precision_sequence_parity(ctx, cfg_id, size, m, k, steps):
    """rGCROT(m,k) sequence with the double-float operator in the Arnoldi
    products: the same bars as the FP64 sequence (tolerance met on the FP64
    true residual, x within the kappa bound of the oracle's, matvecs within
    the oracle's own rounding-level spread) and A U = C, C^T C = I for the
    carried space."""
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    kap = kappa(cfg.grid, cfg.coef)
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=m, k=k, tol=1e-8, max_matvec=5000)
    for s in range(steps):
        b = cfg.rhs(s)
        x, info = prob.solve(t(b), tol=1e-8, m=m, k=k, mode="rGCROT", max_matvec=5000, precision="df")
        U0, C0 = seq.U, seq.C
        xo, io = seq.solve(b)
        slack = 2
        if io["cycles"] > 3:
            run = lambda bb: oracle.rgcrot(op, bb, tol=1e-8, m=m, k=k, U=U0, C=C0, max_matvec=5000)[3]
            slack, _ = mv_slack(run, b, io["matvecs"])
        check_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kap)
        U, C = prob.get_recycle()
        U, C = U.cpu().numpy().T, C.cpu().numpy().T
        A_U = np.stack([op.apply(u) for u in U.T], axis=1)
        assert np.linalg.norm(A_U - C) <= 1e-10 * np.linalg.norm(C) * max(1.0, np.abs(cfg.coef).max())
        assert np.linalg.norm(C.T @ C - np.eye(C.shape[1])) <= 1e-11


def test_df_precision_hybrid_porous(ctx):
    """The hybrid rGCROT -> rBiCGStab sequence on the porous 19-point problem
    with the double-float operator (FP64 vectors in the rBiCGStab phase)."""
    n = (14, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(77, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=4000)
    base = np.random.default_rng(5).standard_normal(grid.n)
    for s in range(4):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=4000,
                             precision="df")
        xo, io = seq.solve(b)
        xg = x.cpu().numpy()
        rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
        assert info["status"] == 0 and rel <= 1e-8, (s, info)
        assert np.linalg.norm(xg - xo) <= max(1e-6, 2 * kap * 1e-8) * np.linalg.norm(xo)


def test_mixed_precision_hybrid_porous(ctx):
    n = (14, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(77, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=4000)
    base = np.random.default_rng(5).standard_normal(grid.n)
    for s in range(4):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=4000,
                             precision="mixed")
        xo, io = seq.solve(b)
        xg = x.cpu().numpy()
        rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
        assert info["status"] == 0 and rel <= 1e-8, (s, info)
        assert np.linalg.norm(xg - xo) <= max(1e-6, 2 * kap * 1e-8) * np.linalg.norm(xo)


def test_zero_rhs_and_exact_recycling(ctx):
    cfg = make_config(1, size=8)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    x, info = prob.solve(t(np.zeros(cfg.n)), mode="rGCROT", m=10, k=4)
    assert info["matvecs"] == 0 and info["status"] == 0 and float(x.abs().max()) == 0.0
    _, U, C, _ = oracle.rgcrot(op, cfg.rhs(0), tol=1e-10, m=10, k=4)
    prob.set_recycle(t(U.T), t(C.T))
    bb = C @ np.array([1.0, -2.0, 0.5, 3.0])[: C.shape[1]]
    for mode in ("rGCROT", "rBiCGStab"):
        prob.set_recycle(t(U.T), t(C.T))
        x, info = prob.solve(t(bb), tol=1e-8, m=10, k=4, mode=mode, update_recycle=False)
        assert info["matvecs"] == 0, (mode, info)
        assert np.linalg.norm(op.residual(bb, x.cpu().numpy())) <= 1e-8 * np.linalg.norm(bb)


def test_invalid_operator_rejected(ctx):
    from paper_1501_03358_gb300.native import RKError, RK_E_INVALID
    g = Grid(4, 4, 4, (False, False, False))
    coef = random_operator(g, 7, np.random.default_rng(0))
    coef[1, 0] = 0.5  # band -x of cell (0,0,0) points out of the x=0 face
    with pytest.raises(RKError) as e:
        gpu_problem(ctx, g, coef)
    assert e.value.code == RK_E_INVALID
    coef = random_operator(g, 7, np.random.default_rng(0))
    coef[0, 5] = 0.0
    with pytest.raises(RKError):
        gpu_problem(ctx, g, coef)


def test_nan_rhs_rejected(ctx):
    from paper_1501_03358_gb300.native import RKError, RK_E_INVALID
    cfg = make_config(1, size=6)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    b[3] = np.nan
    with pytest.raises(RKError) as e:
        prob.solve(t(b))
    assert e.value.code == RK_E_INVALID


def test_not_converged_returns_last_iterate(ctx):
    cfg = make_config(1, size=12)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    x, info = prob.solve(t(b), tol=1e-12, m=5, k=0, mode="GMRES", max_matvec=10)
    assert info["status_name"] == "RK_E_NOT_CONVERGED" and info["matvecs"] == 10
    xo, io = oracle.gmres(op, b, tol=1e-12, m=5, max_matvec=10)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_full_size_channel_operator_and_solve(ctx, precision):
    """At the 128^3 channel size (the benchmark's workload and launch
    configuration): every SpMV output bit-exact against the oracle (the
    double-float operator within its rounding bound); a capped rGCROT(40,20)
    solve whose reported true residual matches the oracle's recomputation of
    ||b - A x||, whose residual history decreases, and whose recycle space
    satisfies A U = C (sampled columns, oracle products) and C^T C = I."""
    cfg = make_config(2)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    v = np.random.default_rng(1).standard_normal(cfg.n)
    if precision == "fp64":
        assert np.array_equal(prob.apply(t(v)).cpu().numpy(), op.apply_prec(v))
        assert np.array_equal(prob.apply(t(v), precond=False).cpu().numpy(), op.apply(v))
    else:
        got = prob.apply(t(v), df=True).cpu().numpy()
        assert np.all(np.abs(got - op.apply_prec(v)) <= df_operator_bound(cfg.grid, cfg.coef, v))
    b = cfg.rhs(0)
    x, info = prob.solve(t(b), tol=1e-8, m=40, k=20, mode="rGCROT", max_matvec=400, precision=precision)
    xg = x.cpu().numpy()
    assert np.all(np.isfinite(xg))
    rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
    assert info["matvecs"] == 400 and info["cycles_or_iters"] == 10
    assert abs(rel - info["relres_true"]) <= 1e-6 * rel
    assert rel < 0.1
    U, C = prob.get_recycle()
    U, C = U.cpu().numpy().T, C.cpu().numpy().T
    assert C.shape[1] >= 19
    G = C.T @ C
    assert np.linalg.norm(G - np.eye(C.shape[1])) <= 1e-10
    anorm = np.abs(cfg.coef).sum(axis=0).max()  # ||A||_inf
    for c in (0, C.shape[1] // 2, C.shape[1] - 1):
        au = op.apply(U[:, c])
        # U and C are stored in double-float (~2^-48 relative per entry)
        assert np.linalg.norm(au - C[:, c]) <= 1e-12 * anorm * np.linalg.norm(U[:, c]) + 1e-12
