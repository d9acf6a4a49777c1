"""The sub-domain Jacobi preconditioner of Sec. 2.1 on the GPU against the
oracle (Stencil.schwarz and the solvers with prec="schwarz").

Bars: M^{-1} v and M^{-1} A v bit for bit (FP64 against the oracle's FP64
form, the mixed precision's FP32 variant against its FP32 restatement) (the same FP64 operations in the
same order on both sides, over grids whose boxes have ragged tails, wrap onto
themselves on periodic axes, or are smaller than one box); solves as in
test_gpu_parity (tolerance met, x within the kappa bound of the oracle's,
matrix-vector products within the oracle's own spread under rounding-level
perturbations of b).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from problems import Grid, make_config, random_operator, porous_skew_19pt
from problems.operators import sphere_pack
from problems.fields import rng_for
import oracle
from test_gpu_parity import ctx, gpu_problem, t, kappa, mv_slack, check_solve  # noqa: F401

pytestmark = pytest.mark.gpu

SD_GRIDS = [
    ((37, 19, 11), (False, False, False)),  # ragged boxes on every axis
    ((40, 16, 17), (True, False, True)),
    ((33, 9, 7), (True, True, True)),
    ((16, 8, 8), (True, True, True)),       # one box whose grown box wraps onto itself
    ((2, 3, 4), (True, True, False)),       # smaller than one box
    ((1, 1, 1), (False, False, False)),
    ((70, 9, 20), (False, True, False)),
]


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", SD_GRIDS)
def test_subdomain_apply_bit_exact(ctx, S, dims, per):
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims, 11)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    v = np.random.default_rng(6).standard_normal(g.n)
    assert np.array_equal(prob.apply(t(v), subdomain="minv").cpu().numpy(), op.schwarz(v))
    assert np.array_equal(prob.apply(t(v), subdomain="left").cpu().numpy(), op.schwarz(op.apply(v)))


def test_subdomain_apply_full_size(ctx):
    """The 128^3 channel operator (2048 boxes): M^{-1} v and M^{-1} A v bit
    for bit over the whole field (the oracle's C loops finish in seconds)."""
    cfg = make_config(2, size=128)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    v = cfg.rhs(0)
    assert np.array_equal(prob.apply(t(v), subdomain="minv").cpu().numpy(), op.schwarz(v))
    assert np.array_equal(prob.apply(t(v), subdomain="left").cpu().numpy(), op.schwarz(op.apply(v)))


def sd_df_bound(op, coef, S, v, y, left):
    """Elementwise bar of the double-float variant against the FP64 oracle.
    One sweep z' = z + omega D^-1 (r - A_loc z) in double-float errs by at
    most (S + 12) 2^-46 (|z| + omega |D^-1| (|r| + |A| |z|)) per cell: the
    band sum within the (S + 8) 2^-46 sum |a| |z| of the double-float
    stencil, four more rounded operations, and the double-float rounding of
    the bands and 1/a_pp (2^-48 each). Later sweeps multiply an error by the
    iteration matrix I - omega D^-1 A_loc, whose infinity norm is at most
    g = max_p |1 - omega| + omega sum_{t>0} |a_t| / |a_p| (1 for diagonally
    dominant rows), and the left product adds the double-float A v. Six
    sweeps (five local and the global one): the bar is
    6 (S + 12) 2^-46 max(1, g)^6 max_p (|z| + omega |D^-1| (|r| + |A| |z|)),
    with z the oracle's result and r its right-hand side."""
    w = 2.0 / 3.0
    a0 = np.abs(coef[0])
    g = float(np.max(abs(1 - w) + w * np.abs(coef[1:]).sum(axis=0) / a0))
    r = op.apply(v) if left else v
    absA = oracle.Stencil(op.grid, np.abs(coef))
    mag = np.abs(y) + w / a0 * (np.abs(r) + absA.apply(np.abs(y)))
    if left:
        mag = mag + w / a0 * absA.apply(np.abs(v))
    return 6 * (S + 12) * 2.0 ** -46 * max(1.0, g) ** 6 * float(mag.max())


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", SD_GRIDS[:4])
def test_subdomain_df_within_bound(ctx, S, dims, per):
    """The double-float variant (precision "df") against the FP64 oracle,
    within the derived bar of sd_df_bound."""
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims, 12)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    v = np.random.default_rng(7).standard_normal(g.n)
    for mode, left in (("minv_df", False), ("left_df", True)):
        yo = op.schwarz(op.apply(v) if left else v)
        yg = prob.apply(t(v), subdomain=mode).cpu().numpy()
        err = float(np.abs(yg - yo).max())
        assert err <= sd_df_bound(op, coef, S, v, yo, left), (mode, err)


def check_sd_left(op, b, xg, info, xo, io, tol, slack, kap):
    rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
    assert rel <= tol * 1.0000001 and info["status"] == 0, (rel, info)
    assert abs(rel - info["relres_true"]) <= 1e-6 * rel + 1e-15
    assert np.linalg.norm(xg - xo) <= max(1e-6, 2.0 * kap * tol) * np.linalg.norm(xo)
    assert abs(info["matvecs"] - io["matvecs"]) <= slack, (info["matvecs"], io["matvecs"], slack)


@pytest.mark.parametrize("cfg_id,size,m", [(1, 12, 30), (2, 12, 40)])
def test_subdomain_left_gmres_parity(ctx, cfg_id, size, m):
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    b = cfg.rhs(0)
    x, info = prob.solve(t(b), tol=1e-8, m=m, k=0, mode="GMRES", max_matvec=4000, precond_side="left",
                         precond="subdomain")
    xo, io = oracle.gmres(op, b, tol=1e-8, m=m, max_matvec=4000, left=True, prec="schwarz")
    run = lambda bb: oracle.gmres(op, bb, tol=1e-8, m=m, max_matvec=4000, left=True, prec="schwarz")[1]
    slack, _ = mv_slack(run, b, io["matvecs"])
    check_sd_left(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kappa(cfg.grid, cfg.coef))


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("cfg_id,size,m,k,steps", [(1, 12, 30, 10, 3), (2, 14, 30, 10, 3)])
def test_subdomain_left_rgcrot_sequence_parity(ctx, cfg_id, size, m, k, steps, precision):
    """Left rGCROT with the sub-domain preconditioner over a sequence: the
    solve bars, and M^{-1} A U = C, C^T C = I for the carried pair."""
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    kap = kappa(cfg.grid, cfg.coef)
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=m, k=k, tol=1e-8, max_matvec=3000, left=True,
                                   prec="schwarz")
    for s in range(steps):
        b = cfg.rhs(s)
        x, info = prob.solve(t(b), tol=1e-8, m=m, k=k, mode="rGCROT", max_matvec=3000, precond_side="left",
                             precond="subdomain", precision=precision)
        U0, C0 = seq.U, seq.C
        xo, io = seq.solve(b)
        run = lambda bb: oracle.rgcrot(op, bb, tol=1e-8, m=m, k=k, U=U0, C=C0, max_matvec=3000, left=True,
                                       prec="schwarz")[3]
        slack, _ = mv_slack(run, b, io["matvecs"])
        check_sd_left(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kap)
        U, C = prob.get_recycle()
        U, C = U.cpu().numpy().T, C.cpu().numpy().T
        BU = np.stack([op.schwarz(op.apply(u)) for u in U.T], axis=1)
        assert np.linalg.norm(BU - C) <= 1e-10 * np.linalg.norm(C) * max(1.0, np.abs(cfg.coef).max())
        assert np.linalg.norm(C.T @ C - np.eye(C.shape[1])) <= 1e-11


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("with_space", [False, True])
def test_subdomain_rbicgstab_parity(ctx, with_space, precision):
    """rBiCGStab right-preconditioned with the sub-domain preconditioner:
    v = A M^{-1} p, x <- x + M^{-1} x~ (Algorithm 4)."""
    cfg = make_config(1, size=14)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    U = C = None
    if with_space:
        _, U, C, _ = oracle.rgcrot(op, cfg.rhs(0), tol=1e-9, m=20, k=8)
        prob.set_recycle(t(U.T), t(C.T))
    b = cfg.rhs(2)
    x, info = prob.solve(t(b), tol=1e-8, k=8 if with_space else 0, mode="rBiCGStab", max_matvec=3000,
                         precond="subdomain", precision=precision)
    xo, io = oracle.rbicgstab(op, b, tol=1e-8, U=U, C=C, max_matvec=3000, prec="schwarz")
    run = lambda bb: oracle.rbicgstab(op, bb, tol=1e-8, U=U, C=C, max_matvec=3000, prec="schwarz")[1]
    slack, _ = mv_slack(run, b, io["matvecs"])
    check_solve(op, b, x.cpu().numpy(), info, xo, io, 1e-8, slack, kappa(cfg.grid, cfg.coef))


def test_subdomain_hybrid_sequence(ctx):
    """Hybrid with the sub-domain preconditioner (Sec. 2.4 with Sec. 2.1's
    Jacobi preconditioner): left rGCROT for the first solves, then
    right-preconditioned rBiCGStab with the pair re-formed as A U = C."""
    n = (20, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(78, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=3000,
                                   left=True, prec="schwarz")
    base = np.random.default_rng(5).standard_normal(grid.n)
    for s in range(4):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=3000,
                             precond_side="left", precond="subdomain")
        xo, io = seq.solve(b)
        xg = x.cpu().numpy()
        assert info["mode_used"] == (1 if s < 2 else 2) and info["status"] == 0, (s, info)
        assert np.linalg.norm(op.residual(b, xg)) <= 1e-8 * np.linalg.norm(b) * 1.0000001
        assert np.linalg.norm(xg - xo) <= max(1e-6, 2.0 * kap * 1e-8) * np.linalg.norm(xo)
    U, C = prob.get_recycle()
    U, C = U.cpu().numpy().T, C.cpu().numpy().T
    AU = np.stack([op.apply(u) for u in U.T], axis=1)
    assert np.linalg.norm(AU - C) <= 1e-10 * np.linalg.norm(C) * np.abs(coef).max()


def test_subdomain_invalid_combinations(ctx):
    from paper_1501_03358_gb300.native import RKError
    cfg = make_config(1, size=8)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    b = t(cfg.rhs(0))
    for kw in (dict(mode="rGCROT", precond_side="right"), dict(mode="GMRES", precond_side="right"),
               dict(mode="hybrid", precond_side="right"), dict(mode="rGCROT", precond_side="right", precision="mixed")):
        with pytest.raises(RKError):
            prob.solve(b, precond="subdomain", check_status=True, **kw)


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("dims,per", SD_GRIDS)
def test_fp32_subdomain_apply_bit_exact(ctx, S, dims, per):
    """The FP32 variant of the mixed precision (RK_MIXED): M32^{-1} v,
    M32^{-1} (A32 v) and the left point-Jacobi FP32 product d32 .* (A32 v),
    bit for bit against the oracle's FP32 restatement (the same FP32
    operations in the same order)."""
    g = Grid(*dims, per)
    coef = random_operator(g, S, np.random.default_rng(hash((S, dims, 13)) % 2**32))
    prob = gpu_problem(ctx, g, coef)
    op = oracle.Stencil(g, coef)
    v = np.random.default_rng(7).standard_normal(g.n)
    assert np.array_equal(prob.apply(t(v), subdomain="minv32").cpu().numpy(), op.schwarz_f32(v))
    assert np.array_equal(prob.apply(t(v), subdomain="left32").cpu().numpy(), op.left_schwarz_f32(v))
    assert np.array_equal(prob.apply(t(v), fp32=True, left=True).cpu().numpy(), op.apply_f32(v, left=True))


def test_fp32_subdomain_apply_full_size(ctx):
    """The FP32 sub-domain products on the full 128^3 channel field."""
    cfg = make_config(2, size=128)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    v = cfg.rhs(0)
    assert np.array_equal(prob.apply(t(v), subdomain="minv32").cpu().numpy(), op.schwarz_f32(v))
    assert np.array_equal(prob.apply(t(v), subdomain="left32").cpu().numpy(), op.left_schwarz_f32(v))


def check_mixed(op, b, xg, info, xo, tol, kap):
    """Mixed-precision solve bars against the FP64 oracle: the FP64 true
    residual meets the tolerance (residual replacement) and x lies within the
    kappa bound of the oracle's solution; the product count of an inexact
    operator is not held to the FP64 one."""
    rel = np.linalg.norm(op.residual(b, xg)) / np.linalg.norm(b)
    assert rel <= tol * 1.0000001 and info["status"] == 0, (rel, info)
    assert abs(rel - info["relres_true"]) <= 1e-6 * rel + 1e-15
    assert np.linalg.norm(xg - xo) <= max(1e-6, 2.0 * kap * tol) * np.linalg.norm(xo)


@pytest.mark.parametrize("precond", ["subdomain", "jacobi"])
@pytest.mark.parametrize("cfg_id,size,m,k,steps", [(1, 12, 30, 10, 3), (2, 14, 30, 10, 3)])
def test_mixed_left_rgcrot_sequence(ctx, cfg_id, size, m, k, steps, precond):
    """Mixed precision from the left (Sec. 2.1's side for GMRES-type
    solvers): the FP32 operator and the FP32 preconditioner (sub-domain
    sweeps or point Jacobi) inside the FP64 recurrence, the true residual
    recomputed in FP64 every cycle; per step the bars of check_mixed against
    the FP64 oracle, and M^{-1} A U = C (re-derived in FP64) for the carried
    pair."""
    cfg = make_config(cfg_id, size=size)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    kap = kappa(cfg.grid, cfg.coef)
    pk = "schwarz" if precond == "subdomain" else "jacobi"
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=m, k=k, tol=1e-8, max_matvec=3000, left=True, prec=pk)
    for s in range(steps):
        b = cfg.rhs(s)
        x, info = prob.solve(t(b), tol=1e-8, m=m, k=k, mode="rGCROT", max_matvec=3000, precond_side="left",
                             precond=precond, precision="mixed")
        xo, io = seq.solve(b)
        check_mixed(op, b, x.cpu().numpy(), info, xo, 1e-8, kap)
        U, C = prob.get_recycle()
        U, C = U.cpu().numpy().T, C.cpu().numpy().T
        left = (lambda u: op.schwarz(op.apply(u))) if precond == "subdomain" else op.apply_left
        BU = np.stack([left(u) for u in U.T], axis=1)
        assert np.linalg.norm(BU - C) <= 1e-10 * np.linalg.norm(C) * max(1.0, np.abs(cfg.coef).max())
        assert np.linalg.norm(C.T @ C - np.eye(C.shape[1])) <= 1e-11


@pytest.mark.parametrize("with_space", [False, True])
def test_mixed_subdomain_rbicgstab(ctx, with_space):
    """rBiCGStab right-preconditioned with the FP32 sub-domain sweeps and the
    FP32 operator in the recurrence; M^{-1} x~ and the true residual in
    FP64."""
    cfg = make_config(1, size=14)
    prob = gpu_problem(ctx, cfg.grid, cfg.coef)
    op = oracle.Stencil(cfg.grid, cfg.coef)
    U = C = None
    if with_space:
        _, U, C, _ = oracle.rgcrot(op, cfg.rhs(0), tol=1e-9, m=20, k=8)
        prob.set_recycle(t(U.T), t(C.T))
    b = cfg.rhs(2)
    x, info = prob.solve(t(b), tol=1e-8, k=8 if with_space else 0, mode="rBiCGStab", max_matvec=3000,
                         precond="subdomain", precision="mixed")
    xo, io = oracle.rbicgstab(op, b, tol=1e-8, U=U, C=C, max_matvec=3000, prec="schwarz")
    check_mixed(op, b, x.cpu().numpy(), info, xo, 1e-8, kappa(cfg.grid, cfg.coef))


def test_mixed_subdomain_hybrid_porous(ctx):
    """The hybrid in mixed precision with the sub-domain preconditioner (left
    rGCROT, then right rBiCGStab with the pair re-formed as A U = C), per step
    against the FP64 oracle's hybrid."""
    n = (20, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(78, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    prob = gpu_problem(ctx, grid, coef)
    op = oracle.Stencil(grid, coef)
    kap = kappa(grid, coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=20, k=10, tol=1e-8, hybrid_switch=2, max_matvec=3000,
                                   left=True, prec="schwarz")
    base = np.random.default_rng(5).standard_normal(grid.n)
    for s in range(4):
        b = base + 0.05 * s * np.random.default_rng(100 + s).standard_normal(grid.n)
        x, info = prob.solve(t(b), tol=1e-8, m=20, k=10, mode="hybrid", hybrid_switch=2, max_matvec=3000,
                             precond_side="left", precond="subdomain", precision="mixed")
        xo, io = seq.solve(b)
        assert info["mode_used"] == (1 if s < 2 else 2), (s, info)
        check_mixed(op, b, x.cpu().numpy(), info, xo, 1e-8, kap)
