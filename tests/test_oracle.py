"""Pins of the CPU oracle against facts fixed by the paper and by linear
algebra, not by the oracle itself: brute-force dense operators, dense LU
solutions, finite termination, monotone residuals (Table 1), the special
cases of Algorithms 3 and 4 with an empty recycle space (their notes), the
invariants of Sec. 2.3 (eqs. V_perp_C, aug-arnoldi-rec, aug-arnoldi-equiv),
harmonic Ritz values computed from explicit dense matrices, and exact
recycling."""
import numpy as np
import pytest
import scipy.linalg as sla

from problems import Grid, make_config, random_operator, porous_skew_19pt
from problems.operators import sphere_pack
from problems.fields import rng_for
import oracle
from oracle import Stencil, dense_matrix, gmres, rgcrot, bicgstab, rbicgstab, harmonic_ritz_update


def tiny_problems():
    out = []
    c1 = make_config(1, size=5)
    out.append(("convdiff", c1.grid, c1.coef, c1.rhs(0)))
    c2 = make_config(2, size=6)
    out.append(("channel", c2.grid, c2.coef, c2.rhs(1)))
    n = (7, 6, 5)
    solid, _ = sphere_pack(n, 1.6, 0.3, rng_for(9, 3), max_attempts=3000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-2, 1.0), 15.0)
    b = np.random.default_rng(3).standard_normal(grid.n)
    out.append(("porous", grid, coef, b))
    g = Grid(4, 5, 3, (True, False, True))
    out.append(("random19", g, random_operator(g, 19, np.random.default_rng(4), 1.2),
                np.random.default_rng(5).standard_normal(g.n)))
    return out


PROBS = tiny_problems()


@pytest.mark.parametrize("per", [(False, False, False), (True, False, True), (True, True, True)])
@pytest.mark.parametrize("S", [7, 19])
def test_stencil_matches_dense(per, S):
    g = Grid(5, 4, 3, per)
    coef = random_operator(g, S, np.random.default_rng(S))
    op = Stencil(g, coef)
    A = dense_matrix(g, coef)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(g.n)
    b = rng.standard_normal(g.n)
    scale = np.abs(A) @ np.abs(v)
    assert np.all(np.abs(op.apply(v) - A @ v) <= 1e-14 * scale)
    z = v / coef[0]
    assert np.all(np.abs(op.apply_prec(v) - A @ z) <= 1e-14 * (np.abs(A) @ np.abs(z)))
    assert np.all(np.abs(op.residual(b, v) - (b - A @ v)) <= 1e-14 * (scale + np.abs(b)))
    assert np.array_equal(op.dinv, 1.0 / coef[0])


@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
@pytest.mark.parametrize("mode", ["GMRES", "rGCROT", "BiCGStab", "rBiCGStab"])
def test_solvers_reach_dense_lu(name, grid, coef, b, mode):
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    xs = sla.solve(A, b)
    kappa = np.linalg.cond(A)
    tol = 1e-12
    if mode == "GMRES":
        x, info = gmres(op, b, tol=tol, m=12, max_matvec=5000)
    elif mode == "rGCROT":
        x, U, C, info = rgcrot(op, b, tol=tol, m=12, k=6, max_matvec=5000)
    elif mode == "BiCGStab":
        x, info = bicgstab(op, b, tol=tol, max_matvec=5000)
    else:
        # recycle space from a preceding rGCROT solve of a neighbouring rhs
        b0 = b + 0.1 * np.random.default_rng(7).standard_normal(b.size)
        _, U, C, _ = rgcrot(op, b0, tol=1e-10, m=12, k=6)
        x, info = rbicgstab(op, b, tol=tol, U=U, C=C, max_matvec=5000)
    rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert rel <= 10 * tol or (mode in ("BiCGStab", "rBiCGStab") and rel <= 1e-10)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= max(1e-9, 10 * kappa * rel)


def test_gmres_finite_termination():
    """Full GMRES (m >= N) terminates within N matrix-vector products."""
    g = Grid(3, 3, 3, (False, False, False))
    coef = random_operator(g, 19, np.random.default_rng(11), dominance=0.6)
    op = Stencil(g, coef)
    b = np.random.default_rng(12).standard_normal(g.n)
    x, info = gmres(op, b, tol=1e-11, m=g.n, max_matvec=g.n)
    assert info["status"] == oracle.OK and info["matvecs"] <= g.n
    assert info["cycles"] == 1


@pytest.mark.parametrize("name,grid,coef,b", PROBS[:3], ids=[p[0] for p in PROBS[:3]])
def test_monotone_true_residual(name, grid, coef, b):
    """GMRES(m) and rGCROT residual norms do not increase (Table 1)."""
    op = Stencil(grid, coef)
    _, i1 = gmres(op, b, tol=1e-11, m=5, max_matvec=3000)
    _, _, _, i2 = rgcrot(op, b, tol=1e-11, m=5, k=4, max_matvec=3000)
    for h in (i1["history"], i2["history"]):
        h = np.array(h)
        assert np.all(h[1:] <= h[:-1] * (1 + 1e-10))
        assert len(h) > 2


@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
def test_rgcrot_k0_is_gmres(name, grid, coef, b):
    """Algorithm 3 without a recycle space is Algorithm 1 (note under Alg. 3)."""
    op = Stencil(grid, coef)
    x1, i1 = gmres(op, b, tol=1e-10, m=7)
    x2, U, C, i2 = rgcrot(op, b, tol=1e-10, m=7, k=0)
    assert np.array_equal(x1, x2) and i1["matvecs"] == i2["matvecs"] and U is None


@pytest.mark.parametrize("prec", ["jacobi", "schwarz"])
@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
def test_rbicgstab_empty_is_bicgstab(name, grid, coef, b, prec):
    """Algorithm 4 with an empty recycle space is Algorithm 2 (note under
    Alg. 4), with either preconditioner."""
    op = Stencil(grid, coef)
    x1, i1 = bicgstab(op, b, tol=1e-10, prec=prec)
    x2, i2 = rbicgstab(op, b, tol=1e-10, max_restarts=0, prec=prec)
    assert np.array_equal(x1, x2) and i1["matvecs"] == i2["matvecs"]


@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
def test_recycle_invariants(name, grid, coef, b):
    """A U = C, C^T C = I (Sec. 2.3), V_{m+1} ⟂ C (eq. V_perp_C) and the
    augmented Arnoldi relation A M^{-1} V_m = C B + V_{m+1} H (eq.
    aug-arnoldi-rec), with dense matrices."""
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    Minv = np.diag(1.0 / coef[0])
    nA = np.linalg.norm(A, 2)
    _, U, C, _ = rgcrot(op, b, tol=1e-12, m=6, k=4, max_matvec=400)
    b2 = b + 0.05 * np.random.default_rng(2).standard_normal(b.size)
    x, U2, C2, info = rgcrot(op, b2, tol=1e-12, m=6, k=4, U=U, C=C, max_matvec=400, keep_cycle=True)
    for UU, CC in ((U, C), (U2, C2)):
        assert np.linalg.norm(A @ UU - CC) <= 1e-11 * nA * np.linalg.norm(UU)
        assert np.linalg.norm(CC.T @ CC - np.eye(CC.shape[1])) <= 1e-12
    lc = info["last_cycle"]
    V, H, B, Cc = lc["V"].T, lc["H"], lc["B"], lc["C"]
    jj = lc["jj"]
    assert np.linalg.norm(V.T @ Cc) <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(jj + 1)) <= 1e-12
    lhs = A @ Minv @ V[:, :jj]
    rhs = Cc @ B + V @ H
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(A @ Minv, 2)
    # eq. aug-arnoldi-equiv: (I - C C^T) A M^{-1} V_m = V_{m+1} H
    P = np.eye(A.shape[0]) - Cc @ Cc.T
    assert np.linalg.norm(P @ lhs - V @ H) <= 1e-12 * np.linalg.norm(A @ Minv, 2)


def test_harmonic_ritz_values_dense():
    """The small pencil (G^T G, G^T F) gives the harmonic Ritz values of
    A M^{-1} on range([M U, V_j]): eigenvalues of ((AY)^T AY, (AY)^T Y) with
    Y = [M U, V_j] formed explicitly."""
    name, grid, coef, b = PROBS[2]
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    M = np.diag(coef[0])
    Ahat = A @ np.linalg.inv(M)
    _, U, C, _ = rgcrot(op, b, tol=1e-12, m=6, k=4, max_matvec=60)
    b2 = b + 0.05 * np.random.default_rng(2).standard_normal(b.size)
    _, _, _, info = rgcrot(op, b2, tol=1e-14, m=6, k=4, U=U, C=C, max_matvec=6, keep_cycle=True, update=False)
    lc = info["last_cycle"]
    jj = lc["jj"]
    Vr = lc["V"]
    Hm = np.zeros((7, 6)); Hm[: jj + 1, :jj] = lc["H"]
    Bm = np.zeros((4, 6)); Bm[:, :jj] = lc["B"]
    Vfull = np.zeros((7, grid.n)); Vfull[: jj + 1] = Vr
    _, _, theta = harmonic_ritz_update(op, lc["U"], lc["C"], Vfull, Bm, Hm, jj, 4, return_theta=True)
    Y = np.concatenate([M @ lc["U"], Vr[:jj].T], axis=1)
    AY = Ahat @ Y
    ref = sla.eigvals(AY.T @ AY, AY.T @ Y)
    got = np.sort_complex(np.asarray(theta))
    ref = np.sort_complex(ref)
    scale = np.abs(ref).max()
    assert np.allclose(got, ref, atol=1e-9 * scale, rtol=1e-9)


def _dense_harmonic_selection(Ahat, Y, k, largest=False):
    """The harmonic Ritz vectors of the k smallest |theta| by definition, from
    explicit dense matrices: eigenpairs of ((AY)^T AY, (AY)^T Y) (Y a basis of
    the space, Ahat = A M^{-1}); the selected set is every eigenvalue with
    |theta| <= tau for the largest tau that keeps their number <= k (a
    conjugate pair shares |theta|, so it is in or out whole). Returns the
    coefficient matrix P (a complex vector enters as its real and imaginary
    parts), so the selected space is range(Y P). ``largest``: the k largest
    instead (a deliberately wrong selection, to show the pin can tell)."""
    AY = Ahat @ Y
    th, vec = sla.eig(AY.T @ AY, AY.T @ Y)
    mag = np.abs(th)
    sel = np.zeros(mag.size, dtype=bool)
    for t in (np.sort(mag)[::-1] if largest else np.sort(mag)):
        s = mag >= t * (1 - 1e-9) if largest else mag <= t * (1 + 1e-9)
        if s.sum() > k:
            break
        sel = s
    cols = []
    for i in np.nonzero(sel)[0]:
        if th[i].imag > 0:
            cols += [vec[:, i].real, vec[:, i].imag]
        elif th[i].imag == 0:
            cols.append(vec[:, i].real)
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("which,k,expect", [
    ("porous", 3, 3),      # real values only below the cut
    ("porous", 6, 5),      # the 6th and 7th smallest are a conjugate pair: dropped whole
    ("random19", 2, 1),    # the cut splits the first pair
    ("random19", 4, 3),    # one real value and one pair kept, the next pair split
    ("random19", 5, 5),    # one real value and two pairs
    ("convdiff", 4, 4),
    ("channel", 5, 5),
    ("skew19", 3, 3),      # the third smallest |theta| is real, but a pair has a smaller real part
    ("skew19", 5, 5),
])
def test_harmonic_ritz_selection_dense(which, k, expect):
    """The subspace that the recycle update keeps (Algorithm 3, "update U and
    C", read as GCRO-DR's harmonic Ritz vectors): range(U_new) must be
    M^{-1} range(Y P) with Y = [M U, V_j] and P the eigenvectors of the k
    smallest |theta| of the dense pencil ((AY)^T AY, (AY)^T Y), formed from the
    explicit matrix A M^{-1} (not from the small G, F of the update), and
    range(C_new) = A M^{-1} range(Y P). Cases where the k largest values span
    a different space and where the cut splits a conjugate pair."""
    if which == "skew19":
        # strongly nonsymmetric bands: complex values whose real parts order
        # differently from their moduli
        grid = Grid(4, 5, 3, (True, False, True))
        coef = random_operator(grid, 19, np.random.default_rng(5), 0.6)
        b = np.random.default_rng(5).standard_normal(grid.n)
    else:
        name, grid, coef, b = {p[0]: p for p in PROBS}[which]
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    M, Minv = np.diag(coef[0]), np.diag(1.0 / coef[0])
    Ahat = A @ Minv
    _, U, C, _ = rgcrot(op, b, tol=1e-12, m=6, k=4, max_matvec=60)
    b2 = b + 0.05 * np.random.default_rng(2).standard_normal(b.size)
    _, _, _, info = rgcrot(op, b2, tol=1e-14, m=6, k=4, U=U, C=C, max_matvec=6, keep_cycle=True, update=False)
    lc = info["last_cycle"]
    jj = lc["jj"]
    Hm = np.zeros((7, 6)); Hm[: jj + 1, :jj] = lc["H"]
    Bm = np.zeros((4, 6)); Bm[:, :jj] = lc["B"]
    Vfull = np.zeros((7, grid.n)); Vfull[: jj + 1] = lc["V"]
    Un, Cn = harmonic_ritz_update(op, lc["U"], lc["C"], Vfull, Bm, Hm, jj, k)
    Y = np.concatenate([M @ lc["U"], lc["V"][:jj].T], axis=1)
    P = _dense_harmonic_selection(Ahat, Y, k)
    assert P.shape[1] == expect
    assert Un.shape[1] == expect and Cn.shape[1] == expect
    assert sla.subspace_angles(Un, Minv @ Y @ P).max() <= 1e-10
    assert sla.subspace_angles(Cn, Ahat @ Y @ P).max() <= 1e-10
    assert np.linalg.norm(A @ Un - Cn) <= 1e-11 * np.linalg.norm(A, 2) * np.linalg.norm(Un)
    assert np.linalg.norm(Cn.T @ Cn - np.eye(expect)) <= 1e-12
    PL = _dense_harmonic_selection(Ahat, Y, k, largest=True)
    if PL.shape[1] == expect:  # the pin separates the smallest from the largest values
        assert sla.subspace_angles(Minv @ Y @ PL, Minv @ Y @ P).max() > 0.5


def test_exact_recycling():
    """If b lies in range(C) the initial projection onto C solves the
    system: no matrix-vector products and x = U C^T b."""
    name, grid, coef, b = PROBS[0]
    op = Stencil(grid, coef)
    _, U, C, _ = rgcrot(op, b, tol=1e-12, m=6, k=4, max_matvec=200)
    bb = C @ np.array([1.0, -2.0, 0.5, 3.0][: C.shape[1]])
    x, _, _, info = rgcrot(op, bb, tol=1e-10, m=6, k=4, U=U, C=C)
    assert info["matvecs"] == 0
    assert np.allclose(x, U @ (C.T @ bb), atol=1e-12 * np.linalg.norm(x))
    x2, info2 = rbicgstab(op, bb, tol=1e-10, U=U, C=C)
    assert info2["matvecs"] == 0
    A = dense_matrix(grid, coef)
    assert np.linalg.norm(bb - A @ x2) <= 1e-10 * np.linalg.norm(bb)


def test_rbicgstab_residuals_orthogonal_to_c_and_solution_relation():
    """Every updated rBiCGStab residual is ⟂ C (eq. rbicgstab-res: r lives in
    the Krylov space of (I - C C^T) A), and after the postponed U update the
    solution's true residual equals the updated one up to rounding
    (eq. sol-update-from-res)."""
    name, grid, coef, b = PROBS[2]
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    _, U, C, _ = rgcrot(op, b, tol=1e-11, m=8, k=5)
    b2 = b + 0.1 * np.random.default_rng(4).standard_normal(b.size)
    rs = []
    x, info = rbicgstab(op, b2, tol=1e-9, U=U, C=C, max_restarts=0, callback=lambda r: rs.append(r.copy()))
    assert len(rs) > 3
    for r in rs:
        assert np.linalg.norm(C.T @ r) <= 1e-10 * np.linalg.norm(b2)
    rtrue = b2 - A @ x
    assert np.linalg.norm(rtrue - rs[-1]) <= 1e-10 * np.linalg.norm(b2)


def test_hybrid_sequence_reuses_space():
    """Hybrid (Sec. 2.4): rGCROT builds U, C over the first steps, then
    rBiCGStab reuses them frozen; every step converges."""
    c = make_config(1, size=6)
    op = Stencil(c.grid, c.coef)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=8, k=6, tol=1e-9, hybrid_switch=2)
    modes = []
    for t in range(4):
        x, info = seq.solve(c.rhs(t))
        modes.append(info["mode"])
        assert info["status"] == oracle.OK and info["relres_true"] <= 1e-9
    assert modes == ["rGCROT", "rGCROT", "rBiCGStab", "rBiCGStab"]
    assert seq.U.shape[1] == 6


def test_zero_rhs():
    name, grid, coef, b = PROBS[0]
    op = Stencil(grid, coef)
    z = np.zeros_like(b)
    for f in (lambda: gmres(op, z), lambda: bicgstab(op, z), lambda: rbicgstab(op, z)):
        x, info = f()
        assert info["matvecs"] == 0 and np.all(x == 0)
    x, U, C, info = rgcrot(op, z)
    assert info["matvecs"] == 0 and np.all(x == 0)


@pytest.mark.parametrize("S", [7, 19])
def test_fp32_operator_within_rounding_bound(S):
    """The mixed-precision inner operator (coefficients, 1/a_pp and v rounded
    to FP32, FP32 accumulation) stays within the FP32 rounding bound of the
    FP64 operator: |w32 - w64| <= (S + 3) u32 sum_s |c_s| |z_s| elementwise."""
    g = Grid(6, 5, 4, (True, False, True))
    coef = random_operator(g, S, np.random.default_rng(S + 7))
    op = Stencil(g, coef)
    A = dense_matrix(g, coef)
    v = np.random.default_rng(8).standard_normal(g.n)
    w64 = op.apply_prec(v)
    w32 = op.apply_prec_f32(v)
    z = v / coef[0]
    bound = (S + 3) * 2.0 ** -24 * (np.abs(A) @ np.abs(z))
    assert np.all(np.abs(w32 - w64) <= bound)
    assert np.any(w32 != w64)  # it is not the FP64 operator


def _porous_small():
    n = (8, 7, 6)
    solid, _ = sphere_pack(n, 1.5, 0.25, rng_for(41, 3), max_attempts=5000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-3, 1.0), 15.0)
    return grid, coef, Stencil(grid, coef)


def test_hybrid_refresh_schedule():
    """Hybrid with intermittent rGCROT solves (Sec. 2.4): with a switch after
    2 solves and a refresh period of 2, the modes run rGCROT, rGCROT,
    rBiCGStab, rGCROT, rBiCGStab, rGCROT; the recycle space changes exactly
    on the rGCROT solves and every solve converges."""
    grid, coef, op = _porous_small()
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=10, k=6, tol=1e-9, hybrid_switch=2, refresh=2,
                                   max_matvec=3000)
    base = np.random.default_rng(9).standard_normal(grid.n)
    modes = []
    for s in range(6):
        b = base + 0.1 * s * np.random.default_rng(50 + s).standard_normal(grid.n)
        C0 = None if seq.C is None else seq.C.copy()
        x, info = seq.solve(b)
        modes.append(info["mode"])
        assert info["status"] == oracle.krylov.OK
        assert np.linalg.norm(op.residual(b, x)) <= 1e-9 * np.linalg.norm(b) * 1.0000001
        changed = C0 is None or C0.shape != seq.C.shape or not np.array_equal(C0, seq.C)
        assert changed == (info["mode"] == "rGCROT"), (s, info["mode"])
    assert modes == ["rGCROT", "rGCROT", "rBiCGStab", "rGCROT", "rBiCGStab", "rGCROT"]


def test_hybrid_fallback_switches_back():
    """Hybrid with the switch back to rGCROT (Sec. 2.4): an rBiCGStab solve
    that has not converged after F products is finished by rGCROT from its
    iterate (converging within the total budget, the products of both parts
    counted), and the next solve runs rGCROT again (a new phase of
    hybrid_switch solves starts with the fallback solve)."""
    grid, coef, op = _porous_small()
    F = 4
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=10, k=6, tol=1e-9, hybrid_switch=2, fallback=F,
                                   max_matvec=3000)
    plain = oracle.RecyclingSequence(op, mode="hybrid", m=10, k=6, tol=1e-9, hybrid_switch=2, max_matvec=3000)
    base = np.random.default_rng(11).standard_normal(grid.n)
    modes = []
    for s in range(5):
        b = base + 0.1 * s * np.random.default_rng(70 + s).standard_normal(grid.n)
        x, info = seq.solve(b)
        _, ip = plain.solve(b)
        modes.append(info["mode"])
        assert info["status"] == oracle.krylov.OK
        assert np.linalg.norm(op.residual(b, x)) <= 1e-9 * np.linalg.norm(b) * 1.0000001
        if s == 2:
            # the plain hybrid needs more than F products here, so this solve fell back
            assert ip["mode"] == "rBiCGStab" and ip["matvecs"] > F
            assert info["mode"] == "rGCROT" and info["matvecs"] > F
    # fallback at solve 2 starts a phase: solve 3 is rGCROT, solve 4 rBiCGStab (falling back again)
    assert modes[:4] == ["rGCROT", "rGCROT", "rGCROT", "rGCROT"]
    assert seq.base in (2, 4)


# ---------------------------------------------------------------- left preconditioning (Sec. 2.1)
@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
@pytest.mark.parametrize("mode", ["GMRES", "rGCROT"])
def test_left_preconditioned_solvers_reach_dense_lu(name, grid, coef, b, mode):
    """GMRES(m) and rGCROT(m,k) preconditioned from the left reach the dense
    LU solution: the true residual meets the tolerance (the stop test; the
    cycles themselves work on M^{-1}(b - A x)), and x is within kappa times
    the reached relative residual."""
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    Minv = np.diag(1.0 / coef[0])
    xs = sla.solve(A, b)
    tol = 1e-12
    if mode == "GMRES":
        x, info = gmres(op, b, tol=tol, m=12, max_matvec=5000, left=True)
    else:
        x, U, C, info = rgcrot(op, b, tol=tol, m=12, k=6, max_matvec=5000, left=True)
    assert info["status"] == oracle.OK
    rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    # relres_true is ||b - A x|| / ||b|| from the stencil residual: equal up
    # to the rounding of forming b - A x in two summation orders
    rounding = 64 * 2.0 ** -53 * np.linalg.norm(np.abs(A) @ np.abs(x)) / np.linalg.norm(b)
    assert abs(rel - info["relres_true"]) <= rounding
    assert info["relres_true"] <= tol and rel <= tol + rounding
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= max(1e-9, 10 * np.linalg.cond(A) * tol)


@pytest.mark.parametrize("prec", ["jacobi", "schwarz"])
@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
def test_left_rgcrot_k0_is_left_gmres(name, grid, coef, b, prec):
    """Without a recycle space, left-preconditioned Algorithm 3 is
    left-preconditioned Algorithm 1, bit for bit, with either preconditioner."""
    op = Stencil(grid, coef)
    x1, i1 = gmres(op, b, tol=1e-10, m=7, left=True, prec=prec)
    x2, U, C, i2 = rgcrot(op, b, tol=1e-10, m=7, k=0, left=True, prec=prec)
    assert np.array_equal(x1, x2) and i1["matvecs"] == i2["matvecs"] and U is None


@pytest.mark.parametrize("name,grid,coef,b", PROBS[:3], ids=[p[0] for p in PROBS[:3]])
def test_left_recycle_invariants_and_side_switch(name, grid, coef, b):
    """After left-preconditioned rGCROT: M^{-1} A U = C and C^T C = I (dense
    matrices). A right-preconditioned solve of the sequence re-forms C from
    U: then A U = C, range(U) unchanged."""
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    Minv = np.diag(1.0 / coef[0])
    seq = oracle.RecyclingSequence(op, mode="rGCROT", m=6, k=4, tol=1e-10, left=True)
    seq.solve(b)
    U, C = seq.U, seq.C
    nB = np.linalg.norm(Minv @ A, 2)
    assert np.linalg.norm(Minv @ A @ U - C) <= 1e-10 * nB * np.linalg.norm(U)
    assert np.linalg.norm(C.T @ C - np.eye(C.shape[1])) <= 1e-12
    seq.left = False
    seq._side(False)
    assert np.linalg.norm(A @ seq.U - seq.C) <= 1e-10 * np.linalg.norm(A, 2) * np.linalg.norm(seq.U)
    assert np.linalg.norm(seq.C.T @ seq.C - np.eye(C.shape[1])) <= 1e-12
    qa = np.linalg.qr(U)[0]
    qb = np.linalg.qr(seq.U)[0]
    assert np.linalg.norm(qb - qa @ (qa.T @ qb), 2) <= 1e-10


# ---------------------------------------------------------------- the sub-domain Jacobi preconditioner (Sec. 2.1)
def _schwarz_dense(grid, coef, box, ov, sweeps, omega):
    """The preconditioner as an explicit matrix, from its definition with
    dense algebra: per box, the extended index set, A restricted to it, the
    damped Jacobi polynomial sum_{t<sweeps} (I - w D^-1 A_b)^t w D^-1; owned
    rows kept (restriction); then the global sweep
    M^-1 = Z + w D^-1 (I - A Z)."""
    A = dense_matrix(grid, coef)
    n = grid.n
    d = np.diag(A).copy()
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    per = grid.periodic
    def wrapc(c, m, p):
        if 0 <= c < m:
            return c
        return (c % m) if p else -1
    Z = np.zeros((n, n))
    bx, by, bz = box
    for kb in range(0, nz, bz):
        for jb in range(0, ny, by):
            for ib in range(0, nx, bx):
                x1, y1, z1 = min(ib + bx, nx), min(jb + by, ny), min(kb + bz, nz)
                ext = []
                for c in range(kb - ov, z1 + ov):
                    for b_ in range(jb - ov, y1 + ov):
                        for a in range(ib - ov, x1 + ov):
                            g = (wrapc(a, nx, per[0]), wrapc(b_, ny, per[1]), wrapc(c, nz, per[2]))
                            ext.append(None if min(g) < 0 else g[0] + nx * (g[1] + ny * g[2]))
                ex, ey = (x1 - ib) + 2 * ov, (y1 - jb) + 2 * ov
                loc = [(e, gidx) for e, gidx in enumerate(ext) if gidx is not None]
                m_ = len(loc)
                Ab = np.zeros((m_, m_))
                pos = {e: t for t, (e, _) in enumerate(loc)}
                for t, (e, gp) in enumerate(loc):
                    a, rem = e % ex, e // ex
                    b_, c = rem % ey, rem // ey
                    for t2, (e2, gq) in enumerate(loc):
                        a2, rem2 = e2 % ex, e2 // ex
                        b2, c2 = rem2 % ey, rem2 // ey
                        da, db, dc = a2 - a, b2 - b_, c2 - c
                        if max(abs(da), abs(db), abs(dc)) > 1:
                            continue
                        # the band coupling cell gp to its (da, db, dc) neighbour
                        for s_, off in enumerate(OFFSETS[:coef.shape[0]]):
                            if off == (da, db, dc):
                                Ab[t, t2] = coef[s_][gp]
                dinv_b = np.array([1.0 / d[gp] for _, gp in loc])
                J = np.eye(m_) - omega * dinv_b[:, None] * Ab
                Pb = np.zeros((m_, m_))
                T = np.eye(m_)
                for _ in range(sweeps):
                    Pb += T
                    T = J @ T
                Pb = Pb * (omega * dinv_b)[None, :]
                # owned rows, columns scattered to their global cells
                for t, (e, gp) in enumerate(loc):
                    a, rem = e % ex, e // ex
                    b_, c = rem % ey, rem // ey
                    if ov <= a < ex - ov and ov <= b_ < ey - ov and ov <= c < (z1 - kb) + ov:
                        for t2, (_, gq) in enumerate(loc):
                            Z[gp, gq] += Pb[t, t2]
    return Z + omega * (1.0 / d)[:, None] * (np.eye(n) - A @ Z)


OFFSETS = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1),
           (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 1, 0), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (1, 0, 1),
           (0, -1, -1), (0, 1, -1), (0, -1, 1), (0, 1, 1)]


@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("per", [(False, False, False), (True, False, True)])
def test_schwarz_preconditioner_matches_its_dense_definition(S, per):
    """The C loops of the sub-domain preconditioner equal the matrix built
    from its definition (dense restriction, damped-Jacobi polynomial,
    restriction to owned cells, global sweep), column by column."""
    g = Grid(7, 6, 5, per)
    coef = random_operator(g, S, np.random.default_rng(S + 31), dominance=0.5)
    op = Stencil(g, coef)
    box, ov, sweeps, omega = (3, 4, 2), 1, 5, 2.0 / 3.0
    Md = _schwarz_dense(g, coef, box, ov, sweeps, omega)
    r = np.random.default_rng(3).standard_normal(g.n)
    z = op.schwarz(r, box=box, overlap=ov, sweeps=sweeps, omega=omega)
    assert np.allclose(z, Md @ r, rtol=1e-12, atol=1e-12 * np.abs(Md @ r).max())


def test_schwarz_preconditioner_is_linear_and_converges_to_the_inverse():
    """A fixed linear operator (so GMRES needs no flexible storage), and with
    one box covering the grid and many sweeps it tends to A^{-1}."""
    c = make_config(1, size=5)  # convection-diffusion M-matrix: damped Jacobi converges
    g, coef = c.grid, c.coef
    op = Stencil(g, coef)
    rng = np.random.default_rng(6)
    r1, r2 = rng.standard_normal(g.n), rng.standard_normal(g.n)
    z = op.schwarz(2.0 * r1 - 3.0 * r2)
    zl = 2.0 * op.schwarz(r1) - 3.0 * op.schwarz(r2)
    assert np.linalg.norm(z - zl) <= 1e-13 * np.linalg.norm(z)
    A = dense_matrix(g, coef)
    # damped Jacobi on the whole (unsplit) problem: spectral radius 0.992 here
    zi = op.schwarz(r1, box=(g.nx, g.ny, g.nz), overlap=1, sweeps=4000, omega=2.0 / 3.0)
    assert np.linalg.norm(A @ zi - r1) <= 1e-12 * np.linalg.norm(r1)


@pytest.mark.parametrize("name,grid,coef,b", PROBS, ids=[p[0] for p in PROBS])
@pytest.mark.parametrize("mode", ["GMRES", "rGCROT", "rBiCGStab"])
def test_schwarz_preconditioned_solvers_reach_dense_lu(name, grid, coef, b, mode):
    """GMRES(m) and rGCROT(m,k) left-preconditioned and rBiCGStab
    right-preconditioned by the sub-domain preconditioner reach the dense LU
    solution: the true residual meets the tolerance and x is within kappa(A)
    times it of A^{-1} b."""
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    xs = sla.solve(A, b)
    tol = 1e-11
    if mode == "GMRES":
        x, info = gmres(op, b, tol=tol, m=12, max_matvec=4000, left=True, prec="schwarz")
    elif mode == "rGCROT":
        x, _, _, info = rgcrot(op, b, tol=tol, m=12, k=6, max_matvec=4000, left=True, prec="schwarz")
    else:
        x, info = rbicgstab(op, b, tol=tol, max_matvec=4000, prec="schwarz")
    assert info["status"] == oracle.OK, info["status"]
    rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    rounding = 64 * 2.0 ** -53 * np.linalg.norm(np.abs(A) @ np.abs(x)) / np.linalg.norm(b)
    assert rel <= tol + rounding
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= max(1e-9, 10 * np.linalg.cond(A) * tol)


def test_left_stop_test_is_on_the_true_residual():
    """The stop test of left solves is on the true residual ||b - A x|| <=
    tol ||b|| (Sec. 4 states the criterion on the residual norm). Scaling the rows of A x = b by s leaves the point-Jacobi
    left-preconditioned system M^-1 A x = M^-1 b unchanged (M = diag(A)
    scales with the rows) but not ||b - A x|| / ||b||. With s spread over six
    decades, the left solve of the unscaled system returns an x whose
    preconditioned residual meets the tolerance while the scaled system's
    true residual does not; the solve of the scaled system continues until
    its true residual does (checked with dense matrices)."""
    c = make_config(1, size=6)
    g, coef, b = c.grid, c.coef, c.rhs(0)
    s = 10.0 ** np.random.default_rng(0).uniform(-3.0, 3.0, g.n)
    coef_s, b_s = coef * s[None, :], b * s
    A, A_s = dense_matrix(g, coef), dense_matrix(g, coef_s)
    tol = 1e-8
    xu, iu = gmres(Stencil(g, coef), b, tol=tol, m=20, left=True, max_matvec=3000)
    minv = 1.0 / coef[0]
    prel = np.linalg.norm(minv * (b - A @ xu)) / np.linalg.norm(minv * b)
    assert prel <= tol
    assert np.linalg.norm(b_s - A_s @ xu) / np.linalg.norm(b_s) > tol
    x, info = gmres(Stencil(g, coef_s), b_s, tol=tol, m=20, left=True, max_matvec=3000)
    assert info["status"] == oracle.OK
    assert np.linalg.norm(b_s - A_s @ x) / np.linalg.norm(b_s) <= tol
    assert info["matvecs"] > iu["matvecs"]


def test_schwarz_hybrid_sequence_sides_and_stop_test():
    """The hybrid with the sub-domain preconditioner (Sec. 2.4 with Sec. 2.1's
    sides): left rGCROT for the first solves (carried pair M^-1 A U = C with
    M^-1 the dense sub-domain matrix), then right rBiCGStab after the pair is
    re-formed as A U = C; every solve meets the true-residual tolerance."""
    name, grid, coef, b = PROBS[2]
    op = Stencil(grid, coef)
    A = dense_matrix(grid, coef)
    Md = _schwarz_dense(grid, coef, (16, 8, 8), 1, 5, 2.0 / 3.0)
    seq = oracle.RecyclingSequence(op, mode="hybrid", m=8, k=4, tol=1e-10, hybrid_switch=2, max_matvec=3000,
                                   left=True, prec="schwarz")
    rng = np.random.default_rng(11)
    modes = []
    for s in range(4):
        bs = b + 0.05 * s * rng.standard_normal(b.size)
        x, info = seq.solve(bs)
        modes.append(info["mode"])
        assert info["status"] == oracle.OK
        assert np.linalg.norm(bs - A @ x) <= 1e-10 * np.linalg.norm(bs) * (1 + 1e-6)
        if s == 0:  # after a left rGCROT solve: M^-1 A U = C
            B = Md @ A
            assert np.linalg.norm(B @ seq.U - seq.C) <= 1e-10 * np.linalg.norm(B, 2) * np.linalg.norm(seq.U)
    assert modes == ["rGCROT", "rGCROT", "rBiCGStab", "rBiCGStab"]
    assert np.linalg.norm(A @ seq.U - seq.C) <= 1e-10 * np.linalg.norm(A, 2) * np.linalg.norm(seq.U)
    assert np.linalg.norm(seq.C.T @ seq.C - np.eye(seq.C.shape[1])) <= 1e-11


@pytest.mark.parametrize("per", [(False, False, False), (True, False, True)])
@pytest.mark.parametrize("S", [7, 19])
def test_fp32_subdomain_preconditioner_near_its_fp64_form(S, per):
    """The FP32 restatement of the sub-domain preconditioner (the mixed
    precision's M^{-1}: bands, 1/a_pp, r and omega rounded to FP32 once,
    every sweep in FP32 in the FP64 order) stays within FP32 rounding of the
    FP64 preconditioner, which is pinned against its dense definition
    (test_schwarz_preconditioner_matches_its_dense_definition); a dropped
    band, a wrong sign or omega, or a skipped sweep moves it by O(1). The
    same for the FP32 operator with and without left point Jacobi, and for
    the left and right preconditioned products."""
    g = Grid(37, 11, 9, per)
    coef = random_operator(g, S, np.random.default_rng(S + 3))
    op = Stencil(g, coef)
    A = dense_matrix(g, coef)
    r = np.random.default_rng(9).standard_normal(g.n)
    z64 = op.schwarz(r)
    z32 = op.schwarz_f32(r)
    assert np.linalg.norm(z32 - z64) <= 1e-5 * np.linalg.norm(z64)
    assert np.any(z32 != z64)
    # the FP32 operator: elementwise FP32 rounding bound of A v
    w32 = op.apply_f32(r)
    assert np.all(np.abs(w32 - A @ r) <= (S + 2) * 2.0 ** -24 * (np.abs(A) @ np.abs(r)))
    wl = op.apply_f32(r, left=True)
    assert np.all(np.abs(wl - (A @ r) / coef[0]) <= (S + 4) * 2.0 ** -24 * (np.abs(A) @ np.abs(r)) / np.abs(coef[0]))
    left = op.left_schwarz_f32(r)
    assert np.linalg.norm(left - op.schwarz(op.apply(r))) <= 1e-5 * np.linalg.norm(left)
    right = op.right_schwarz_f32(r)
    assert np.linalg.norm(right - op.apply(op.schwarz(r))) <= 1e-5 * np.linalg.norm(right)
