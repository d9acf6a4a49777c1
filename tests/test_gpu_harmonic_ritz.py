"""The device harmonic Ritz selection (Algorithm 3's recycle update) through the C
ABI, against SciPy's generalized eigensolver on the same small pencils."""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_1501_03358_gb300 import Context
    c = Context()
    yield c
    c.close()


def pencil(kc, jj, seed):
    """G = [[I, B], [0, H]] (H (jj+1) x jj upper Hessenberg) and
    F = [[C^T M U, 0], [V^T M U, [I; 0]]] as in a cycle of rGCROT."""
    rng = np.random.default_rng(seed)
    n = kc + jj
    G = np.zeros((n + 1, n))
    F = np.zeros((n + 1, n))
    G[:kc, :kc] = np.eye(kc)
    G[:kc, kc:] = 0.3 * rng.standard_normal((kc, jj))
    H = np.triu(rng.standard_normal((jj + 1, jj)), -1)
    H[np.arange(1, jj + 1), np.arange(jj)] = np.abs(H[np.arange(1, jj + 1), np.arange(jj)]) + 0.1
    G[kc:, kc:] = H
    if kc:
        F[:kc, :kc] = np.eye(kc) + 0.2 * rng.standard_normal((kc, kc))
        F[kc:, :kc] = 0.1 * rng.standard_normal((jj + 1, kc))
    F[kc:kc + jj, kc:] = np.eye(jj)
    return G, F


def reference_basis(G, F, k):
    ab, vr = sla.eig(G.T @ G, G.T @ F, homogeneous_eigvals=True)
    theta = ab[0] / ab[1]
    order = np.argsort(np.abs(theta))
    cols, used = [], set()
    for i in order:
        if len(cols) >= k:
            break
        if i in used:
            continue
        if abs(theta[i].imag) > 0:
            if len(cols) + 2 > k:
                break
            cols += [vr[:, i].real, vr[:, i].imag]
            j = min((j for j in order if j != i and j not in used), key=lambda j: abs(theta[j] - np.conj(theta[i])))
            used |= {i, j}
        else:
            cols.append(vr[:, i].real)
            used.add(i)
    return np.linalg.qr(np.stack(cols, axis=1))[0], np.sort(np.abs(theta))


def gap(A, B):
    """sin of the largest principal angle, ||(I - Qa Qa^T) Qb||_2 (accurate
    for small angles, unlike sqrt(1 - cos^2))."""
    qa = np.linalg.qr(A)[0]
    qb = np.linalg.qr(B)[0]
    return float(np.linalg.norm(qb - qa @ (qa.T @ qb), 2))


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("kc,jj,k,seed", [(0, 10, 4, 1), (0, 40, 20, 2), (8, 12, 6, 3), (20, 40, 20, 4),
                                         (10, 30, 10, 5), (20, 40, 20, 6), (5, 3, 8, 7)])
def test_harmonic_ritz_matches_scipy(ctx, kc, jj, k, seed, precision):
    """The Schur iteration in FP64 (RK_FP64 / RK_MIXED solves) and in
    double-float (RK_DF solves) select SciPy's subspace."""
    G, F = pencil(kc, jj, seed)
    n = kc + jj
    k = min(k, n)
    QC, PU = ctx.harmonic_ritz(torch.from_numpy(G), torch.from_numpy(F), k, precision=precision)
    QC, PU = QC.cpu().numpy(), PU.cpu().numpy()
    P, mags = reference_basis(G, F, k)
    assert PU.shape[1] == P.shape[1]
    assert np.linalg.norm(QC.T @ QC - np.eye(QC.shape[1])) <= 1e-12
    assert np.linalg.norm(G @ PU - QC) <= 1e-11 * np.linalg.norm(G) * np.linalg.norm(PU)
    # subspace agreement within the pencil's own rounding sensitivity: SciPy's
    # selected subspace for G, F perturbed by 1e-14 relative shows how far
    # rounding alone moves it (near-tied |theta| at the cut make it large)
    rng = np.random.default_rng(seed + 100)
    sens = 0.0
    for _ in range(2):
        Gp = G * (1 + 1e-14 * rng.standard_normal(G.shape))
        Fp = F * (1 + 1e-14 * rng.standard_normal(F.shape))
        Pp, _ = reference_basis(Gp, Fp, k)
        if Pp.shape[1] == P.shape[1]:
            sens = max(sens, gap(Pp, P))
    assert gap(PU, P) <= 100.0 * sens + 1e-10, (gap(PU, P), sens)


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_pencil_with_near_zero_eigenvalues(ctx, precision):
    """The second-cycle pencil of rGCROT(20,10) on a small skewed porous
    problem: M'' has eigenvalues near zero, whose neighbouring diagonal
    entries are tiny, so a purely relative deflation test never fires at the
    double-float noise level of the subdiagonal. The Schur iteration must
    still converge (status ok) and select the oracle's subspace."""
    import oracle
    import oracle.krylov as K
    from problems.operators import sphere_pack, porous_skew_19pt
    from problems.fields import rng_for
    n = (14, 12, 10)
    solid, _ = sphere_pack(n, 2.5, 0.3, rng_for(77, 3), max_attempts=20000)
    grid, coef = porous_skew_19pt(n, np.where(solid, 1e-4, 1.0), 15.0)
    op = oracle.Stencil(grid, coef)
    b = np.random.default_rng(5).standard_normal(grid.n)
    pens = []
    orig = K.harmonic_ritz_update

    def hook(op_, U, C, V, B, H, jj, k, return_theta=False, left=False):
        kc = 0 if U is None else U.shape[1]
        nn = kc + jj
        G = np.zeros((nn + 1, nn))
        F = np.zeros((nn + 1, nn))
        if kc:
            G[:kc, :kc] = np.eye(kc)
            G[:kc, kc:] = B[:kc, :jj]
            MU = U * op_.coef[0][:, None]
            F[:kc, :kc] = C.T @ MU
            F[kc:, :kc] = V[: jj + 1] @ MU
        G[kc:, kc:] = H[: jj + 1, :jj]
        F[kc:kc + jj, kc:] = np.eye(jj)
        pens.append((G, F))
        return orig(op_, U, C, V, B, H, jj, k, return_theta, left)

    K.harmonic_ritz_update = hook
    try:
        oracle.rgcrot(op, b, tol=1e-8, m=20, k=10, max_matvec=40)
    finally:
        K.harmonic_ritz_update = orig
    G, F = pens[1]
    QC, PU = ctx.harmonic_ritz(torch.from_numpy(G), torch.from_numpy(F), 10, precision=precision)
    PU = PU.cpu().numpy()
    P, _ = reference_basis(G, F, 10)
    assert PU.shape[1] == P.shape[1] == 9  # the third complex pair is split by the cut and dropped
    assert gap(PU, P) <= 1e-8
