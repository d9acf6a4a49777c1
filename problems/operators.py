"""Finite-volume operators on structured grids, in banded storage.

Stand-ins for the pressure Poisson operator of eq. (1) (Sec. 2.1): the FVM
turns it into A x = b with 7 coefficients per cell on orthogonal grids and 19
on non-orthogonal ones; A is nonsymmetric for non-Cartesian meshes or some
boundary conditions. Every operator returns ``coef`` of shape (S, N), float64,
with bands ordered as in ``problems.grid.OFFSETS`` and every band that points
out of a non-periodic face set to exactly 0.
"""
import math

import numpy as np

from .grid import Grid, OFFSETS


def _flat(c3):
    return np.ascontiguousarray(c3.reshape(-1))


def _pack(grid: Grid, bands: dict, S: int) -> np.ndarray:
    coef = np.zeros((S, grid.n), dtype=np.float64)
    for s in range(S):
        off = OFFSETS[s]
        if off in bands:
            coef[s] = _flat(bands[off])
    # structural zero outside the domain
    for s in range(1, S):
        coef[s][~grid.band_valid(s).reshape(-1)] = 0.0
    return coef


def convection_diffusion_7pt(n: int, c_vec, h: float = 1.0):
    """-lap(p) + c.grad(p) on an n^3 cell grid, first-order upwind convection.

    Diffusion coefficient 1, cell size h (=1 by default). Dirichlet p=0 on the
    x=0 face through an antisymmetric ghost (diffusion weight 2; the upwind
    convective flux through that face is |F| p_P whichever its sign); every
    other face is Neumann with zero total flux (no diffusive and no convective
    term). The result is a nonsingular, nonsymmetric M-matrix. Per unit volume.
    """
    grid = Grid(n, n, n, (False, False, False))
    c = np.asarray(c_vec, dtype=float)
    shape = grid.shape3
    diag = np.zeros(shape)
    bands = {}
    inv_h2 = 1.0 / (h * h)
    # face normals in band order 1..6
    for s in range(1, 7):
        off = OFFSETS[s]
        normal = np.array(off, dtype=float)
        F = float(c @ normal) / h  # convective flux per unit volume (area h^2, volume h^3)
        valid = grid.band_valid(s)
        off_c = np.where(valid, -(inv_h2 + max(-F, 0.0)), 0.0)
        bands[off] = off_c
        diag += np.where(valid, inv_h2 + max(F, 0.0), 0.0)
        if s == 1:  # x = 0 face: Dirichlet
            diag[:, :, 0] += 2.0 * inv_h2 + abs(F)
    bands[(0, 0, 0)] = diag
    return grid, _pack(grid, bands, 7)


def channel_geometry(nx, ny, nz, beta=2.0, lx=4 * math.pi, lz=4 * math.pi / 3):
    """Cell widths of the wall-refined channel: uniform in x and z, y faces
    y_j = tanh(beta*(2j/ny - 1))/tanh(beta) on [-1, 1]."""
    j = np.arange(ny + 1)
    yf = np.tanh(beta * (2.0 * j / ny - 1.0)) / math.tanh(beta)
    hy = np.diff(yf)
    hx = np.full(nx, lx / nx)
    hz = np.full(nz, lz / nz)
    return hx, hy, hz, yf


def channel_7pt(nx, ny, nz, beta=2.0, lx=4 * math.pi, lz=4 * math.pi / 3, pin=True):
    """Pressure operator of a periodic (x, z) channel with Neumann walls in y.

    Per-unit-volume form: a_PN = -A_f / (d_PN * V_P), a_P = -sum a_PN. Rows are
    not multiplied back by V_P, so A is nonsymmetric on the stretched y-grid
    (V_P A is symmetric). With ``pin``, cell 0 keeps its diagonal and loses
    its off-diagonals, which removes the constant null space (b must be 0
    there)."""
    grid = Grid(nx, ny, nz, (True, False, True))
    hx, hy, hz, yf = channel_geometry(nx, ny, nz, beta, lx, lz)
    yc = 0.5 * (yf[:-1] + yf[1:])
    shape = grid.shape3
    HX = hx[None, None, :] * np.ones(shape)
    HY = hy[None, :, None] * np.ones(shape)
    HZ = hz[:, None, None] * np.ones(shape)
    bands = {}
    # x faces: A = hy*hz, d = hx, V = hx*hy*hz  -> 1/hx^2 (periodic)
    cx = 1.0 / (HX * HX)
    bands[(-1, 0, 0)] = -cx
    bands[(1, 0, 0)] = -cx.copy()
    cz = 1.0 / (HZ * HZ)
    bands[(0, 0, -1)] = -cz
    bands[(0, 0, 1)] = -cz.copy()
    # y faces: A = hx*hz, d = yc[j+1]-yc[j], V = hx*hy_j*hz -> 1/(d*hy_j)
    dyc = np.diff(yc)  # ny-1 interior distances
    cyp = np.zeros(shape)
    cym = np.zeros(shape)
    cyp[:, :-1, :] = (1.0 / (dyc[None, :, None] * hy[None, :-1, None])) * np.ones((nz, ny - 1, nx))
    cym[:, 1:, :] = (1.0 / (dyc[None, :, None] * hy[None, 1:, None])) * np.ones((nz, ny - 1, nx))
    bands[(0, 1, 0)] = -cyp
    bands[(0, -1, 0)] = -cym
    diag = 2 * cx + 2 * cz + cyp + cym
    bands[(0, 0, 0)] = diag
    coef = _pack(grid, bands, 7)
    if pin:
        coef[1:, 0] = 0.0
    return grid, coef, (hx, hy, hz)


def _fold_ghosts(grid: Grid, st: dict, signs) -> dict:
    """Fold references to ghost cells back into the domain.

    ``st`` maps a 3x3x3 offset to an (nz, ny, nx) coefficient array. A ghost
    across a non-periodic face of axis a equals sign[a] times the mirrored
    interior cell (the cell itself, for a one-cell stencil): sign -1 for a
    Dirichlet-zero face (antisymmetric ghost), +1 for a Neumann face."""
    dims = (grid.nx, grid.ny, grid.nz)
    for a in range(3):
        if grid.periodic[a]:
            continue
        ax = 2 - a
        for off in list(st.keys()):
            d = off[a]
            if d == 0:
                continue
            arr = st[off]
            sl = [slice(None)] * 3
            sl[ax] = 0 if d < 0 else dims[a] - 1
            sl = tuple(sl)
            moved = arr[sl].copy()
            if not np.any(moved):
                continue
            arr[sl] = 0.0
            tgt = list(off)
            tgt[a] = 0
            tgt = tuple(tgt)
            if tgt not in st:
                st[tgt] = np.zeros(grid.shape3)
            sign = signs[a][0 if d < 0 else 1]
            st[tgt][sl] += sign * moved
    return st


def porous_skew_19pt(n_xyz, kappa: np.ndarray, skew_deg: float):
    """Variable-conductivity diffusion on an affinely skewed grid, 19 bands.

    Physical X = xi + eta*tan(theta), Y = eta, Z = zeta, so sqrt(g) = 1,
    g11 = 1 + tan^2, g12 = -tan, g22 = g33 = 1 (unit cells). Operator
    (A p)_P = -(sum of outward face fluxes) with face flux
    kappa_f * (g^{aa} d_a p + g^{ab} d_b p), kappa_f the harmonic mean of the
    two cells, d_a p the two-point difference across the face and the cross
    derivative d_b p the mean of the two cells' central differences.
    Dirichlet p = 0 on both x faces (antisymmetric ghosts), Neumann (zero total
    flux, mirror ghosts in cross differences) on the y and z faces. Only the xy
    edge bands are populated; the xz and yz bands are stored as zeros."""
    nx, ny, nz = n_xyz
    grid = Grid(nx, ny, nz, (False, False, False))
    shape = grid.shape3
    k = np.asarray(kappa, dtype=float).reshape(shape)
    t = math.tan(math.radians(skew_deg))
    g11, g12, g22, g33 = 1.0 + t * t, -t, 1.0, 1.0

    def hm(a, b):
        return 2.0 * a * b / (a + b)

    # face conductivities toward +x, -x, +y, -y, +z, -z (boundary: the cell's own)
    ke = k.copy(); ke[:, :, :-1] = hm(k[:, :, :-1], k[:, :, 1:])
    kw = k.copy(); kw[:, :, 1:] = hm(k[:, :, 1:], k[:, :, :-1])
    kn = k.copy(); kn[:, :-1, :] = hm(k[:, :-1, :], k[:, 1:, :])
    ks = k.copy(); ks[:, 1:, :] = hm(k[:, 1:, :], k[:, :-1, :])
    kt = k.copy(); kt[:-1, :, :] = hm(k[:-1, :, :], k[1:, :, :])
    kb = k.copy(); kb[1:, :, :] = hm(k[1:, :, :], k[:-1, :, :])
    # Neumann faces carry zero total flux
    kn[:, -1, :] = 0.0
    ks[:, 0, :] = 0.0
    kt[-1, :, :] = 0.0
    kb[0, :, :] = 0.0

    st = {}

    def add(off, arr):
        if off in st:
            st[off] = st[off] + arr
        else:
            st[off] = arr.copy()

    q = g12 / 4.0
    # A p = -F_e + F_w - F_n + F_s - F_t + F_b
    # F_e = ke[g11 (pE - pP) + q((pN - pS) + (pNE - pSE))]
    add((1, 0, 0), -ke * g11); add((0, 0, 0), ke * g11)
    add((0, 1, 0), -ke * q); add((0, -1, 0), ke * q); add((1, 1, 0), -ke * q); add((1, -1, 0), ke * q)
    # F_w = kw[g11 (pP - pW) + q((pN - pS) + (pNW - pSW))]
    add((0, 0, 0), kw * g11); add((-1, 0, 0), -kw * g11)
    add((0, 1, 0), kw * q); add((0, -1, 0), -kw * q); add((-1, 1, 0), kw * q); add((-1, -1, 0), -kw * q)
    # F_n = kn[g22 (pN - pP) + q((pE - pW) + (pNE - pNW))]
    add((0, 1, 0), -kn * g22); add((0, 0, 0), kn * g22)
    add((1, 0, 0), -kn * q); add((-1, 0, 0), kn * q); add((1, 1, 0), -kn * q); add((-1, 1, 0), kn * q)
    # F_s = ks[g22 (pP - pS) + q((pE - pW) + (pSE - pSW))]
    add((0, 0, 0), ks * g22); add((0, -1, 0), -ks * g22)
    add((1, 0, 0), ks * q); add((-1, 0, 0), -ks * q); add((1, -1, 0), ks * q); add((-1, -1, 0), -ks * q)
    # F_t, F_b
    add((0, 0, 1), -kt * g33); add((0, 0, 0), kt * g33)
    add((0, 0, 0), kb * g33); add((0, 0, -1), -kb * g33)

    signs = ((-1.0, -1.0), (1.0, 1.0), (1.0, 1.0))  # x Dirichlet both ends; y, z Neumann
    st = _fold_ghosts(grid, st, signs)
    return grid, _pack(grid, st, 19)


def sphere_pack(n_xyz, radius: float, target: float, rng: np.random.Generator, max_attempts: int = 1_000_000):
    """Random sequential addition of non-overlapping spheres.

    Centres are uniform in the box (spheres may be clipped by the boundary);
    a candidate is accepted when its centre is more than 2*radius from every
    accepted centre. Stops when the voxel solid fraction (cells whose centre
    lies within ``radius`` of a centre) reaches ``target`` or after
    ``max_attempts`` candidates. Returns (solid mask (nz, ny, nx), fraction)."""
    nx, ny, nz = n_xyz
    L = np.array([nx, ny, nz], float)
    cell = 2.0 * radius
    nb = np.maximum(1, (L // cell).astype(int))
    buckets = {}
    centres = []
    solid = np.zeros((nz, ny, nx), dtype=bool)
    r = int(math.ceil(radius))
    ox = np.arange(-r, r + 1)
    count = 0
    total = nx * ny * nz
    batch = 4096
    attempts = 0
    while attempts < max_attempts and count < target * total:
        cand = rng.random((batch, 3)) * L
        for c in cand:
            attempts += 1
            b = tuple(np.minimum((c // cell).astype(int), nb - 1))
            ok = True
            for dxb in (-1, 0, 1):
                for dyb in (-1, 0, 1):
                    for dzb in (-1, 0, 1):
                        for cc in buckets.get((b[0] + dxb, b[1] + dyb, b[2] + dzb), ()):
                            dd = c - cc
                            if dd @ dd <= cell * cell:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                buckets.setdefault(b, []).append(c)
                centres.append(c)
                # voxelise: cell centres at (i + 0.5)
                ci = np.floor(c).astype(int)
                xs = ci[0] + ox; ys = ci[1] + ox; zs = ci[2] + ox
                xs = xs[(xs >= 0) & (xs < nx)]; ys = ys[(ys >= 0) & (ys < ny)]; zs = zs[(zs >= 0) & (zs < nz)]
                ZZ, YY, XX = np.meshgrid(zs, ys, xs, indexing="ij")
                inside = ((XX + 0.5 - c[0]) ** 2 + (YY + 0.5 - c[1]) ** 2 + (ZZ + 0.5 - c[2]) ** 2) <= radius * radius
                sub = solid[zs[0]:zs[-1] + 1, ys[0]:ys[-1] + 1, xs[0]:xs[-1] + 1]
                newly = inside & ~sub
                count += int(newly.sum())
                sub |= inside
                if count >= target * total:
                    break
            if attempts >= max_attempts:
                break
    return solid, count / total


def random_operator(grid: Grid, S: int, rng: np.random.Generator, dominance: float = 1.5):
    """Random fully populated S-band operator (tests only): off-diagonals
    U(-1, 1) on every valid band, diagonal = dominance * sum|off| + 0.1."""
    coef = np.zeros((S, grid.n))
    for s in range(1, S):
        v = rng.uniform(-1.0, 1.0, grid.n)
        v[~grid.band_valid(s).reshape(-1)] = 0.0
        coef[s] = v
    coef[0] = dominance * np.abs(coef[1:]).sum(axis=0) + 0.1
    return coef
