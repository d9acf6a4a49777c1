"""Pins of the seeded problem generators: closed forms, exactness on
polynomials, conservation, structure. None of these use the oracle."""
import math

import numpy as np
import pytest

from problems import Grid, OFFSETS, make_config, porous_skew_19pt, channel_7pt, convection_diffusion_7pt, random_operator
from problems.fields import face_velocity, divergence, rng_for
from problems.operators import channel_geometry, sphere_pack


def apply_bands(grid, coef, u3):
    """Reference application by array shifts (np.roll + explicit masking)."""
    out = np.zeros(grid.shape3)
    for s in range(coef.shape[0]):
        dx, dy, dz = OFFSETS[s]
        shifted = np.roll(u3, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        c = coef[s].reshape(grid.shape3)
        out += np.where(grid.band_valid(s), c * shifted, 0.0)
    return out


@pytest.mark.parametrize("maker", ["cd", "ch", "po"])
def test_bands_out_of_domain_are_zero(maker):
    if maker == "cd":
        grid, coef = convection_diffusion_7pt(5, [0.3, -0.2, 0.1])
    elif maker == "ch":
        grid, coef, _ = channel_7pt(6, 5, 4)
    else:
        grid, coef = porous_skew_19pt((6, 5, 4), np.ones((4, 5, 6)), 15.0)
    for s in range(1, coef.shape[0]):
        bad = ~grid.band_valid(s).reshape(-1)
        assert np.all(coef[s][bad] == 0.0)


def test_laplacian_closed_form_eigenpairs():
    """Unskewed unit-conductivity operator (x Dirichlet, y/z Neumann): the
    cell-centred Laplacian's eigenvectors sin(pi p (i+1/2)/n) (Dirichlet, p>=1)
    and cos(pi q (j+1/2)/n) (Neumann, q>=0) with eigenvalue sum of
    4 sin^2(pi p / (2n))."""
    nx, ny, nz = 6, 5, 4
    grid, coef = porous_skew_19pt((nx, ny, nz), np.ones((nz, ny, nx)), 0.0)
    i, j, k = np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5
    for p, q, r in [(1, 0, 0), (2, 1, 0), (6, 4, 3), (3, 2, 1)]:
        ux = np.sin(math.pi * p * i / nx)
        uy = np.cos(math.pi * q * j / ny)
        uz = np.cos(math.pi * r * k / nz)
        u = uz[:, None, None] * uy[None, :, None] * ux[None, None, :]
        lam = (4 * math.sin(math.pi * p / (2 * nx)) ** 2 + 4 * math.sin(math.pi * q / (2 * ny)) ** 2
               + 4 * math.sin(math.pi * r / (2 * nz)) ** 2)
        Au = apply_bands(grid, coef, u)
        assert np.allclose(Au, lam * u, atol=1e-12)


def test_skewed_operator_exact_on_quadratics():
    """With unit conductivity the skewed 19-point operator is -lap in physical
    coordinates X = xi + eta tan(theta), Y = eta: it annihilates X and Y and
    maps X^2 + Y^2 to -4, exactly in cells whose stencil stays inside."""
    n = 8
    t = math.tan(math.radians(15.0))
    grid, coef = porous_skew_19pt((n, n, n), np.ones((n, n, n)), 15.0)
    zz, yy, xx = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    X = xx + yy * t
    Y = yy
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.allclose(apply_bands(grid, coef, X)[inner], 0.0, atol=1e-11)
    assert np.allclose(apply_bands(grid, coef, Y)[inner], 0.0, atol=1e-11)
    q = apply_bands(grid, coef, X * X + Y * Y)[inner]
    assert np.allclose(q, -4.0, atol=1e-10)
    # populated bands: centre, faces and the xy edges only
    nz_bands = [s for s in range(19) if np.any(coef[s] != 0)]
    assert set(nz_bands) <= set(range(11))
    assert set(range(7, 11)) <= set(nz_bands)


def test_channel_structure():
    """Per-unit-volume channel operator: V A is symmetric, A 1 = 0 without the
    pin, A annihilates fields linear in y in the interior and maps X^2 to -2
    away from the periodic seam; the pin zeroes the off-diagonals of cell 0."""
    nx, ny, nz = 6, 8, 5
    grid, coef, (hx, hy, hz) = channel_7pt(nx, ny, nz, pin=False)
    vol = (hz[:, None, None] * hy[None, :, None] * hx[None, None, :]).reshape(-1)
    from oracle import dense_matrix  # brute-force assembly used only as a reader of the bands
    A = dense_matrix(grid, coef)
    VA = vol[:, None] * A
    assert np.allclose(VA, VA.T, atol=1e-12 * np.abs(VA).max())
    assert not np.allclose(A, A.T)
    assert np.allclose(A @ np.ones(grid.n), 0.0, atol=1e-10 * np.abs(A).max())
    _, _, _, yf = channel_geometry(nx, ny, nz)
    yc = 0.5 * (yf[:-1] + yf[1:])
    u = np.broadcast_to(yc[None, :, None], grid.shape3).copy()
    Au = apply_bands(grid, coef, u)
    assert np.allclose(Au[:, 1:-1, :], 0.0, atol=1e-9 * np.abs(A).max())
    xc = (np.arange(nx) + 0.5) * hx[0]
    u = np.broadcast_to((xc ** 2)[None, None, :], grid.shape3).copy()
    Au = apply_bands(grid, coef, u)
    assert np.allclose(Au[:, :, 1:-1], -2.0, atol=1e-9)
    _, coefp, _ = channel_7pt(nx, ny, nz, pin=True)
    assert np.all(coefp[1:, 0] == 0.0) and coefp[0, 0] == coef[0, 0]
    assert np.array_equal(coefp[:, 1:], coef[:, 1:])


def test_upwind_conservation_and_m_matrix():
    """First-order upwind convection is conservative (interior column sums of
    the convective part vanish) and the operator is an M-matrix."""
    n = 5
    c = np.array([0.3, -0.4, 0.1])
    grid, A1 = convection_diffusion_7pt(n, c)
    _, A0 = convection_diffusion_7pt(n, [0.0, 0.0, 0.0])
    from oracle import dense_matrix
    D1 = dense_matrix(grid, A1)
    D0 = dense_matrix(grid, A0)
    conv = D1 - D0
    cols = conv.sum(axis=0).reshape(grid.shape3)
    assert np.allclose(cols[:, :, 1:], 0.0, atol=1e-14)
    off = D1 - np.diag(np.diag(D1))
    assert np.all(off <= 0.0)
    assert np.all(D1.sum(axis=0) >= -1e-14)
    assert not np.allclose(D1, D1.T)


def test_divergence_gauss_theorem():
    """Sum of V_P div_P vanishes for face fields with zero normal velocity at
    walls and periodic wrap elsewhere (discrete Gauss theorem)."""
    nx, ny, nz = 8, 6, 5
    grid = Grid(nx, ny, nz, (True, False, True))
    hx, hy, hz, _ = channel_geometry(nx, ny, nz)
    u = face_velocity(grid, 2.0, rng_for(1, 2), walls=(False, True, False))
    d = divergence(grid, hx, hy, hz, *u)
    vol = hz[:, None, None] * hy[None, :, None] * hx[None, None, :]
    assert abs(np.sum(d * vol)) < 1e-12 * np.sum(np.abs(d * vol))
    # a uniform flow has zero divergence
    ux = np.ones((nz, ny, nx))
    uy = np.zeros((nz, ny + 1, nx))
    uz = np.ones((nz, ny, nx))
    assert np.allclose(divergence(grid, hx, hy, hz, ux, uy, uz), 0.0)


def test_sphere_pack_disjoint():
    n = (30, 28, 26)
    solid, frac = sphere_pack(n, 3.0, 0.25, rng_for(5, 3), max_attempts=20000)
    assert 0.05 < frac <= 0.45
    assert abs(solid.mean() - frac) < 1e-12


def test_config_determinism_and_sequence():
    c1 = make_config(2, size=8)
    c2 = make_config(2, size=8)
    assert np.array_equal(c1.coef, c2.coef)
    b0, b1 = c1.rhs(0), c1.rhs(1)
    assert np.array_equal(b0, c2.rhs(0))
    assert b0[0] == 0.0 and b1[0] == 0.0
    rel = np.linalg.norm(b1 - b0) / np.linalg.norm(b0)
    assert 0.0 < rel < 0.2  # slowly varying sequence
    c3 = make_config(1, size=6)
    assert np.linalg.norm(c3.rhs(2) - c3.rhs(0)) > 0


def test_random_operator_structure():
    g = Grid(4, 3, 5, (True, False, True))
    coef = random_operator(g, 19, np.random.default_rng(1))
    for s in range(1, 19):
        assert np.all(coef[s][~g.band_valid(s).reshape(-1)] == 0.0)
    assert np.all(coef[0] > np.abs(coef[1:]).sum(axis=0))
