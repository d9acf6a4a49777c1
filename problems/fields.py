"""Smooth random fields and divergence right-hand sides.

The paper's right-hand sides are local balances of intermediate volume fluxes
at cell faces (eq. 1 and the text after it, Sec. 2.1); between time steps the
matrix is fixed and only b changes slowly (Sec. 1, Sec. 3). These helpers
make seeded stand-ins: Gaussian-filtered N(0,1) noise (truncated at 4 sigma,
reflecting at walls, wrapping on periodic axes, normalised to unit RMS) and
the discrete divergence of such face-velocity fields.
"""
import numpy as np
from scipy.ndimage import gaussian_filter


def rng_for(seed: int, *tags: int) -> np.random.Generator:
    """Independent PCG64 stream for (seed, tags...). Random access by tag
    (e.g. the time-step index) without drawing earlier streams."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed)] + [int(t) for t in tags])))


def smooth_noise(shape3, sigma: float, rng: np.random.Generator, wrap=(False, False, False)) -> np.ndarray:
    """Gaussian-filtered N(0,1) field of shape (nz, ny, nx), unit RMS.

    ``wrap`` is given per (x, y, z) axis; wrapped axes filter periodically,
    the others reflect."""
    x = rng.standard_normal(shape3)
    modes = ["wrap" if wrap[2] else "reflect", "wrap" if wrap[1] else "reflect", "wrap" if wrap[0] else "reflect"]
    y = gaussian_filter(x, sigma=sigma, mode=modes, truncate=4.0)
    rms = np.sqrt(np.mean(y * y))
    return y / rms


def face_velocity(grid, sigma: float, rng: np.random.Generator, walls=(False, True, True)):
    """Smoothed random face-normal velocities (ux, uy, uz).

    Axis a has n_a faces when periodic (face n_a is face 0) and n_a + 1
    otherwise. Faces on a wall (``walls[a]``) carry zero normal velocity; open
    non-periodic boundaries (inflow/outflow) keep their values."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    per = grid.periodic
    out = []
    for a, (n_a, p_a) in enumerate(((nx, per[0]), (ny, per[1]), (nz, per[2]))):
        dims = [nx, ny, nz]
        dims[a] = n_a if p_a else n_a + 1
        shape3 = (dims[2], dims[1], dims[0])
        u = smooth_noise(shape3, sigma, rng, wrap=per)
        if not p_a and walls[a]:
            sl = [slice(None)] * 3
            ax = 2 - a
            sl[ax] = 0
            u[tuple(sl)] = 0.0
            sl[ax] = -1
            u[tuple(sl)] = 0.0
        out.append(u)
    return out


def divergence(grid, hx, hy, hz, ux, uy, uz) -> np.ndarray:
    """Per-unit-volume discrete divergence: (1/V_P) * sum of outward face fluxes."""
    per = grid.periodic
    hx = np.asarray(hx, float)
    hy = np.asarray(hy, float)
    hz = np.asarray(hz, float)
    HX = hx[None, None, :]
    HY = hy[None, :, None]
    HZ = hz[:, None, None]
    vol = HX * HY * HZ

    def diff(u, axis, periodic):
        if periodic:
            return np.roll(u, -1, axis=axis) - u
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[axis] = slice(1, None)
        sl_lo[axis] = slice(0, -1)
        return u[tuple(sl_hi)] - u[tuple(sl_lo)]

    flux = diff(ux, 2, per[0]) * (HY * HZ) + diff(uy, 1, per[1]) * (HX * HZ) + diff(uz, 0, per[2]) * (HX * HY)
    return flux / vol


def normalise_div(d: np.ndarray, vol: np.ndarray) -> np.ndarray:
    """Remove the volume-weighted mean and scale to unit RMS."""
    d = d - np.sum(d * vol) / np.sum(vol)
    return d / np.sqrt(np.mean(d * d))


def divergence_sequence(grid, hx, hy, hz, sigma, seed, t, walls=(False, True, True), weight=0.05):
    """b_t of the slowly varying sequence b_0 = D(u_0), b_{t+1} = b_t + w*D(u_{t+1}).

    D is the normalised divergence of an independent smoothed face-velocity
    field per step. Returns the (nz, ny, nx) array for step ``t``."""
    vol = (np.asarray(hz, float)[:, None, None] * np.asarray(hy, float)[None, :, None]
           * np.asarray(hx, float)[None, None, :])
    b = None
    for s in range(t + 1):
        u = face_velocity(grid, sigma, rng_for(seed, 7, s), walls=walls)
        d = normalise_div(divergence(grid, hx, hy, hz, *u), vol)
        b = d if b is None else b + weight * d
    return b
