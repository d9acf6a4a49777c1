"""The five synthetic workloads (seeded) that stand in for the paper's runs.

1. 32^3 convection-diffusion, 7 points, 5 right-hand sides (GMRES(30) vs
   rGCROT(30,10)).
2. 128^3 wall-refined channel (periodic x, z; Neumann walls), 7 points,
   50 steps; the stand-in for the paper's turbulent channel (Sec. 3.1).
3. 192^3 skewed porous medium (spheres of low conductivity), 19 points,
   100 steps; the stand-in for the paper's porous-medium flow (Sec. 3.2).
4. 64 uneven porous problems with 20 right-hand sides each (batched).
5. 32 resident problems for the serving loop.

The seed of config i is ``CONFIG_SEED_BASE + i``. A ``size`` argument shrinks
the grid (same generator, same structure) for tests.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from .fields import rng_for, smooth_noise, face_velocity, divergence, normalise_div
from .grid import Grid
from .operators import convection_diffusion_7pt, channel_7pt, porous_skew_19pt, sphere_pack

CONFIG_SEED_BASE = 20150113


@dataclass
class ConfigProblem:
    name: str
    grid: Grid
    S: int
    coef: np.ndarray
    solver: dict
    n_steps: int
    seed: int
    rhs_kind: str
    rhs_args: dict = field(default_factory=dict)
    pinned: bool = False
    solid_fraction: float = float("nan")
    _cache: dict = field(default_factory=dict, repr=False)

    @property
    def n(self):
        return self.grid.n

    def rhs(self, t: int) -> np.ndarray:
        """Right-hand side of time step t, flat float64 of length N."""
        if self.rhs_kind == "noise":
            g = self.grid
            f0 = smooth_noise(g.shape3, self.rhs_args["sigma"], rng_for(self.seed, 5, 0), wrap=g.periodic)
            if t == 0:
                b = f0
            else:
                ft = smooth_noise(g.shape3, self.rhs_args["sigma"], rng_for(self.seed, 5, t), wrap=g.periodic)
                b = f0 + 0.05 * t * ft
            return np.ascontiguousarray(b.reshape(-1))
        # divergence recurrence b_0 = D(u_0), b_{t+1} = b_t + 0.05 D(u_{t+1})
        start, b = self._cache.get("last", (-1, None))
        if start > t:
            start, b = -1, None
        a = self.rhs_args
        vol = (a["hz"][:, None, None] * a["hy"][None, :, None] * a["hx"][None, None, :])
        for s in range(start + 1, t + 1):
            u = face_velocity(self.grid, a["sigma"], rng_for(self.seed, 7, s), walls=a["walls"])
            d = normalise_div(divergence(self.grid, a["hx"], a["hy"], a["hz"], *u), vol)
            b = d if b is None else b + 0.05 * d
        self._cache["last"] = (t, b)
        out = np.ascontiguousarray(b.reshape(-1)).copy()
        if self.pinned:
            out[0] = 0.0
        return out


def _unit_vector(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def config1(seed=None, size=32):
    seed = CONFIG_SEED_BASE + 1 if seed is None else seed
    c = 0.5 * _unit_vector(rng_for(seed, 1))
    grid, coef = convection_diffusion_7pt(size, c)
    return ConfigProblem("convdiff32", grid, 7, coef,
                         dict(mode="rGCROT", m=30, k=10, tol=1e-8, compare=[("GMRES", 30, 0)]),
                         5, seed, "noise", dict(sigma=3.0))


def config2(seed=None, size=128):
    seed = CONFIG_SEED_BASE + 2 if seed is None else seed
    grid, coef, (hx, hy, hz) = channel_7pt(size, size, size, beta=2.0)
    return ConfigProblem("channel128", grid, 7, coef,
                         dict(mode="rGCROT", m=40, k=20, tol=1e-8,
                              compare=[("GMRES", 40, 0), ("BiCGStab", 0, 0)]),
                         50, seed, "div", dict(sigma=8.0, hx=hx, hy=hy, hz=hz, walls=(False, True, False)),
                         pinned=True)


def porous_problem(n_xyz, fraction, skew_deg, seed, radius=6.0, max_attempts=1_000_000):
    solid, frac = sphere_pack(n_xyz, radius, fraction, rng_for(seed, 3), max_attempts=max_attempts)
    kappa = np.where(solid, 1e-4, 1.0)
    grid, coef = porous_skew_19pt(n_xyz, kappa, skew_deg)
    return grid, coef, frac


def config3(seed=None, size=192, max_attempts=1_000_000):
    seed = CONFIG_SEED_BASE + 3 if seed is None else seed
    n = (size, size, size)
    grid, coef, frac = porous_problem(n, 0.4, 15.0, seed, max_attempts=max_attempts)
    ones = lambda k: np.ones(k)
    return ConfigProblem("porous192", grid, 19, coef,
                         dict(mode="hybrid", m=40, k=20, tol=1e-8, hybrid_switch=5),
                         100, seed, "div",
                         dict(sigma=8.0, hx=ones(size), hy=ones(size), hz=ones(size), walls=(False, True, True)),
                         solid_fraction=frac)


def config4_problem(p: int, seed=None, max_edge=96, min_edge=24):
    """Problem p (0..63) of the batched uneven set."""
    seed = CONFIG_SEED_BASE + 4 if seed is None else seed
    rng = rng_for(seed, 11, p)
    edges = tuple(int(round(math.exp(rng.uniform(math.log(min_edge), math.log(max_edge))))) for _ in range(3))
    frac = rng.uniform(0.1, 0.4)
    skew = rng.uniform(0.0, 15.0)
    grid, coef, got = porous_problem(edges, frac, skew, seed * 131 + p, max_attempts=200_000)
    ones = lambda k: np.ones(k)
    return ConfigProblem(f"batch{p}", grid, 19, coef,
                         dict(mode="hybrid", m=40, k=10, tol=1e-8, hybrid_switch=5),
                         20, seed * 131 + p, "div",
                         dict(sigma=4.0, hx=ones(edges[0]), hy=ones(edges[1]), hz=ones(edges[2]),
                              walls=(False, True, True)),
                         solid_fraction=got)


def make_config(i: int, seed=None, size=None, **kw) -> ConfigProblem:
    """Config i (1-based, as listed in the module docstring)."""
    if i == 1:
        return config1(seed, size or 32)
    if i == 2:
        return config2(seed, size or 128)
    if i == 3:
        return config3(seed, size or 192, **kw)
    if i == 4:
        return config4_problem(kw.get("p", 0), seed)
    raise ValueError(f"unknown config {i}")
