"""Structured grid and band geometry.

Band order (fixed by this package and restated, independently, by every
consumer): 0 centre; 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z; then the xy edges
7 (-1,-1,0), 8 (+1,-1,0), 9 (-1,+1,0), 10 (+1,+1,0); the xz edges
11 (-1,0,-1), 12 (+1,0,-1), 13 (-1,0,+1), 14 (+1,0,+1); the yz edges
15 (0,-1,-1), 16 (0,+1,-1), 17 (0,-1,+1), 18 (0,+1,+1).
A 7-point operator uses bands 0-6, a 19-point operator all 19 (the paper's
7- and 19-point stencils for orthogonal and non-orthogonal grids, Sec. 2.1).
"""
from dataclasses import dataclass

import numpy as np

OFFSETS = (
    (0, 0, 0),
    (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1),
    (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 1, 0),
    (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (1, 0, 1),
    (0, -1, -1), (0, 1, -1), (0, -1, 1), (0, 1, 1),
)
S7 = 7
S19 = 19


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    periodic: tuple = (False, False, False)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape3(self):
        """Array shape (nz, ny, nx): x is the fastest (last) axis."""
        return (self.nz, self.ny, self.nx)

    def band_valid(self, s: int) -> np.ndarray:
        """Boolean (nz, ny, nx): True where band s points at a cell inside the
        domain (or wraps on a periodic axis)."""
        dx, dy, dz = OFFSETS[s]
        ok = np.ones(self.shape3, dtype=bool)
        for d, n, per, ax in ((dx, self.nx, self.periodic[0], 2),
                              (dy, self.ny, self.periodic[1], 1),
                              (dz, self.nz, self.periodic[2], 0)):
            if d == 0 or per:
                continue
            idx = np.arange(n)
            good = (idx + d >= 0) & (idx + d < n)
            shape = [1, 1, 1]
            shape[ax] = n
            ok = ok & good.reshape(shape)
        return ok
