"""Dense matrix of a banded operator by brute force (test infrastructure).

Walks every cell and every band with plain Python index arithmetic, written
independently of stencil.c, so that the C loops can be pinned against
``dense_matrix(...) @ v`` on tiny grids."""
import numpy as np

_OFF = (
    (0, 0, 0),
    (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1),
    (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 1, 0),
    (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (1, 0, 1),
    (0, -1, -1), (0, 1, -1), (0, -1, 1), (0, 1, 1),
)


def dense_matrix(grid, coef) -> np.ndarray:
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    n = nx * ny * nz
    S = coef.shape[0]
    A = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = i + nx * (j + ny * k)
                for s in range(S):
                    c = coef[s, row]
                    ii, jj, kk = i + _OFF[s][0], j + _OFF[s][1], k + _OFF[s][2]
                    inside = True
                    for val, lim, per, name in ((ii, nx, grid.periodic[0], "x"),
                                                (jj, ny, grid.periodic[1], "y"),
                                                (kk, nz, grid.periodic[2], "z")):
                        if not (0 <= val < lim) and not per:
                            inside = False
                    if not inside:
                        assert c == 0.0, f"band {s} of cell {row} points outside but is {c}"
                        continue
                    col = (ii % nx) + nx * ((jj % ny) + ny * (kk % nz))
                    A[row, col] += c
    return A
