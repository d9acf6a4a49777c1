"""Host logic of bench.py's roofline: the instruction count of the
sub-domain local sweeps (separable per-axis sums) against a direct
enumeration of boxes and grown-box cells."""
import itertools

import pytest

import bench
from problems import Grid


def _direct(grid, S, df):
    box, ov = (16, 8, 8), 1
    dims = (grid.nx, grid.ny, grid.nz)
    first, per_cell = (14, 4 + 12 * (S - 1) + 3 * (1 if S == 7 else 3) + 11 + 7 + 15) if df else (2, S + 3)
    total = 0
    starts = [range(0, n, b) for n, b in zip(dims, box)]
    for x0, y0, z0 in itertools.product(*starts):
        grown = 1
        owned = 1
        for c0, n, b, per in zip((x0, y0, z0), dims, box, grid.periodic):
            w = min(b, n - c0)
            cells = [c for c in range(c0 - ov, c0 + w + ov) if per or 0 <= c < n]
            grown *= len(cells)
            owned *= w
        total += first * grown + 3 * per_cell * grown + per_cell * owned
    return float(total)


@pytest.mark.parametrize("dims,per", [((37, 19, 11), (False, False, False)), ((40, 16, 17), (True, False, True)),
                                      ((16, 8, 8), (True, True, True)), ((2, 3, 4), (True, True, False))])
@pytest.mark.parametrize("S", [7, 19])
@pytest.mark.parametrize("df", [False, True])
def test_subdomain_instruction_count(dims, per, S, df):
    g = Grid(*dims, per)
    assert bench.subdomain_ops(g, S, df) == _direct(g, S, df)
