"""Writes the frozen oracle fixtures of tests/test_golden.py (oracle_tiny.json).

Calls only oracle/ (and the seeded input generators of problems/): every
stored value is the oracle's, as exact hex floats. The fixtures make any later
change of the oracle's arithmetic visible: test_golden.py recomputes them and
compares bit for bit, so such a change must come with regenerated fixtures
and a stated reason.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from problems import Grid, make_config, random_operator  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json")


def hexlist(a):
    return [float(v).hex() for v in np.asarray(a, dtype=np.float64).ravel()]


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<f8").tobytes()).hexdigest()


def cases():
    """(name, grid, coef, v, b): the inputs, from the seeded generators."""
    out = []
    g = Grid(5, 4, 3, (True, False, True))
    for S in (7, 19):
        coef = random_operator(g, S, np.random.default_rng(100 + S))
        v = np.random.default_rng(200 + S).standard_normal(g.n)
        b = np.random.default_rng(300 + S).standard_normal(g.n)
        out.append((f"random{S}", g, coef, v, b))
    c = make_config(1, size=5)
    out.append(("convdiff5", c.grid, c.coef, c.rhs(1), c.rhs(0)))
    c = make_config(2, size=6)
    out.append(("channel6", c.grid, c.coef, c.rhs(1), c.rhs(0)))
    return out


def compute(name, grid, coef, v, b):
    """The oracle's C loops only (the products, the residual and the
    sub-domain preconditioner): IEEE arithmetic in a fixed order with explicit
    fma and no contraction, so the values are the same on every machine.
    Full hex values for grids of at most 64 cells, SHA-256 digests of the
    little-endian FP64 bytes otherwise."""
    op = oracle.Stencil(grid, coef)
    outs = {
        "apply": op.apply(v),
        "apply_prec": op.apply_prec(v),
        "apply_left": op.apply_left(v),
        "residual": op.residual(b, v),
        "schwarz": op.schwarz(v),
    }
    if grid.n <= 64:
        return {k: hexlist(a) for k, a in outs.items()}
    return {k: {"sha256": digest(a), "head": hexlist(a[:4])} for k, a in outs.items()}


def main():
    data = {name: compute(name, g, c, v, b) for name, g, c, v, b in cases()}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
