"""The oracle against its frozen fixtures (tests/golden/oracle_tiny.json,
written by tests/golden/make_golden.py from the oracle alone): stencil
products, residual and the sub-domain preconditioner bit for bit. A change
of the oracle's arithmetic shows up here and has to come with regenerated
fixtures and its reason."""
import json
import os

import numpy as np
import pytest

from golden.make_golden import cases, compute

HERE = os.path.dirname(os.path.abspath(__file__))

with open(os.path.join(HERE, "golden", "oracle_tiny.json")) as f:
    GOLD = json.load(f)


@pytest.mark.parametrize("case", cases(), ids=[c[0] for c in cases()])
def test_oracle_matches_frozen_fixtures(case):
    name = case[0]
    assert compute(*case) == GOLD[name]


def test_fixtures_cover_every_case():
    assert sorted(GOLD) == sorted(c[0] for c in cases())
    for rec in GOLD.values():
        assert set(rec) == {"apply", "apply_prec", "apply_left", "residual", "schwarz"}
