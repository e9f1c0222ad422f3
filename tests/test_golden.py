"""The FP64 oracle against its stored regression values (tests/golden/, written
by tests/golden/make_golden.py from the oracle alone).  A change of the
oracle's arithmetic shows up here; its commit must name the passage of the
paper, or the reading of it, that justifies the change."""

import json
import os

import pytest

from tests.golden import make_golden

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _close(a, b, path):
    if isinstance(a, dict):
        assert sorted(a) == sorted(b), path
        for k in a:
            _close(a[k], b[k], f"{path}.{k}")
    elif isinstance(a, list):
        assert len(a) == len(b), path
        for i, (x, y) in enumerate(zip(a, b)):
            _close(x, y, f"{path}[{i}]")
    elif isinstance(a, int) and isinstance(b, int):
        assert a == b, path
    else:
        assert abs(a - b) <= 1e-9 * max(1.0, abs(b)), (path, a, b)


def test_oracle_matches_stored_regression_values():
    with open(os.path.join(HERE, "oracle_regression.json")) as f:
        want = json.load(f)
    _close(make_golden.compute(), want, "oracle")
