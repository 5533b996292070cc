"""Shared pytest set-up: repository root on sys.path, the `gpu` marker, fixtures."""
import os
import sys
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbsc.so")


def read_golden(name):
    """Rows of a whitespace-separated golden file, comments dropped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def table1():
    """Table 1 as a list of (belt, |c|^2, links, Fraction p)."""
    return [(b, int(e), int(n), Fraction(p)) for b, e, n, p in read_golden("table1_weights.txt")]


@pytest.fixture(scope="session")
def d2q9():
    return [(int(e), int(n), Fraction(w)) for e, n, w in read_golden("d2q9_weights.txt")]


@pytest.fixture(scope="session")
def constants():
    out = {}
    for row in read_golden("paper_constants.txt"):
        out[row[0]] = row[1]
    return out
