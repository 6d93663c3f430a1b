"""Shared test helpers.

Tests marked ``gpu`` need a CUDA device and the compiled library; the rest run
on the CPU (oracle pins, host logic, library loading and exported symbols).
"""
from __future__ import annotations

import ast
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled bsort library")


def load_golden():
    """Parses ``tests/golden/*.txt`` into dicts (text, W, words, perm, counts...)."""
    cases = []
    for name in sorted(os.listdir(GOLDEN)):
        if not name.endswith(".txt"):
            continue
        d = {"name": name[:-4]}
        with open(os.path.join(GOLDEN, name)) as f:
            for line in f:
                line = line.rstrip("\n")
                if not line or line.startswith("#"):
                    continue
                k, _, v = line.partition("=")
                k, v = k.strip(), v.strip()
                if k in ("text", "packed"):
                    d[k] = ast.literal_eval(v)
                elif k in ("W", "status"):
                    d[k] = int(v)
                elif k == "words":
                    d[k] = [w.encode() for w in v.split()]
                elif k in ("perm", "offsets"):
                    d[k] = [int(x) for x in v.split()]
                elif k in ("counts", "swaps"):
                    d[k] = {int(a): int(b) for a, b in (p.split(":") for p in v.split())}
        d.setdefault("status", 0)
        cases.append(d)
    return cases


def sort_key_order(rec: np.ndarray, ln: np.ndarray) -> list[int]:
    """Indices ordered by (length, bytes, index), by Python's own sort."""
    n = ln.size
    return sorted(range(n), key=lambda i: (int(ln[i]), bytes(rec[i, :ln[i]]), i))


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
