"""The oracle reproduces its stored fixtures (guards against silent drift)."""
import os

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    path = os.path.join(HERE, f"{name}_solution.txt")
    inertia = None
    with open(path) as f:
        for line in f:
            if line.startswith("# inertia"):
                inertia = [int(v) for v in line.split()[2:]]
    x = np.loadtxt(path, comments="#")
    return x, inertia


@pytest.mark.parametrize("name", ["tiny", "grid30_n24"])
def test_oracle_matches_golden(name):
    p = make_problem(CONFIGS[name])
    x, inertia = load_golden(name)
    out = oracle.kkt_solve(p)
    assert list(out["inertia"]) == inertia
    assert np.allclose(out["x"], x, rtol=1e-12, atol=1e-14 * np.abs(x).max())
