"""The CUDA path on the other input families: the paper's own MPOPF coupling
(Sec. 4.1, eq. B12N: C = 0, dense negative definite S) and the SCOPF workload
(Sec. 3.1: scenario blocks, dense C).  Each solution meets the refinement
target against the oracle's residual, matches the oracle's solution within
the conditioning bound, and the pivot signs give the inertia of K."""
import numpy as np
import pytest

import oracle
from gen import CONFIGS, GridSpec, make_problem, make_scopf
from kkt_dense import dense_K

pytestmark = pytest.mark.gpu


def _solve(p, prec, **opts):
    from paper_1907_05420_gb300 import binding as B

    h = B.kkt_analyze(p, B.kkt_default_options(prec, **opts))
    try:
        B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                     np.ascontiguousarray(p.c_vals))
        x = np.empty(p.nK)
        B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
        info = B.kkt_get_info(h)
    finally:
        B.kkt_destroy(h)
    return x, info


CASES = {
    "paper_tiny": lambda: make_problem(CONFIGS["tiny"], coupling="paper"),
    "paper_grid30": lambda: make_problem(CONFIGS["grid30_n24"], coupling="paper"),
    "scopf14": lambda: make_scopf(GridSpec(14, 20, 5, 0, 1, 1e-4, 1e4, 5, "scopf14"), 4),
    "scopf30": lambda: make_scopf(GridSpec(30, 41, 6, 0, 1, 1e-6, 1e6, 7, "scopf30"), 8),
}


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_other_input_families(name, prec):
    p = CASES[name]()
    # TF32: GMRES refinement to 1e-12, so that the forward-error bound below means something
    tight = {"refine_mode": 1, "refine_tol": 1e-12} if prec == "tf32" else {}
    x, info = _solve(p, prec, **tight)
    eta = oracle.backward_error(p, x)
    assert eta <= (1e-12 if tight else 1e-10), eta
    ref = oracle.kkt_solve(p)
    kappa = np.linalg.cond(dense_K(p))
    err = np.max(np.abs(x - ref["x"])) / np.max(np.abs(ref["x"]))
    # the forward error is bounded only while kappa * eta is small
    bound = 10 * kappa * max(eta, np.finfo(np.float64).eps)
    if bound < 0.5:
        assert err <= 2 * bound, (err, kappa, eta)
    if prec == "fp64":
        assert [info["n_pos"], info["n_neg"], info["n_zero"]] == list(ref["inertia"])
