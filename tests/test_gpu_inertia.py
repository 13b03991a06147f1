"""Inertia correction (Sec. 2, inertia correction and curvature detection).

kkt_factor_inertia refactors K + diag(dw I on the primal rows and on C, -dc I
on the dual rows) with growing trial shifts until the pivot signs give the
inertia (N nP + nC, N nD, 0).  The trial sequence is fixed by the options, so
the accepted shift is the first trial value whose shifted K has that inertia;
the tests find that value from the eigenvalues of the dense K (numpy, on
systems small enough to assemble) and compare.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem
from kkt_dense import dense_K

pytestmark = pytest.mark.gpu


def _diag_positions(p):
    pos = np.empty(p.nA, dtype=np.int64)
    for r in range(p.nA):
        cols = p.a_col[p.a_rowptr[r]:p.a_rowptr[r + 1]]
        pos[r] = p.a_rowptr[r] + int(np.nonzero(cols == r)[0][0])
    return pos


def shifted(p, dw, dc=0.0):
    """p with dw added to every primal diagonal and to C's, dc subtracted from
    every dual diagonal."""
    pos = _diag_positions(p)
    a = np.array(p.a_vals, dtype=np.float64, copy=True)
    a[:, pos[:p.nP]] += dw
    a[:, pos[p.nP:]] -= dc
    c = np.array(p.c_vals, dtype=np.float64, copy=True)
    if p.c_kind == 0:
        c += dw
    else:
        c.reshape(p.nC, p.nC)[np.diag_indices(p.nC)] += dw
    return replace(p, a_vals=a, c_vals=c)


def eig_inertia(p):
    w = np.linalg.eigvalsh(dense_K(p))
    tol = 1e-13 * np.abs(w).max()
    return int((w > tol).sum()), int((w < -tol).sum()), int((np.abs(w) <= tol).sum())


def expected(p):
    return p.N * p.nP + p.nC, p.N * (p.nA - p.nP), 0


def first_accepted(p, trials):
    """Index and value of the first trial shift with the expected inertia."""
    for i, d in enumerate(trials):
        if eig_inertia(shifted(p, d)) == expected(p):
            return i, d
    raise AssertionError("no trial shift gives the expected inertia")


def _factor(B, p, prec, h=None, **kw):
    if h is None:
        h = B.kkt_analyze(p, B.kkt_default_options(prec))
    res = B.kkt_factor_inertia(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                               np.ascontiguousarray(p.c_vals), B.kkt_default_inertia_options(**kw))
    return h, res


@pytest.mark.parametrize("prec", ["fp64", "tf32", "f64emu"])
def test_no_shift_when_inertia_is_right(prec):
    """A system with the expected inertia is factored once, unshifted, and (in
    FP64) gives bitwise the solution of kkt_factor."""
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["small"])
    assert eig_inertia(p) == expected(p)
    h, res = _factor(B, p, prec)
    try:
        assert res["trials"] == 1 and res["delta_w"] == 0.0 and res["delta_c"] == 0.0
        x = np.empty(p.nK)
        B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
        info = B.kkt_get_info(h)
        assert (info["n_pos"], info["n_neg"], info["n_zero"]) == expected(p)
        assert oracle.backward_error(p, x) <= 1e-10
        if prec == "fp64":
            h2 = B.kkt_analyze(p, B.kkt_default_options(prec))
            try:
                B.kkt_factor(h2, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                             np.ascontiguousarray(p.c_vals))
                x2 = np.empty(p.nK)
                B.kkt_solve(h2, np.ascontiguousarray(p.rhs), x2)
            finally:
                B.kkt_destroy(h2)
            assert np.array_equal(x, x2)
    finally:
        B.kkt_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
@pytest.mark.parametrize("name,s", [("tiny", 5.0), ("small", 2.0)])
def test_negative_curvature_is_shifted_away(prec, name, s):
    """Primal diagonals lowered by s give K too many negative eigenvalues.  The
    first call accepts the first trial of delta_w_init * grow_first^k with the
    right inertia; a second call on the handle starts from shrink * that shift
    and grows by `grow`.  The solution solves the shifted system."""
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS[name])
    q = shifted(p, -s)
    assert eig_inertia(q) != expected(q)
    o = B.kkt_default_inertia_options()
    first = [o.delta_w_init * o.grow_first ** k for k in range(8)]
    i1, d1 = first_accepted(q, first)
    h, res = _factor(B, q, prec)
    try:
        assert res["delta_w"] == pytest.approx(d1, rel=1e-12) and res["trials"] == i1 + 2
        assert res["delta_c"] == 0.0
        info = B.kkt_get_info(h)
        assert (info["n_pos"], info["n_neg"], info["n_zero"]) == expected(q)
        x = np.empty(q.nK)
        B.kkt_solve(h, np.ascontiguousarray(q.rhs), x)
        assert oracle.backward_error(shifted(q, res["delta_w"]), x) <= 1e-10

        second = [max(o.delta_w_min, o.shrink * res["delta_w"]) * o.grow ** k for k in range(8)]
        i2, d2 = first_accepted(q, second)
        _, res2 = _factor(B, q, prec, h=h)
        assert res2["delta_w"] == pytest.approx(d2, rel=1e-12) and res2["trials"] == i2 + 2
    finally:
        B.kkt_destroy(h)


def test_gives_up_within_the_limits():
    """With delta_w_max below the needed shift the call reports
    KKT_ERR_INERTIA after the trials it may take."""
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["tiny"])
    q = shifted(p, -5.0)
    h = B.kkt_analyze(q, B.kkt_default_options("fp64"))
    try:
        res = B.kkt_factor_inertia(h, np.ascontiguousarray(q.a_vals), np.ascontiguousarray(q.b_vals),
                                   np.ascontiguousarray(q.c_vals),
                                   B.kkt_default_inertia_options(delta_w_max=1.0), allow_wrong_inertia=True)
        assert res["status"] == 5
        assert res["trials"] == 4 and res["delta_w"] == pytest.approx(1.0)  # 0, 1e-4, 1e-2, 1
    finally:
        B.kkt_destroy(h)
