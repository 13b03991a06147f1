"""Pins of the oracle's slack elimination (oracle/slack.py, Sec. 2) on the CPU.

The reduction (eq. SCOPFhessianReduced) and the recovery (eqs.
SCOPFslackReduction, SCOPFhessianSymmetricRecovery) are checked against the
unreduced Newton system of eq. SCOPFhessian, assembled densely and solved by
LAPACK: the reduced solution and the recovered slacks and bound multipliers
must together be the solution of the full system.  A dropped term or a wrong
sign in any of the six block rows breaks that equality.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, GridSpec, make_ipm_state, make_problem
from oracle import slack
from tests.kkt_dense import dense_K

EPS = np.finfo(np.float64).eps

CASES = {
    "tiny_L4": (CONFIGS["tiny"], 4),
    "small_L10": (CONFIGS["small"], 10),
    "st20_L26": (GridSpec(20, 26, 4, 3, 6, 1e-4, 1e4, 5, "st20"), 26),
}


def _split(p, st, full, ix):
    N, nP, nC, L = p.N, p.nP, p.nC, st.n_ineq
    nx = N * nP + nC
    nE = p.nA - p.nP - L
    return {"dx": full[ix["x"]:ix["x"] + nx], "ds": full[ix["s"]:ix["s"] + N * L],
            "dlE": full[ix["lE"]:ix["lE"] + N * nE], "dlI": full[ix["lI"]:ix["lI"] + N * L],
            "dz": full[ix["z"]:ix["z"] + nx], "dy": full[ix["y"]:ix["y"] + N * L]}


@pytest.mark.parametrize("case", sorted(CASES))
def test_reduction_and_recovery_solve_the_unreduced_system(case):
    spec, L = CASES[case]
    p = make_problem(spec, flow_limits=L)
    st = make_ipm_state(p, 17)
    a, c, rhs = slack.slack_reduce(p, st)
    pr = replace(p, a_vals=a, c_vals=c, rhs=rhs)
    K = dense_K(pr)
    xr = np.linalg.solve(K, rhs)
    # the oracle's Schur-complement solve of the reduced K agrees with LAPACK
    xo = oracle.kkt_solve(pr)["x"]
    assert np.max(np.abs(xo - xr)) <= 1e3 * np.linalg.cond(K) * EPS * np.max(np.abs(xr))
    ds, dz, dy = slack.slack_recover(p, st, xr)
    M, r, ix = slack.unreduced_system(p, st)
    full = np.linalg.solve(M, r)
    want = _split(p, st, full, ix)
    kap = np.linalg.cond(M)
    tol = lambda v: 1e2 * kap * EPS * max(1.0, np.max(np.abs(v)))  # noqa: E731
    N, nP, nA = p.N, p.nP, p.nA
    blocks = xr[:N * nA].reshape(N, nA)
    dx = np.concatenate([blocks[:, :nP].reshape(-1), xr[N * nA:]])
    ineq = np.asarray(p.ineq_rows)
    eq = np.setdiff1d(np.arange(nP, nA), ineq)
    got = {"dx": dx, "dlE": blocks[:, eq].reshape(-1), "dlI": blocks[:, ineq].reshape(-1), "ds": ds, "dz": dz, "dy": dy}
    for k, v in want.items():
        assert np.max(np.abs(got[k] - v)) <= tol(v), k


def test_without_inequality_rows_only_the_bound_terms_enter():
    """L = 0: the primal diagonals take z/x, C takes z_g/x_g, the multiplier
    rows and the rest of A keep their base values, and the right-hand side is
    -(l_a + l_e/x) on the primal rows and -l_c on the others."""
    p = make_problem(CONFIGS["small"])
    st = make_ipm_state(p, 3)
    assert st.n_ineq == 0
    a, c, rhs = slack.slack_reduce(p, st)
    base = np.asarray(st.a_base)
    diff = a - base
    pos = np.asarray(p.bar_pos)
    N, nP, nA = p.N, p.nP, p.nA
    zb, xb = st.z[:N * nP].reshape(N, nP), st.x[:N * nP].reshape(N, nP)
    assert np.array_equal(a[:, pos], base[:, pos] + zb / xb)
    mask = np.ones(p.nnzA, bool)
    mask[pos] = False
    assert np.all(diff[:, mask] == 0.0)
    assert np.array_equal(c, st.z[N * nP:] / st.x[N * nP:])
    r = rhs[:N * nA].reshape(N, nA)
    assert np.array_equal(r[:, nP:], -st.lcd.reshape(N, nA - nP))
    assert np.array_equal(r[:, :nP], -(st.la[:N * nP].reshape(N, nP) + st.le[:N * nP].reshape(N, nP) / xb))
    ds, dz, dy = slack.slack_recover(p, st, rhs)
    assert ds.size == 0 and dy.size == 0 and dz.size == N * nP + p.nC


def test_generator_inequality_rows():
    """flow_limits=L appends L multiplier rows with the linearised flow
    pattern (4 entries and the diagonal) and leaves L = 0 instances as they were."""
    p0 = make_problem(CONFIGS["grid30_n24"])
    pL = make_problem(CONFIGS["grid30_n24"], flow_limits=12)
    assert pL.nA == p0.nA + 12 and list(pL.ineq_rows) == list(range(p0.nA, p0.nA + 12))
    rp = np.asarray(pL.a_rowptr)
    for r in pL.ineq_rows:
        assert rp[r + 1] - rp[r] == 5
    q = make_problem(CONFIGS["grid30_n24"], flow_limits=0)
    assert np.array_equal(q.a_vals, p0.a_vals) and np.array_equal(q.rhs, p0.rhs)
    with pytest.raises(ValueError):
        make_problem(CONFIGS["tiny"], flow_limits=100)
