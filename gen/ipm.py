"""A seeded interior-point iterate for the slack elimination (Sec. 2).

For a system built with inequality rows (make_problem(..., flow_limits=L)),
the state of the barrier method at one iteration: the primal variables x and
their bound multipliers z (every primal variable of every period and every
coupling variable has a bound), the slacks s of the inequality rows and their
bound multipliers y, and the residuals l_a .. l_f of the primal-dual
equations (eq. OC).  x, z, s, y are positive: z/x is log-uniform over the
instance's barrier range (the values the plain instances put on the primal
diagonal), y/s log-uniform in [1e-2, 1e2]; the residuals are N(0, 1).  The
base values are those of the blocks and of C without any barrier term: H and
J as the instance has them, the dual regularisation -1e-8 on the multiplier
rows, and C = 0.

This module only draws inputs; the elimination itself is the solver's (and
the oracle's).
"""
from __future__ import annotations

import types

import numpy as np

from .mpopf import KKTProblem, _loguniform


def make_ipm_state(prob: KKTProblem, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    N, nP, nA, nC = prob.N, prob.nP, prob.nA, prob.nC
    L = 0 if prob.ineq_rows is None else len(prob.ineq_rows)
    nx = N * nP + nC
    x = _loguniform(rng, 1e-2, 1.0, nx)
    z = x * _loguniform(rng, prob.spec.bar_lo, prob.spec.bar_hi, nx)
    s = _loguniform(rng, 1e-2, 1.0, N * L)
    y = s * _loguniform(rng, 1e-2, 1e2, N * L)
    la = rng.standard_normal(nx)
    le = rng.standard_normal(nx)
    lcd = rng.standard_normal(N * (nA - nP))  # l_c on the equality rows, l_d on the inequality rows
    lb = rng.standard_normal(N * L)
    lf = rng.standard_normal(N * L)
    a_base = np.broadcast_to(prob.a_const, (N, prob.nnzA)).copy()
    c_base = np.zeros(nC)
    return types.SimpleNamespace(x=x, z=z, s=s, y=y, la=la, lcd=lcd, lb=lb, le=le, lf=lf,
                                 a_base=a_base, c_base=c_base, n_ineq=L)
