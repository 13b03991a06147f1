"""Slack elimination and recovery (Sec. 2) in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY: the test-suite uses it; the library's product path
never imports it.

The barrier method's Newton system (eq. SCOPFhessian) has the unknowns
(dx, ds, dlE, dlI, dz, dy) and the rows

    (a)  H dx + JE^T dlE + JI^T dlI - dz = -l_a
    (b)  -dlI - dy                       = -l_b
    (c)  JE dx                           = -l_c
    (d)  JI dx - ds                      = -l_d
    (e)  Z dx + X dz                     = -l_e
    (f)  Y ds + S dy                     = -l_f

Eliminating (e) and (f) gives the symmetric system of eq.
SCOPFhessianSymmetric, and eliminating the slacks (the diagonal block
L_s = S^-1 Y once the slacks are ordered last, eq. SCOPFslackAtEnd) gives the
reduced system of eq. SCOPFhessianReduced,

    [ H + X^-1 Z   JE^T   JI^T     ] [dx ]     [ l_a + X^-1 l_e                 ]
    [ JE           0      0        ] [dlE] = - [ l_c                            ]
    [ JI           0      -L_s^-1  ] [dlI]     [ l_d + L_s^-1 (l_b + S^-1 l_f)  ]

which is the arrowhead K of the solver: per period the primal rows of A_i
take H + X^-1 Z, the inequality rows take -L_s^-1 = -S Y^-1 on their diagonal
(any base value there is replaced), the equality rows keep their dual
regularisation (-1e-8, also on the lE diagonal of the full system below), and
the coupling variables, which are primal, take C + X_g^-1 Z_g.  The
eliminated unknowns come back from eq. SCOPFslackReduction and eq.
SCOPFhessianSymmetricRecovery:

    ds = L_s^-1 (dlI - l_b - S^-1 l_f),  dz = -X^-1 (l_e + Z dx),  dy = -S^-1 (l_f + Y ds).

Layouts (per block contiguous, block i first): x, z, l_a, l_e hold the nP
primal rows of every block and then the nC coupling variables; l_cd holds
the nA - nP multiplier rows of every block (l_d on the inequality rows, l_c
on the others); s, y, l_b, l_f the inequality rows of every block in the
order of prob.ineq_rows.  Parity pins: tests/test_oracle_slack.py.
"""
from __future__ import annotations

import numpy as np


def _maps(prob):
    ineq = np.asarray(prob.ineq_rows, dtype=np.int64)
    L = len(ineq)
    dual = np.arange(prob.nP, prob.nA)
    eq = np.setdiff1d(dual, ineq)
    return ineq, L, eq


def _diag_pos(prob):
    rp, col = np.asarray(prob.a_rowptr), np.asarray(prob.a_col)
    pos = np.empty(prob.nA, dtype=np.int64)
    for r in range(prob.nA):
        lo, hi = rp[r], rp[r + 1]
        j = lo + int(np.searchsorted(col[lo:hi], r))
        assert col[j] == r
        pos[r] = j
    return pos


def slack_reduce(prob, st):
    """(a_vals, c_vals, rhs) of the reduced system (eq. SCOPFhessianReduced)."""
    N, nP, nA, nC = prob.N, prob.nP, prob.nA, prob.nC
    ineq, L, _ = _maps(prob)
    dpos = _diag_pos(prob)
    a = np.array(st.a_base, dtype=np.float64, copy=True).reshape(N, -1)
    rhs = np.empty(N * nA + nC)
    xb = st.x[:N * nP].reshape(N, nP)
    zb = st.z[:N * nP].reshape(N, nP)
    lab = st.la[:N * nP].reshape(N, nP)
    leb = st.le[:N * nP].reshape(N, nP)
    lcd = st.lcd.reshape(N, nA - nP)
    s, y = st.s.reshape(N, L), st.y.reshape(N, L)
    lb, lf = st.lb.reshape(N, L), st.lf.reshape(N, L)
    for i in range(N):
        a[i, dpos[:nP]] += zb[i] / xb[i]                       # H + X^-1 Z
        a[i, dpos[ineq]] = -(s[i] / y[i])                      # -L_s^-1
        r = rhs[i * nA:(i + 1) * nA]
        r[:nP] = -(lab[i] + leb[i] / xb[i])                    # -(l_a + X^-1 l_e)
        r[nP:] = -lcd[i]                                       # -l_c
        r[ineq] = -(lcd[i, ineq - nP] + (s[i] / y[i]) * (lb[i] + lf[i] / s[i]))
    xg, zg = st.x[N * nP:], st.z[N * nP:]
    c = np.asarray(st.c_base, dtype=np.float64) + zg / xg
    rhs[N * nA:] = -(st.la[N * nP:] + st.le[N * nP:] / xg)
    return a, c, rhs


def slack_recover(prob, st, dsol):
    """(ds, dz, dy) from the reduced solution dsol = [dx_i, dl_i ..., dx_g]."""
    N, nP, nA = prob.N, prob.nP, prob.nA
    ineq, L, _ = _maps(prob)
    d = np.asarray(dsol).reshape(-1)
    blocks = d[:N * nA].reshape(N, nA)
    dx = np.concatenate([blocks[:, :nP].reshape(-1), d[N * nA:]])
    dlI = blocks[:, ineq].reshape(-1)
    s, y, lb, lf = st.s, st.y, st.lb, st.lf
    ds = (s / y) * (dlI - lb - lf / s)
    dz = -(st.le + st.z * dx) / st.x
    dy = -(lf + y * ds) / s
    return ds, dz, dy


def unreduced_system(prob, st):
    """The full Newton system (eq. SCOPFhessian, with the equality rows'
    regularisation), dense: (M, rhs, index maps).  Tiny inputs only."""
    N, nP, nA, nC = prob.N, prob.nP, prob.nA, prob.nC
    ineq, L, eq = _maps(prob)
    nE = len(eq)
    nx = N * nP + nC
    ix = {"x": 0, "s": nx, "lE": nx + N * L, "lI": nx + N * L + N * nE, "z": nx + N * L + N * (nE + L)}
    ix["y"] = ix["z"] + nx
    n = ix["y"] + N * L
    M = np.zeros((n, n))
    rhs = np.zeros(n)
    rp, col = np.asarray(prob.a_rowptr), np.asarray(prob.a_col)
    eq_of = {int(r): k for k, r in enumerate(eq)}
    in_of = {int(r): k for k, r in enumerate(ineq)}
    dual_diag = np.zeros(nA)

    def xi(i, r):  # primal row r of block i
        return ix["x"] + i * nP + r

    for i in range(N):
        av = np.asarray(st.a_base).reshape(N, -1)[i]
        for r in range(nA):
            for p in range(rp[r], rp[r + 1]):
                c_, v = int(col[p]), av[p]
                if r < nP:                       # H (lower triangle, mirrored)
                    M[xi(i, r), xi(i, c_)] += v
                    if c_ != r:
                        M[xi(i, c_), xi(i, r)] += v
                elif c_ < nP:                    # J: row r, primal column c_
                    if r in eq_of:
                        ml = ix["lE"] + i * nE + eq_of[r]
                    else:
                        ml = ix["lI"] + i * L + in_of[r]
                    M[ml, xi(i, c_)] += v        # (c)/(d): J dx
                    M[xi(i, c_), ml] += v        # (a): J^T dl
                elif c_ == r:
                    dual_diag[r] = v
        for r in eq:                             # (c): - delta dlE
            M[ix["lE"] + i * nE + eq_of[int(r)], ix["lE"] + i * nE + eq_of[int(r)]] = dual_diag[r]
    # B: (block i, multiplier row r) x coupling column c: part of JE (or JI)
    bp = np.asarray(prob.b_blockptr)
    for i in range(N):
        for q in range(bp[i], bp[i + 1]):
            r, c_, v = int(prob.b_row[q]), int(prob.b_col[q]), float(prob.b_vals[q])
            ml = ix["lE"] + i * nE + eq_of[r] if r in eq_of else ix["lI"] + i * L + in_of[r]
            M[ml, ix["x"] + N * nP + c_] += v
            M[ix["x"] + N * nP + c_, ml] += v
    cb = np.asarray(st.c_base, dtype=np.float64)
    for c_ in range(nC):
        M[ix["x"] + N * nP + c_, ix["x"] + N * nP + c_] += cb[c_]
    for k in range(nx):                          # (a): - dz ; (e): Z dx + X dz
        M[ix["x"] + k, ix["z"] + k] = -1.0
        M[ix["z"] + k, ix["x"] + k] = st.z[k]
        M[ix["z"] + k, ix["z"] + k] = st.x[k]
    for k in range(N * L):                       # (b): -dlI - dy ; (d): - ds ; (f): Y ds + S dy
        rb = ix["s"] + k                         # row (b) placed at the s index
        M[rb, ix["lI"] + k] = -1.0
        M[rb, ix["y"] + k] = -1.0
        M[ix["lI"] + k, ix["s"] + k] = -1.0
        M[ix["y"] + k, ix["s"] + k] = st.y[k]
        M[ix["y"] + k, ix["y"] + k] = st.s[k]
    rhs[ix["x"]:ix["x"] + nx] = -st.la
    rhs[ix["s"]:ix["s"] + N * L] = -st.lb
    lcd = st.lcd.reshape(N, nA - nP)
    for i in range(N):
        rhs[ix["lE"] + i * nE:ix["lE"] + (i + 1) * nE] = -lcd[i, eq - nP]
        rhs[ix["lI"] + i * L:ix["lI"] + (i + 1) * L] = -lcd[i, ineq - nP]
    rhs[ix["z"]:ix["z"] + nx] = -st.le
    rhs[ix["y"]:ix["y"] + N * L] = -st.lf
    return M, rhs, ix
