"""Synthetic security-constrained OPF (SCOPF) KKT systems in arrowhead form.

The paper's SCOPF problem (Sec. 3.1, eq. SCOPF; the arrowhead ordering of
eq. orderingSCOPF) gives the structure: one block per scenario -- the nominal
grid c_0 and N_c contingencies, each the grid with one line out -- and, as
coupling variables, the quantities the nonanticipatory constraints hold equal
in every scenario: the voltage magnitude at the generator (PV) buses and the
real power of their generators.  The reference generator's real power stays
local to each scenario (it covers the losses of that scenario).

Recipe (one numpy PCG64 stream per instance, in this order): topology and
lines as the MPOPF generator (random spanning tree plus extra lines;
x ~ U[0.02, 0.3], r = 0.1 x); generators on distinct uniform buses, the
first one the reference; the outaged lines, distinct and drawn among the
non-tree lines so every scenario stays connected; barrier diagonals,
log-uniform in [bar_lo, bar_hi], per scenario and local primal variable; the
barrier diagonal of the coupling variables; the right-hand side ~ N(0, 1).

Scenario c's block A_c, primal first: theta (all buses), v at the non-PV
buses, P of the reference generator, Q of every generator; then the
multipliers of the P and Q balance of every bus.  With L_c the line
Laplacian of scenario c (the outaged line's admittance set to zero, so all
blocks share one pattern):

    H_c  = L_c (x) [[|b|, g], [g, |b|]] on (theta, v) + barrier diagonal
    J_c: P rows <- L_c (x) [|b|, g] on (theta, v), Q rows <- L_c (x) [-g, |b|],
         -1 on the reference generator's P and on every generator's Q in its
         bus's P / Q row
    A_c  = [H_c  J_c^T; J_c  -1e-8 I] on the local variables,

and the parts of H_c and J_c on the PV-bus voltages, together with -1 on the
PV generators' P in their buses' P rows, form B_c (nA x nC).  C is the Hessian
on the coupling variables: the PV-bus block of the sum over scenarios of
L_c (x) |b|, plus their barrier diagonal; it is dense (c_kind 1).

This module only constructs inputs; it contains nothing of the Schur method.
"""
from __future__ import annotations

import numpy as np

from .mpopf import DUAL_REG, GridSpec, KKTProblem, _loguniform, _topology


def make_scopf(spec: GridSpec, n_cont: int) -> KKTProblem:
    """The seeded SCOPF instance on the grid of ``spec`` (its n_stor and n_per
    are not used) with ``n_cont`` line contingencies: N = n_cont + 1 blocks."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    nb, ng = spec.n_bus, spec.n_gen
    if ng < 2:
        raise ValueError("SCOPF needs a reference generator and at least one PV generator")
    edges = _topology(rng, nb, spec.n_line)
    x = rng.uniform(0.02, 0.3, size=len(edges))
    r = 0.1 * x
    den = r * r + x * x
    g = r / den
    bmag = x / den
    gen_bus = rng.choice(nb, size=ng, replace=False)
    n_tree = nb - 1  # the first nb - 1 edges form the spanning tree
    if n_cont > len(edges) - n_tree:
        raise ValueError("more contingencies than non-tree lines")
    out_line = n_tree + rng.choice(len(edges) - n_tree, size=n_cont, replace=False)
    N = n_cont + 1

    # index maps
    pv_bus = gen_bus[1:]
    nPV = len(pv_bus)
    pv_of = -np.ones(nb, dtype=np.int64)
    pv_of[pv_bus] = np.arange(nPV)
    non_pv = np.nonzero(pv_of < 0)[0]
    vloc = -np.ones(nb, dtype=np.int64)
    vloc[non_pv] = nb + np.arange(len(non_pv))
    PREF = nb + len(non_pv)
    QG = PREF + 1
    nP = QG + ng
    Prow = lambda k: nP + k        # noqa: E731
    Qrow = lambda k: nP + nb + k   # noqa: E731
    nA = nP + 2 * nb
    nC = 2 * nPV                   # v at PV buses, then P of the PV generators

    # every matrix entry as (kind, row, col, coefficient, line, weight): value =
    # coefficient * (|b| or g of the line in scenario c), or the coefficient
    # itself for line -1; kind 0: A, 1: B, 2: C
    ent = []

    def var_v(k):
        """('a', local column) or ('g', coupling column) of v at bus k."""
        return ("g", int(pv_of[k])) if pv_of[k] >= 0 else ("a", int(vloc[k]))

    for li, (f, t) in enumerate(edges):
        for (a, b_, sgn) in ((f, f, 1.0), (t, t, 1.0), (f, t, -1.0), (t, f, -1.0)):
            # H on (theta, v): [[|b|, g], [g, |b|]]
            for (ra, ca, wk) in ((("a", int(a)), ("a", int(b_)), "b"), (("a", int(a)), var_v(b_), "g"),
                                 (var_v(a), ("a", int(b_)), "g"), (var_v(a), var_v(b_), "b")):
                if ra[0] == "a" and ca[0] == "a":
                    ent.append((0, ra[1], ca[1], sgn, li, wk))
                elif ra[0] == "a" and ca[0] == "g":
                    ent.append((1, ra[1], ca[1], sgn, li, wk))
                elif ra[0] == "g" and ca[0] == "g":
                    ent.append((2, ra[1], ca[1], sgn, li, wk))
                # (g, a) entries are the transposes of (a, g) ones: B holds them once
            # J: P row of a <- [|b|, g] on (theta_b, v_b); Q row <- [-g, |b|]
            for (row, wt, wv) in ((Prow(a), ("b", 1.0), ("g", 1.0)), (Qrow(a), ("g", -1.0), ("b", 1.0))):
                ent.append((0, row, int(b_), sgn * wt[1], li, wt[0]))
                cv = var_v(b_)
                ent.append((0 if cv[0] == "a" else 1, row, cv[1], sgn * wv[1], li, wv[0]))
    ent.append((0, Prow(int(gen_bus[0])), PREF, -1.0, -1, "1"))
    for k in range(ng):
        ent.append((0, Qrow(int(gen_bus[k])), QG + k, -1.0, -1, "1"))
    for j in range(nPV):
        ent.append((1, Prow(int(pv_bus[j])), nPV + j, -1.0, -1, "1"))
    for k in range(nP):
        ent.append((0, k, k, 0.0, -1, "1"))          # primal diagonal (barrier added per scenario)
    for k in range(nP, nA):
        ent.append((0, k, k, DUAL_REG, -1, "1"))

    kind = np.array([e[0] for e in ent])
    row = np.array([e[1] for e in ent], dtype=np.int64)
    col = np.array([e[2] for e in ent], dtype=np.int64)
    coef = np.array([e[3] for e in ent])
    line = np.array([e[4] for e in ent], dtype=np.int64)
    wsel = np.array([e[5] for e in ent])

    def weights(c):
        """Entry values of scenario c."""
        wb, wg = bmag.copy(), g.copy()
        if c > 0:
            wb[out_line[c - 1]] = 0.0
            wg[out_line[c - 1]] = 0.0
        li = np.maximum(line, 0)
        w = np.where(wsel == "b", wb[li], wg[li])
        return np.where(line >= 0, coef * w, coef)

    # A: lower triangle of the local block, one pattern for every scenario
    mA = (kind == 0) & (row >= col)
    keyA = row[mA] * nA + col[mA]
    ukey, inv = np.unique(keyA, return_inverse=True)
    a_r, a_c = ukey // nA, ukey % nA
    a_rowptr = np.zeros(nA + 1, dtype=np.int64)
    np.add.at(a_rowptr, a_r + 1, 1)
    a_rowptr = np.cumsum(a_rowptr).astype(np.int32)
    a_col = a_c.astype(np.int32)
    nnz = len(ukey)
    bar_pos = np.searchsorted(ukey, np.arange(nP) * nA + np.arange(nP))

    # B: per scenario, entries (row, col) summed, sorted by (row, col)
    mB = kind == 1
    keyB = row[mB] * nC + col[mB]
    ukB, invB = np.unique(keyB, return_inverse=True)
    mC = kind == 2

    barrier = _loguniform(rng, spec.bar_lo, spec.bar_hi, (N, nP))
    a_vals = np.zeros((N, nnz))
    bp, br, bc, bv = [0], [], [], []
    Cm = np.zeros((nC, nC))
    for c in range(N):
        v = weights(c)
        np.add.at(a_vals[c], inv, v[mA])
        a_vals[c, bar_pos] += barrier[c]
        vb = np.zeros(len(ukB))
        np.add.at(vb, invB, v[mB])
        br.extend((ukB // nC).tolist())
        bc.extend((ukB % nC).tolist())
        bv.extend(vb.tolist())
        bp.append(len(br))
        np.add.at(Cm, (row[mC], col[mC]), v[mC])
    Cm[np.diag_indices(nC)] += _loguniform(rng, spec.bar_lo, spec.bar_hi, nC)
    rhs = rng.standard_normal(N * nA + nC)
    return KKTProblem(
        spec=spec, N=N, nA=nA, nP=nP, nC=nC,
        a_rowptr=a_rowptr, a_col=a_col, a_vals=a_vals,
        b_blockptr=np.array(bp, dtype=np.int32),
        b_row=np.array(br, dtype=np.int32), b_col=np.array(bc, dtype=np.int32),
        b_vals=np.array(bv, dtype=np.float64), c_kind=1, c_vals=Cm.reshape(-1), rhs=rhs,
        bar_pos=bar_pos, a_const=None,
    )
