"""Synthetic multiperiod AC-OPF-with-storage KKT systems in arrowhead form.

The paper's MPOPF problem (Sec. 3.2, eq. MPOPF and the storage update
eq. linup) gives the structure; its grids (MATPOWER / PEGASE case files) are
not available, so seeded synthetic grids with the same shape stand in for
them.  Recipe (all draws from one numpy PCG64 stream per instance, in this
order):

1. topology: bus j >= 1 attaches to a uniformly drawn earlier bus (random
   spanning tree), then ``n_line - (n_bus - 1)`` extra distinct bus pairs are
   drawn uniformly;
2. lines: reactance x ~ U[0.02, 0.3], resistance r = 0.1 x, series
   admittance 1/(r + jx) = g + jb;
3. generators on ``n_gen`` distinct uniform buses, storage units on
   ``n_stor`` distinct uniform buses;
4. barrier diagonal, log-uniform in [bar_lo, bar_hi], i.i.d. per primal
   variable and per period;
5. coupling diagonal C, log-uniform in the same range;
6. right-hand side ~ N(0, 1).

Per period i the variables of block A_i are ordered primal first:
theta (n_bus), v (n_bus), P_g (n_gen), Q_g (n_gen), p_dis (n_stor),
p_chg (n_stor); then the multipliers of the P balance (n_bus), the Q balance
(n_bus) and the storage dynamics rows (n_stor).  The coupling variables are
the storage states of charge eps_{i,s}, one per unit and period, so
n_C = n_per * n_stor and column i*n_stor + s of B belongs to eps_{i,s}.

    A_i = [H_i  J_i^T; J_i  -1e-8 I]
    H_i = sum_lines (e_f - e_t)(e_f - e_t)^T (x) [[|b|, g], [g, |b|]]  (on (theta, v))
          + barrier diagonal on every primal variable
    J_i: P rows  <- line Laplacian (x) [|b|,  g] on (theta, v),
         Q rows  <- line Laplacian (x) [-g, |b|] on (theta, v),
         -1 on P_g / Q_g in the generator bus's P / Q row,
         +1 / -1 on p_dis / p_chg in the storage bus's P row,
         dynamics row s: -eta_c on p_chg_s, +1/eta_d on p_dis_s (eq. linup)
    B_i: dynamics row s has +1 in column (i, s) and -1 in column (i-1, s)
         (the previous period's state of charge; absent for i = 0)
    C   = diag(log-uniform)

This module only constructs inputs; it contains nothing of the Schur method.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np
import scipy.sparse as sp

ETA_C = 0.95
ETA_D = 0.95
DUAL_REG = -1e-8


@dataclass(frozen=True)
class GridSpec:
    """Sizes and seed of one synthetic MPOPF instance."""

    n_bus: int
    n_line: int
    n_gen: int
    n_stor: int
    n_per: int
    bar_lo: float = 1e-6
    bar_hi: float = 1e6
    seed: int = 1907
    name: str = ""

    @property
    def n_primal(self) -> int:
        return 2 * self.n_bus + 2 * self.n_gen + 2 * self.n_stor

    @property
    def n_dual(self) -> int:
        return 2 * self.n_bus + self.n_stor

    @property
    def n_a(self) -> int:
        return self.n_primal + self.n_dual

    @property
    def n_c(self) -> int:
        return self.n_per * self.n_stor


# Named workloads.  Sizes follow the multiperiod storage workloads: a 30-bus
# grid over 24 periods, a 2,383-bus grid over 96 periods and a 9,241-bus grid
# over 168 periods (late-IPM barrier range 1e-8..1e8 for the two large ones).
CONFIGS = {
    "tiny": GridSpec(5, 6, 2, 1, 3, 1e-3, 1e3, 7, "tiny"),
    "small": GridSpec(12, 15, 3, 2, 5, 1e-4, 1e4, 11, "small"),
    "grid30_n24": GridSpec(30, 40, 6, 3, 24, 1e-6, 1e6, 1907, "grid30_n24"),
    "grid2383_n96": GridSpec(2383, 2900, 327, 100, 96, 1e-8, 1e8, 2383, "grid2383_n96"),
    "grid9241_n168": GridSpec(9241, 16049, 1445, 400, 168, 1e-8, 1e8, 9241, "grid9241_n168"),
    # the same grid over 8 periods: a few GB on the device, for kernel profiles
    "grid9241_n8": GridSpec(9241, 16049, 1445, 400, 8, 1e-8, 1e8, 9241, "grid9241_n8"),
}


def mix_spec(k: int) -> GridSpec:
    """Instance k of the 64-instance size mix.

    Bus count log-uniform in [118, 3000], horizon uniform in {12, 24, 48, 96},
    storage on round(U[0.05, 0.10] * n_bus) buses, generators on
    round(0.15 * n_bus) buses, round(1.3 * n_bus) lines, barrier 1e-6..1e6.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([1000 + k, 1])))
    nb = int(round(np.exp(rng.uniform(np.log(118.0), np.log(3000.0)))))
    n_per = int(rng.choice([12, 24, 48, 96]))
    frac = rng.uniform(0.05, 0.10)
    ns = max(1, int(round(frac * nb)))
    ng = max(1, int(round(0.15 * nb)))
    nl = max(nb - 1, int(round(1.3 * nb)))
    return GridSpec(nb, nl, ng, ns, n_per, 1e-6, 1e6, 1000 + k, f"mix{k}")


@dataclass
class KKTProblem:
    """One arrowhead KKT system K = [blockdiag(A_0..A_{N-1}) B; B^T C].

    a_rowptr/a_col: CSR of the lower triangle of A (pattern shared by all
    blocks, 0-based, sorted columns, diagonal present).  a_vals[i] holds
    block i's values in that pattern.  B is given per block in COO form:
    entries b_blockptr[i]..b_blockptr[i+1] belong to block i, with row in
    [0, nA) and column in [0, nC), sorted by (row, col).  C is diagonal
    (c_kind 0, c_vals has nC entries).  rhs stacks r_0..r_{N-1}, r_g.
    """

    spec: GridSpec
    N: int
    nA: int
    nP: int
    nC: int
    a_rowptr: np.ndarray
    a_col: np.ndarray
    a_vals: np.ndarray
    b_blockptr: np.ndarray
    b_row: np.ndarray
    b_col: np.ndarray
    b_vals: np.ndarray
    c_kind: int
    c_vals: np.ndarray
    rhs: np.ndarray
    bar_pos: np.ndarray = field(repr=False, default=None)  # CSR positions of primal diagonals
    a_const: np.ndarray = field(repr=False, default=None)  # block values without the barrier
    ineq_rows: np.ndarray = field(repr=False, default=None)  # rows of A that are inequality constraints

    @property
    def nnzA(self) -> int:
        return int(self.a_rowptr[-1])

    @property
    def nK(self) -> int:
        return self.N * self.nA + self.nC


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def _topology(rng, nb, nl):
    parent = np.array([rng.integers(0, j) for j in range(1, nb)], dtype=np.int64)
    edges = [(int(p), j) for j, p in zip(range(1, nb), parent)]
    have = {(min(a, b), max(a, b)) for a, b in edges}
    extra = nl - (nb - 1)
    if extra > nb * (nb - 1) // 2 - len(have):
        raise ValueError("too many lines for the bus count")
    while extra > 0:
        a, b = (int(t) for t in rng.integers(0, nb, size=2))
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key in have:
            continue
        have.add(key)
        edges.append(key)
        extra -= 1
    return np.array(edges, dtype=np.int64)


def make_problem(spec: GridSpec, *, zero_b: bool = False, coupling: str = "adjacent",
                 flow_limits: int = 0, own_period_scale: float = 1.0) -> KKTProblem:
    """Build the seeded instance described by ``spec``.

    flow_limits=L > 0 appends L inequality rows to every A_i, after the other
    multiplier rows: the linearised flow limit of line l (l < L), with entries
    |b_l|, -|b_l| on the angles and g_l, -g_l on the magnitudes of its two
    buses.  Their multipliers and slacks are those of the slack elimination
    (Sec. 2, eq. SCOPFslackAtEnd): the rows are listed in ``ineq_rows`` and get
    the dual regularisation -1e-8 on their diagonal like the other multiplier
    rows.  L = 0 (the default) draws the same instance as before.

    zero_b=True keeps B's pattern but sets its values to zero (a special case
    in which the arrowhead system decouples).

    coupling="adjacent" (default): the coupling variables are the states of
    charge, C is a positive diagonal and B_i couples adjacent periods through
    the storage dynamics rows of A_i (S is SPD and block-tridiagonal).
    coupling="paper": the coupling of Sec. 4.1 (eq. B12N): the coupling
    variables are the multipliers of the cumulative energy constraints, one
    per storage unit and period, C = 0, A_i has no dynamics rows, and B_i
    puts period i's charge and discharge into the energy constraints of every
    period m >= i (coefficients eta_c and -1/eta_d), so S is dense and
    negative definite and K's inertia is (N nP, N nD + nC, 0).
    own_period_scale (paper coupling only) multiplies the coefficient of
    period i's charging power in period i's own energy constraint, so that
    the block of B_i for its own period (the paper's C_1) differs from the one
    repeated for the later periods (C_0) and is not a multiple of it; 1.0
    (the default) keeps them equal.
    """
    if coupling not in ("adjacent", "paper"):
        raise ValueError("coupling must be 'adjacent' or 'paper'")
    paper = coupling == "paper"
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    nb, ng, ns, N = spec.n_bus, spec.n_gen, spec.n_stor, spec.n_per
    edges = _topology(rng, nb, spec.n_line)
    x = rng.uniform(0.02, 0.3, size=len(edges))
    r = 0.1 * x
    den = r * r + x * x
    g = r / den                  # > 0
    bmag = x / den               # |b|
    gen_bus = rng.choice(nb, size=ng, replace=False)
    sto_bus = rng.choice(nb, size=ns, replace=False)

    nP = spec.n_primal
    if not 0 <= flow_limits <= spec.n_line:
        raise ValueError("flow_limits must be between 0 and the number of lines")
    nA0 = spec.n_a - (ns if paper else 0)
    nA = nA0 + flow_limits
    th = lambda k: k                      # noqa: E731
    vv = lambda k: nb + k                 # noqa: E731
    PG = 2 * nb
    QG = 2 * nb + ng
    PD = 2 * nb + 2 * ng
    PC = PD + ns
    Prow = lambda k: nP + k               # noqa: E731
    Qrow = lambda k: nP + nb + k          # noqa: E731
    DYN = nP + 2 * nb

    rows, cols, vals = [], [], []

    def add(rr, cc, vv_):
        rows.append(np.asarray(rr, dtype=np.int64))
        cols.append(np.asarray(cc, dtype=np.int64))
        vals.append(np.asarray(vv_, dtype=np.float64))

    f, t = edges[:, 0], edges[:, 1]
    # H: Laplacian (x) [[|b|, g], [g, |b|]] on (theta, v); full symmetric form
    for (ra, ca, w) in ((th, th, bmag), (vv, vv, bmag), (th, vv, g), (vv, th, g)):
        add(ra(f), ca(f), w)
        add(ra(t), ca(t), w)
        add(ra(f), ca(t), -w)
        add(ra(t), ca(f), -w)
    # J: P rows <- Laplacian (x) [|b|, g]; Q rows <- Laplacian (x) [-g, |b|]
    for (rr, ca, w) in ((Prow, th, bmag), (Prow, vv, g), (Qrow, th, -g), (Qrow, vv, bmag)):
        add(rr(f), ca(f), w)
        add(rr(t), ca(t), w)
        add(rr(f), ca(t), -w)
        add(rr(t), ca(f), -w)
    gi = np.arange(ng)
    add(Prow(gen_bus), PG + gi, -np.ones(ng))
    add(Qrow(gen_bus), QG + gi, -np.ones(ng))
    si = np.arange(ns)
    add(Prow(sto_bus), PD + si, np.ones(ns))
    add(Prow(sto_bus), PC + si, -np.ones(ns))
    if not paper:
        add(DYN + si, PC + si, -ETA_C * np.ones(ns))
        add(DYN + si, PD + si, (1.0 / ETA_D) * np.ones(ns))
    if flow_limits:
        li = np.arange(flow_limits)
        fl, tl = f[:flow_limits], t[:flow_limits]
        add(nA0 + li, th(fl), bmag[:flow_limits])
        add(nA0 + li, th(tl), -bmag[:flow_limits])
        add(nA0 + li, vv(fl), g[:flow_limits])
        add(nA0 + li, vv(tl), -g[:flow_limits])
    # diagonal present everywhere: zero placeholder on primal (barrier added
    # per period), dual regularisation on the multipliers
    add(np.arange(nP), np.arange(nP), np.zeros(nP))
    add(np.arange(nP, nA), np.arange(nP, nA), DUAL_REG * np.ones(nA - nP))

    R = np.concatenate(rows)
    Cc = np.concatenate(cols)
    V = np.concatenate(vals)
    # the J entries were generated as (dual row, primal col): already lower.
    # H entries: keep the lower triangle only.
    keep = R >= Cc
    R, Cc, V = R[keep], Cc[keep], V[keep]
    M = sp.coo_matrix((V, (R, Cc)), shape=(nA, nA)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    a_rowptr = M.indptr.astype(np.int32)
    a_col = M.indices.astype(np.int32)
    a_const = M.data.astype(np.float64)
    nnz = len(a_col)

    # positions of the primal diagonal entries in the CSR
    bar_pos = np.empty(nP, dtype=np.int64)
    for k in range(nP):
        lo, hi = a_rowptr[k], a_rowptr[k + 1]
        j = lo + np.searchsorted(a_col[lo:hi], k)
        assert a_col[j] == k
        bar_pos[k] = j

    barrier = _loguniform(rng, spec.bar_lo, spec.bar_hi, (N, nP))
    a_vals = np.broadcast_to(a_const, (N, nnz)).copy()
    a_vals[:, bar_pos] += barrier

    bp, br, bc, bv = [0], [], [], []
    if paper:
        # B_i: p_dis then p_chg of unit s (rows sorted) into the energy
        # constraints of unit s in periods m >= i
        for i in range(N):
            for row, coef in sorted([(PD + s, -1.0 / ETA_D) for s in range(ns)] +
                                    [(PC + s, ETA_C) for s in range(ns)]):
                s = row - PD if row < PC else row - PC
                for m in range(i, N):
                    br.append(row)
                    bc.append(m * ns + s)
                    bv.append(coef * own_period_scale if (m == i and row >= PC) else coef)
            bp.append(len(br))
    else:
        # B_i: dynamics row s couples eps_{i,s} (+1) and eps_{i-1,s} (-1)
        for i in range(N):
            for s in range(ns):
                if i > 0:
                    br.append(DYN + s)
                    bc.append((i - 1) * ns + s)
                    bv.append(-1.0)
                br.append(DYN + s)
                bc.append(i * ns + s)
                bv.append(1.0)
            bp.append(len(br))
    b_vals = np.array(bv, dtype=np.float64)
    if zero_b:
        b_vals[:] = 0.0

    nC = N * ns
    c_vals = _loguniform(rng, spec.bar_lo, spec.bar_hi, nC)
    if paper:
        c_vals[:] = 0.0  # drawn all the same, so the right-hand side's draws do not move
    rhs = rng.standard_normal(N * nA + nC)

    return KKTProblem(
        spec=spec, N=N, nA=nA, nP=nP, nC=nC,
        a_rowptr=a_rowptr, a_col=a_col, a_vals=a_vals,
        b_blockptr=np.array(bp, dtype=np.int32),
        b_row=np.array(br, dtype=np.int32), b_col=np.array(bc, dtype=np.int32),
        b_vals=b_vals, c_kind=0, c_vals=c_vals, rhs=rhs,
        bar_pos=bar_pos, a_const=a_const, ineq_rows=np.arange(nA0, nA, dtype=np.int32),
    )


def reseed_barrier(prob: KKTProblem, seed: int) -> KKTProblem:
    """Same pattern, B and C; fresh barrier diagonals and a fresh right-hand side.

    This is the re-solve request of the serving mix: a later IPM iterate of an
    instance already seen.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    s = prob.spec
    barrier = _loguniform(rng, s.bar_lo, s.bar_hi, (prob.N, prob.nP))
    a_vals = np.broadcast_to(prob.a_const, (prob.N, prob.nnzA)).copy()
    a_vals[:, prob.bar_pos] += barrier
    rhs = rng.standard_normal(prob.nK)
    return replace(prob, a_vals=a_vals, rhs=rhs)
