"""The structured Schur complement of the paper's cumulative MPOPF coupling
(Sec. 4.3, eqs. LocalSchurBs, LocalSchurBs3, GlobalSchur) in plain FP64.

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark's CPU legs use it;
the library's product path never imports it.

Coupling (Sec. 4.1, eq. B12N): the coupling variables are ordered by period,
n_s of them per period (n_C = N n_s).  In block i the coupling columns of
period m are zero for m < i, Y_i for m = i (the paper's C_1) and one and the
same Z_i for every m > i (the paper's C_0).  With C diagonal, S = C + sum_i S_i,
S_i = -B_i^T A_i^{-1} B_i, and S_i has only three distinct n_s x n_s blocks
(eq. LocalSchurBs, collected in eq. LocalSchurBs3):

    (i, i):              S11_i = -Y_i^T A_i^{-1} Y_i
    (m, i), m > i:       S10_i = -Z_i^T A_i^{-1} Y_i
    (m, m'), m, m' > i:  S00_i = -Z_i^T A_i^{-1} Z_i

so that S (eq. GlobalSchur) has in block column j the diagonal block and one
block repeated in every row m > j, kept as the two block vectors

    S_d[j] = C_j + S11_j + sum_{i<j} S00_i
    S_o[j] = S10_j + sum_{i<j} S00_i          (j < N - 1).

The factor (Sec. 4.3 states its O(n^2) cost but not its steps; these are
ours): block LDL^T without pivoting.  Eliminating block column j subtracts the
same matrix from every trailing block, because all its subdiagonal blocks are
equal, so the trailing matrix keeps the structure with S_d and S_o lowered by
one accumulated matrix U:

    U_0 = 0
    Delta_j = S_d[j] - U_j = L_j D_j L_j^T      (scalar LDL^T, no pivoting)
    P_j     = S_o[j] - U_j
    L21_j   = P_j L_j^{-T} D_j^{-1}             (the block below the diagonal
                                                 in every row m > j)
    U_{j+1} = U_j + L21_j D_j L21_j^T

and S x = t is solved by

    forward:   y_j = L_j^{-1} (t_j - R_j),  R_{j+1} = R_j + L21_j y_j,  R_0 = 0
    diagonal:  z_j = D_j^{-1} y_j
    backward:  x_j = L_j^{-T} (z_j - L21_j^T Q_j),  Q_{j-1} = Q_j + x_j,  Q_{N-1} = 0.

The pivots of all Delta_j are those of an LDL^T of S: their signs give S's
inertia.  Parity pins: tests/test_oracle_structured.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import dense_ldlt, min_degree, sparse_solve_multi


def cumulative_split(prob):
    """(n_s, Y, Z): per block the dense n_A x n_s coupling columns of its own
    period (Y[i]) and of the later periods (Z[i], None for the last block).
    ValueError if B does not have the cumulative structure or C is dense."""
    N, nA, nC = prob.N, prob.nA, prob.nC
    if prob.c_kind != 0:
        raise ValueError("the cumulative structure needs a diagonal C")
    if nC % N:
        raise ValueError("n_C is not a multiple of N")
    ns = nC // N
    bp = np.asarray(prob.b_blockptr)
    rows, cols, vals = np.asarray(prob.b_row), np.asarray(prob.b_col), np.asarray(prob.b_vals)
    Y, Z = [], []
    for i in range(N):
        groups = [np.zeros((nA, ns)) for _ in range(N)]
        seen = [np.zeros((nA, ns), dtype=bool) for _ in range(N)]
        for q in range(bp[i], bp[i + 1]):
            m, s = divmod(int(cols[q]), ns)
            if m < i:
                raise ValueError(f"block {i} couples to the earlier period {m}")
            groups[m][rows[q], s] += vals[q]
            seen[m][rows[q], s] = True
        for m in range(i + 2, N):
            if not (np.array_equal(seen[m], seen[i + 1]) and np.array_equal(groups[m], groups[i + 1])):
                raise ValueError(f"block {i}: the columns of period {m} differ from those of period {i + 1}")
        Y.append(groups[i])
        Z.append(groups[i + 1] if i + 1 < N else None)
    return ns, Y, Z


def local_blocks(prob, i, Y, Z, perm=None):
    """(S11_i, S10_i, S00_i) of eq. LocalSchurBs3 (S10, S00 None for the last block)."""
    if perm is None:
        perm = min_degree(prob.nA, prob.a_rowptr, prob.a_col, prob.nP)
    F = Y[i] if Z[i] is None else np.hstack([Y[i], Z[i]])
    X = sparse_solve_multi(prob.nA, prob.a_rowptr, prob.a_col, prob.a_vals[i], perm, F)  # A_i^{-1} [Y Z]
    ns = Y[i].shape[1]
    XY = X[:, :ns]
    S11 = -(Y[i].T @ XY)
    if Z[i] is None:
        return S11, None, None
    XZ = X[:, ns:]
    return S11, -(Z[i].T @ XY), -(Z[i].T @ XZ)


def global_blocks(prob, perm=None):
    """S_d (N x n_s x n_s) and S_o ((N-1) x n_s x n_s) of eq. GlobalSchur."""
    ns, Y, Z = cumulative_split(prob)
    if perm is None:
        perm = min_degree(prob.nA, prob.a_rowptr, prob.a_col, prob.nP)
    N = prob.N
    c = np.asarray(prob.c_vals, dtype=np.float64)
    Sd = np.empty((N, ns, ns))
    So = np.empty((max(N - 1, 0), ns, ns))
    acc = np.zeros((ns, ns))  # sum_{i<j} S00_i
    for j in range(N):
        S11, S10, S00 = local_blocks(prob, j, Y, Z, perm)
        Sd[j] = np.diag(c[j * ns:(j + 1) * ns]) + S11 + acc
        if j < N - 1:
            So[j] = S10 + acc
            acc = acc + S00
    return Sd, So


def expand(Sd, So):
    """The dense S of eq. GlobalSchur from its two block vectors."""
    N, ns = Sd.shape[0], Sd.shape[1]
    S = np.zeros((N * ns, N * ns))
    for j in range(N):
        S[j * ns:(j + 1) * ns, j * ns:(j + 1) * ns] = Sd[j]
        for m in range(j + 1, N):
            S[m * ns:(m + 1) * ns, j * ns:(j + 1) * ns] = So[j]
            S[j * ns:(j + 1) * ns, m * ns:(m + 1) * ns] = So[j].T
    return S


def block_factor(Sd, So):
    """[(L_j, d_j, L21_j)]: the structured block LDL^T (L21 None for the last)."""
    N, ns = Sd.shape[0], Sd.shape[1]
    U = np.zeros((ns, ns))
    out = []
    for j in range(N):
        F, _ = dense_ldlt(Sd[j] - U)                 # Delta_j = L_j D_j L_j^T
        L = np.tril(F, -1) + np.eye(ns)
        d = np.diag(F).copy()
        if j == N - 1:
            out.append((L, d, None))
            break
        P = So[j] - U
        L21 = sla.solve_triangular(L, P.T, lower=True, unit_diagonal=True).T / d  # P L^{-T} D^{-1}
        U = U + (L21 * d) @ L21.T
        out.append((L, d, L21))
    return out


def block_solve(factors, t):
    """x = S^{-1} t from block_factor's output."""
    N = len(factors)
    ns = factors[0][0].shape[0]
    t = np.asarray(t, dtype=np.float64).reshape(N, ns)
    y = np.empty((N, ns))
    R = np.zeros(ns)
    for j, (L, d, L21) in enumerate(factors):
        y[j] = sla.solve_triangular(L, t[j] - R, lower=True, unit_diagonal=True)
        if L21 is not None:
            R = R + L21 @ y[j]
    x = np.empty((N, ns))
    Q = np.zeros(ns)
    for j in range(N - 1, -1, -1):
        L, d, L21 = factors[j]
        rhs = y[j] / d
        if L21 is not None:
            rhs = rhs - L21.T @ Q
        x[j] = sla.solve_triangular(L, rhs, lower=True, unit_diagonal=True, trans="T")
        Q = Q + x[j]
    return x.reshape(-1)


def inertia(factors):
    d = np.concatenate([f[1] for f in factors])
    return np.array([(d > 0).sum(), (d < 0).sum(), (d == 0).sum()], dtype=np.int64)


def kkt_solve_structured(prob, rhs=None, perm=None):
    """Algorithm 1 (eqs. SCform, SCsolve, SCsolve1) with the structured S:
    dict(x, Sd, So, t, inertia_s)."""
    ns, Y, Z = cumulative_split(prob)
    if perm is None:
        perm = min_degree(prob.nA, prob.a_rowptr, prob.a_col, prob.nP)
    N, nA, nC = prob.N, prob.nA, prob.nC
    r = np.asarray(prob.rhs if rhs is None else rhs, dtype=np.float64)
    c = np.asarray(prob.c_vals, dtype=np.float64)
    Sd = np.empty((N, ns, ns))
    So = np.empty((max(N - 1, 0), ns, ns))
    t = r[N * nA:].copy()
    acc = np.zeros((ns, ns))
    sols = []
    for i in range(N):
        ri = r[i * nA:(i + 1) * nA]
        F = np.hstack([Y[i], ri[:, None]] if Z[i] is None else [Y[i], Z[i], ri[:, None]])
        X = sparse_solve_multi(nA, prob.a_rowptr, prob.a_col, prob.a_vals[i], perm, F)
        XY, u = X[:, :ns], X[:, -1]
        sols.append((XY, X[:, ns:2 * ns] if Z[i] is not None else None, u))
        Sd[i] = np.diag(c[i * ns:(i + 1) * ns]) - Y[i].T @ XY + acc
        t[i * ns:(i + 1) * ns] -= Y[i].T @ u                 # t = r_g - sum_i B_i^T A_i^{-1} r_i
        if Z[i] is not None:
            So[i] = -(Z[i].T @ XY) + acc
            acc = acc - Z[i].T @ sols[i][1]
            t[(i + 1) * ns:] -= np.tile(Z[i].T @ u, N - i - 1)
    factors = block_factor(Sd, So)
    xg = block_solve(factors, t)
    x = np.empty(N * nA + nC)
    x[N * nA:] = xg
    xg_b = xg.reshape(N, ns)
    for i in range(N):
        XY, XZ, u = sols[i]
        # x_i = A_i^{-1} (r_i - B_i x_g) = u - A_i^{-1} Y_i x_g,i - A_i^{-1} Z_i sum_{m>i} x_g,m
        xi = u - XY @ xg_b[i]
        if XZ is not None:
            xi = xi - XZ @ xg_b[i + 1:].sum(axis=0)
        x[i * nA:(i + 1) * nA] = xi
    return {"x": x, "Sd": Sd, "So": So, "t": t, "inertia_s": inertia(factors)}
