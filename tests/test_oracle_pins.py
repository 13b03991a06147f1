"""Pins of the CPU oracle to facts fixed outside the oracle itself.

The paper prints no numeric solve example (its only printed KKT figures are
sparsity plots), so the oracle is pinned by:

* an independent dense LAPACK LU solve of the fully assembled K (tiny cases);
* the inertia of K from a dense symmetric eigensolver, against the count the
  inertia-correction section (Sec. 2.3) requires: one positive eigenvalue per
  primal variable and coupling variable, one negative per multiplier;
* closed forms: N = 1 without coupling (a plain sparse solve), B = 0
  (S = C, decoupled blocks), diagonal A_i (S = C - sum B_i^T diag(A_i)^-1 B_i);
* structure: S symmetric positive definite and block-tridiagonal in
  n_stor x n_stor blocks when B couples adjacent periods;
* factor identities: P L D L^T P^T = A, L_s D_s L_s^T = S;
* ordering facts: a valid permutation, no fill on trees, and every multiplier
  row after its primal neighbours in the constrained order.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, GridSpec, make_problem
from tests.kkt_dense import b_dense, block_dense, c_dense, dense_K, lower_dense

SMALL = ["tiny", "small", "grid30_n24"]
EPS = np.finfo(np.float64).eps


def _problem(name):
    return make_problem(CONFIGS[name])


@pytest.mark.parametrize("name", SMALL)
def test_solution_matches_dense_lu(name):
    p = _problem(name)
    out = oracle.kkt_solve(p)
    K = dense_K(p)
    x_lu = np.linalg.solve(K, p.rhs)
    kappa = np.linalg.cond(K)
    err = np.max(np.abs(out["x"] - x_lu)) / np.max(np.abs(x_lu))
    # both solutions are backward stable; their difference is bounded by
    # kappa * (backward errors); with kappa <= 1e11 here that is well below 1e-4
    assert kappa < 1e11
    assert err <= max(1e-12, 1e3 * kappa * EPS), (err, kappa)


@pytest.mark.parametrize("name", SMALL)
def test_backward_error(name):
    p = _problem(name)
    out = oracle.kkt_solve(p)
    eta = oracle.backward_error(p, out["x"])
    assert eta <= 1e-14, eta


def test_backward_error_2383_bus_grid_short_horizon():
    spec = replace(CONFIGS["grid2383_n96"], n_per=4, name="grid2383_n4")
    p = make_problem(spec)
    out = oracle.kkt_solve(p)
    assert oracle.backward_error(p, out["x"]) <= 1e-14
    assert list(out["inertia"]) == [p.N * p.nP + p.nC, p.N * (p.nA - p.nP), 0]


@pytest.mark.parametrize("name", SMALL)
def test_inertia_matches_eigenvalues(name):
    p = _problem(name)
    out = oracle.kkt_solve(p)
    ev = np.linalg.eigvalsh(dense_K(p))
    expect = [p.N * p.nP + p.nC, p.N * (p.nA - p.nP), 0]
    assert [int((ev > 0).sum()), int((ev < 0).sum()), 0] == expect
    assert list(out["inertia"]) == expect


def test_single_block_without_coupling_is_plain_sparse_solve():
    p = _problem("small")
    q = replace(p, N=1, nC=0, a_vals=p.a_vals[:1].copy(),
                b_blockptr=np.zeros(2, np.int32), b_row=np.zeros(0, np.int32),
                b_col=np.zeros(0, np.int32), b_vals=np.zeros(0),
                c_vals=np.zeros(0), rhs=p.rhs[: p.nA].copy())
    out = oracle.kkt_solve(q)
    x = np.linalg.solve(block_dense(p, 0), q.rhs)
    assert np.allclose(out["x"], x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_zero_coupling_decouples():
    p = make_problem(CONFIGS["small"], zero_b=True)
    out = oracle.kkt_solve(p, want_S=True)
    assert np.array_equal(out["S"], np.diag(p.c_vals))
    g = p.N * p.nA
    assert np.allclose(out["x"][g:], p.rhs[g:] / p.c_vals, rtol=1e-14)
    for i in range(p.N):
        xi = np.linalg.solve(block_dense(p, i), p.rhs[i * p.nA:(i + 1) * p.nA])
        got = out["x"][i * p.nA:(i + 1) * p.nA]
        assert np.allclose(got, xi, rtol=1e-9, atol=1e-12 * np.abs(xi).max())


def _diagonal_blocks(p, seed=5):
    rng = np.random.default_rng(seed)
    d = np.exp(rng.uniform(-3, 3, size=(p.N, p.nA)))
    d[:, p.nP:] *= -1.0
    return replace(p, a_rowptr=np.arange(p.nA + 1, dtype=np.int32),
                   a_col=np.arange(p.nA, dtype=np.int32), a_vals=d)


def test_diagonal_blocks_closed_form_schur():
    p = _diagonal_blocks(_problem("grid30_n24"))
    out = oracle.kkt_solve(p, want_S=True)
    S = np.diag(p.c_vals).copy()
    t = p.rhs[p.N * p.nA:].copy()
    for i in range(p.N):
        B = b_dense(p, i)
        dinv = 1.0 / p.a_vals[i]
        S -= B.T @ (dinv[:, None] * B)
        t -= B.T @ (dinv * p.rhs[i * p.nA:(i + 1) * p.nA])
    assert np.allclose(out["S"], S, rtol=1e-13, atol=1e-13 * np.abs(S).max())
    assert np.allclose(out["t"], t, rtol=1e-13, atol=1e-13 * np.abs(t).max())


@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_schur_structure(name):
    p = _problem(name)
    out = oracle.kkt_solve(p, want_S=True)
    S = out["S"]
    ns = p.spec.n_stor
    # symmetric up to the rounding of the column-by-column solves
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    blk = np.arange(p.nC) // ns
    outside = np.abs(blk[:, None] - blk[None, :]) > 1
    assert np.all(S[outside] == 0.0)
    assert np.all(np.linalg.eigvalsh(S) > 0)
    # against the definition evaluated with dense LAPACK solves
    S_ref = c_dense(p).copy()
    for i in range(p.N):
        B = b_dense(p, i)
        S_ref -= B.T @ np.linalg.solve(block_dense(p, i), B)
    assert np.allclose(S, S_ref, rtol=1e-8, atol=1e-10 * np.abs(S_ref).max())


@pytest.mark.parametrize("name", ["tiny", "small"])
@pytest.mark.parametrize("constrained", [False, True])
def test_sparse_ldlt_reconstructs_block(name, constrained):
    p = _problem(name)
    perm = oracle.min_degree(p.nA, p.a_rowptr, p.a_col, p.nP if constrained else None)
    for i in range(p.N):
        L, D = oracle.ldlt_dense(p.nA, p.a_rowptr, p.a_col, p.a_vals[i], perm)
        A = block_dense(p, i)
        Ap = A[np.ix_(perm, perm)]
        # componentwise bound of LDL^T without pivoting: |A - LDL^T| <= c n u |L||D||L^T|
        bound = 4 * p.nA * EPS * (np.abs(L) @ np.diag(np.abs(D)) @ np.abs(L).T)
        assert np.all(np.abs(L @ np.diag(D) @ L.T - Ap) <= bound + 1e-300)
        assert np.allclose(np.diag(L), 1.0)
        assert np.all(np.triu(L, 1) == 0.0)
        # quasidefinite: primal pivots positive, multiplier pivots negative
        assert np.all((D > 0) == (perm < p.nP))


def test_dense_ldlt_identity_and_inertia():
    rng = np.random.default_rng(3)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.exp(rng.uniform(-2, 2, 25)), -np.exp(rng.uniform(-2, 2, 15))])
    S = (Q * lam) @ Q.T
    S = 0.5 * (S + S.T)
    F, inertia = oracle.dense_ldlt(S)
    L = np.tril(F, -1) + np.eye(n)
    D = np.diag(F)
    assert np.allclose(L @ np.diag(D) @ L.T, S, atol=1e-10)
    assert list(inertia) == [25, 15, 0]
    b = rng.standard_normal(n)
    assert np.allclose(oracle.dense_ldlt_solve(F, b), np.linalg.solve(S, b), rtol=1e-8)


def _path_csr(n):
    rowptr = [0]
    col = []
    for r in range(n):
        if r > 0:
            col.append(r - 1)
        col.append(r)
        rowptr.append(len(col))
    return np.array(rowptr, np.int32), np.array(col, np.int32)


def test_min_degree_no_fill_on_tree_and_star():
    # a path and a star are trees: eliminating a leaf never creates fill, so a
    # minimum-degree order gives nnz(L) = n - 1
    n = 50
    rp, c = _path_csr(n)
    perm = oracle.min_degree(n, rp, c)
    assert sorted(perm) == list(range(n))
    assert oracle.nnz_l(n, rp, c, perm) == n - 1
    rowptr = [0, 1]
    col = [0]
    for r in range(1, n):
        col += [0, r]
        rowptr.append(len(col))
    rp, c = np.array(rowptr, np.int32), np.array(col, np.int32)
    perm = oracle.min_degree(n, rp, c)
    assert perm[-1] == 0 or perm[-2] == 0
    assert oracle.nnz_l(n, rp, c, perm) == n - 1


@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_constrained_order_puts_multipliers_after_primal_neighbours(name):
    p = _problem(name)
    perm = oracle.min_degree(p.nA, p.a_rowptr, p.a_col, p.nP)
    pos = np.empty(p.nA, np.int64)
    pos[perm] = np.arange(p.nA)
    A = lower_dense(p.a_rowptr, p.a_col, np.ones(p.nnzA), p.nA)
    for r in range(p.nP, p.nA):
        nb = np.nonzero(A[r, :p.nP])[0]
        assert np.all(pos[nb] < pos[r])


@pytest.mark.parametrize("name", SMALL)
def test_matvec_and_norm(name):
    p = _problem(name)
    K = dense_K(p)
    x = np.random.default_rng(1).standard_normal(p.nK)
    assert np.allclose(oracle.kkt_matvec(p, x), K @ x, rtol=1e-13, atol=1e-12)
    assert np.isclose(oracle.kkt_norm_inf(p), np.abs(K).sum(1).max(), rtol=1e-14)


def test_generator_is_deterministic_and_shaped():
    a = make_problem(CONFIGS["grid30_n24"])
    b = make_problem(CONFIGS["grid30_n24"])
    assert np.array_equal(a.a_vals, b.a_vals) and np.array_equal(a.rhs, b.rhs)
    assert (a.nA, a.nP, a.nC, a.N) == (141, 78, 72, 24)
    spec = GridSpec(30, 40, 6, 3, 24, 1e-6, 1e6, 1908)
    c = make_problem(spec)
    assert not np.array_equal(a.rhs, c.rhs)


# ---- the paper's own MPOPF coupling (Sec. 4.1, eq. B12N; Sec. 4.3) ----
# Coupling variables are the multipliers of the cumulative energy constraints,
# C = 0, and B_i feeds period i's storage injections into the constraints of
# every later period.  The oracle is the same program; these pins check it on
# that structure against LAPACK and against the block structure Sec. 4.3
# derives for S.

@pytest.mark.parametrize("name", ["tiny", "small"])
def test_paper_coupling_matches_dense_lu_and_eigenvalues(name):
    p = make_problem(CONFIGS[name], coupling="paper")
    out = oracle.kkt_solve(p)
    K = dense_K(p)
    x_lu = np.linalg.solve(K, p.rhs)
    kappa = np.linalg.cond(K)
    err = np.max(np.abs(out["x"] - x_lu)) / np.max(np.abs(x_lu))
    assert err <= max(1e-12, 1e3 * kappa * EPS), (err, kappa)
    assert oracle.backward_error(p, out["x"]) <= 1e-14
    # the coupling variables are multipliers now: nC more negative eigenvalues
    expect = [p.N * p.nP, p.N * (p.nA - p.nP) + p.nC, 0]
    ev = np.linalg.eigvalsh(K)
    assert [int((ev > 0).sum()), int((ev < 0).sum()), 0] == expect
    assert list(out["inertia"]) == expect


@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_paper_coupling_schur_structure(name):
    """S is dense and negative definite, and in every block column the blocks
    on and below the diagonal are one and the same n_stor x n_stor block (the
    identical subdiagonal blocks of Sec. 4.3; with the energy constraint of a
    period taking that period's injections, the diagonal block equals them
    too), so S is determined by N such blocks."""
    p = make_problem(CONFIGS[name], coupling="paper")
    out = oracle.kkt_solve(p, want_S=True)
    S = out["S"]
    ns = p.spec.n_stor
    assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) < 0)
    scale = np.abs(S).max()
    for j in range(p.N):
        col = S[:, j * ns:(j + 1) * ns]
        ref = col[j * ns:(j + 1) * ns]
        for m in range(j + 1, p.N):
            assert np.allclose(col[m * ns:(m + 1) * ns], ref, rtol=1e-12, atol=1e-14 * scale)
    # against the definition evaluated with dense LAPACK solves
    S_ref = c_dense(p).copy()
    for i in range(p.N):
        B = b_dense(p, i)
        S_ref -= B.T @ np.linalg.solve(block_dense(p, i), B)
    assert np.allclose(S, S_ref, rtol=1e-8, atol=1e-10 * scale)


# ---- the SCOPF workload (Sec. 3.1, eq. SCOPF, eq. orderingSCOPF) ----
# Blocks are scenarios (nominal and line outages); coupling variables are the
# PV-bus voltages and PV generator powers; C is a dense Hessian block.

SCOPF_CASES = [(GridSpec(9, 12, 3, 0, 1, 1e-4, 1e4, 3, "scopf9"), 2),
               (GridSpec(14, 20, 5, 0, 1, 1e-4, 1e4, 5, "scopf14"), 4),
               (GridSpec(30, 41, 6, 0, 1, 1e-6, 1e6, 7, "scopf30"), 8)]


@pytest.mark.parametrize("case", range(len(SCOPF_CASES)))
def test_scopf_matches_dense_lu_and_inertia(case):
    from gen import make_scopf

    p = make_scopf(*SCOPF_CASES[case])
    assert p.c_kind == 1
    out = oracle.kkt_solve(p)
    K = dense_K(p)
    x_lu = np.linalg.solve(K, p.rhs)
    kappa = np.linalg.cond(K)
    err = np.max(np.abs(out["x"] - x_lu)) / np.max(np.abs(x_lu))
    assert err <= max(1e-12, 1e3 * kappa * EPS), (err, kappa)
    assert oracle.backward_error(p, out["x"]) <= 1e-14
    expect = [p.N * p.nP + p.nC, p.N * (p.nA - p.nP), 0]
    ev = np.linalg.eigvalsh(K)
    assert [int((ev > 0).sum()), int((ev < 0).sum()), 0] == expect
    assert list(out["inertia"]) == expect


def test_scopf_schur_complement():
    """S = C - sum B_c^T A_c^-1 B_c is SPD and equals its definition evaluated
    with dense LAPACK solves; the contingency blocks differ from the nominal
    one only in the outaged line's entries."""
    from gen import make_scopf

    p = make_scopf(*SCOPF_CASES[1])
    S = oracle.kkt_solve(p, want_S=True)["S"]
    S_ref = c_dense(p).copy()
    for i in range(p.N):
        B = b_dense(p, i)
        S_ref -= B.T @ np.linalg.solve(block_dense(p, i), B)
    assert np.allclose(S, S_ref, rtol=1e-8, atol=1e-10 * np.abs(S_ref).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) > 0)
    base = block_dense(p, 0) - np.diag(np.diag(block_dense(p, 0)))
    for c in range(1, p.N):
        d = (block_dense(p, c) - np.diag(np.diag(block_dense(p, c)))) - base
        # one line out: only the theta, v and balance rows of its two buses change
        rows = np.nonzero(np.any(d != 0, axis=1))[0]
        assert 0 < len(rows) <= 8 and np.array_equal(d, d.T)
