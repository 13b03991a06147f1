"""Pins of the oracle's structured Schur complement (Sec. 4.3, eqs.
LocalSchurBs, LocalSchurBs3, GlobalSchur) to facts fixed outside it:

* the block vectors S_d, S_o expanded to a dense matrix equal the oracle's
  dense S (one full solve per coupling column, another code path) and the
  definition C - sum_i B_i^T A_i^{-1} B_i evaluated with dense LAPACK solves;
* the local S_i evaluated densely has exactly the zero and replicated blocks of
  eq. LocalSchurBs;
* the block factor rebuilds S (L D L^T), its solve matches LAPACK on random
  matrices of the structure (symmetric indefinite and with distinct diagonal,
  subdiagonal and trailing blocks, so a transposed or dropped term shows), and
  its pivot signs match the eigenvalues;
* Algorithm 1 with the structured S reproduces the oracle's dense-S solution.

The own-period scale 0.5 makes the paper's C_1 differ from C_0, so that
S11, S10 and S00 all differ.
"""
import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem
from oracle import structured as st
from tests.kkt_dense import b_dense, block_dense, c_dense, dense_K

EPS = np.finfo(np.float64).eps
CASES = [("tiny", 1.0), ("small", 1.0), ("small", 0.5), ("grid30_n24", 1.0), ("grid30_n24", 0.5)]


def _paper(name, scale):
    return make_problem(CONFIGS[name], coupling="paper", own_period_scale=scale)


def test_split_rejects_other_couplings():
    with pytest.raises(ValueError):
        st.cumulative_split(make_problem(CONFIGS["small"]))  # adjacent periods


def test_split_rejects_values_that_break_the_repetition():
    p = _paper("small", 1.0)
    # change one entry of block 0 in the last period only
    q = int(np.flatnonzero((np.asarray(p.b_col) // (p.nC // p.N) == p.N - 1))[0])
    b = p.b_vals.copy()
    b[q] *= 2.0
    from dataclasses import replace
    with pytest.raises(ValueError):
        st.cumulative_split(replace(p, b_vals=b))


@pytest.mark.parametrize("name,scale", CASES)
def test_global_blocks_equal_dense_schur(name, scale):
    p = _paper(name, scale)
    Sd, So = st.global_blocks(p)
    S = st.expand(Sd, So)
    S_orc = oracle.kkt_solve(p, want_S=True)["S"]
    scale_s = np.abs(S_orc).max()
    assert np.allclose(S, S_orc, rtol=1e-10, atol=1e-12 * scale_s)
    S_ref = c_dense(p).copy()
    for i in range(p.N):
        B = b_dense(p, i)
        S_ref -= B.T @ np.linalg.solve(block_dense(p, i), B)
    assert np.allclose(S, S_ref, rtol=1e-8, atol=1e-10 * scale_s)


@pytest.mark.parametrize("name,scale", [("small", 0.5), ("grid30_n24", 0.5)])
def test_local_blocks_have_the_replicated_structure(name, scale):
    """S_i = -B_i^T A_i^{-1} B_i: zero outside periods >= i, S11 at (i, i), S10
    in every row below it, S00 everywhere in the trailing part (eq. LocalSchurBs)."""
    p = _paper(name, scale)
    ns, Y, Z = st.cumulative_split(p)
    for i in (0, 1, p.N - 2):
        B = b_dense(p, i)
        Si = -(B.T @ np.linalg.solve(block_dense(p, i), B))
        S11, S10, S00 = st.local_blocks(p, i, Y, Z)
        tol = 1e-9 * np.abs(Si).max()
        blk = lambda m, j: Si[m * ns:(m + 1) * ns, j * ns:(j + 1) * ns]  # noqa: E731
        for m in range(p.N):
            for j in range(p.N):
                if m < i or j < i:
                    assert np.abs(blk(m, j)).max() == 0.0
                elif m == i and j == i:
                    assert np.allclose(blk(m, j), S11, atol=tol)
                elif j == i:
                    assert np.allclose(blk(m, j), S10, atol=tol)
                elif m == i:
                    assert np.allclose(blk(m, j), S10.T, atol=tol)
                else:
                    assert np.allclose(blk(m, j), S00, atol=tol)
        if scale != 1.0:  # the three blocks are distinct
            assert not np.allclose(S11, S10) and not np.allclose(S10, S00)


def _random_structured(rng, N, ns, definite):
    """A matrix of the GlobalSchur pattern: S = F^-1 T F^-T for a block
    tridiagonal T and the block difference operator F (F^-1 forms prefix sums,
    which gives exactly that pattern).  T is diagonally dominant with positive
    or alternating signs, so the LDL^T of S needs no pivoting and S has T's
    inertia."""
    n = N * ns
    T = np.zeros((n, n))
    sgn = np.ones(ns) if definite else np.where(np.arange(ns) % 2 == 0, 1.0, -1.0)
    for j in range(N):
        X = rng.standard_normal((ns, ns))
        D = 0.5 * (X + X.T) + np.diag(3.0 * ns * sgn)  # diagonally dominant, signs sgn
        T[j * ns:(j + 1) * ns, j * ns:(j + 1) * ns] = D
        if j + 1 < N:
            E = 0.3 * rng.standard_normal((ns, ns))
            T[(j + 1) * ns:(j + 2) * ns, j * ns:(j + 1) * ns] = E
            T[j * ns:(j + 1) * ns, (j + 1) * ns:(j + 2) * ns] = E.T
    Finv = np.kron(np.tril(np.ones((N, N))), np.eye(ns))  # prefix sums: inverse of differences
    S = Finv @ T @ Finv.T
    Sd = np.stack([S[j * ns:(j + 1) * ns, j * ns:(j + 1) * ns] for j in range(N)])
    So = np.array([S[(j + 1) * ns:(j + 2) * ns, j * ns:(j + 1) * ns] for j in range(N - 1)]).reshape(N - 1, ns, ns)
    assert np.allclose(st.expand(Sd, So), S)
    return S, Sd, So


@pytest.mark.parametrize("definite", [True, False])
@pytest.mark.parametrize("N,ns", [(1, 4), (2, 3), (6, 5), (9, 2)])
def test_block_factor_and_solve_match_lapack(N, ns, definite):
    rng = np.random.default_rng(100 * N + ns + (0 if definite else 7))
    S, Sd, So = _random_structured(rng, N, ns, definite)
    f = st.block_factor(Sd, So)
    # L D L^T rebuilt densely
    n = N * ns
    L = np.zeros((n, n))
    d = np.zeros(n)
    for j, (Lj, dj, L21) in enumerate(f):
        L[j * ns:(j + 1) * ns, j * ns:(j + 1) * ns] = Lj
        d[j * ns:(j + 1) * ns] = dj
        for m in range(j + 1, N):
            L[m * ns:(m + 1) * ns, j * ns:(j + 1) * ns] = L21
    assert np.allclose((L * d) @ L.T, S, rtol=1e-10, atol=1e-10 * np.abs(S).max())
    t = rng.standard_normal(n)
    x = st.block_solve(f, t)
    x_ref = np.linalg.solve(S, t)
    assert np.max(np.abs(x - x_ref)) <= 1e3 * np.linalg.cond(S) * EPS * np.max(np.abs(x_ref))
    ev = np.linalg.eigvalsh(S)
    assert list(st.inertia(f)) == [int((ev > 0).sum()), int((ev < 0).sum()), 0]


@pytest.mark.parametrize("name,scale", CASES)
def test_structured_algorithm1_matches_dense_oracle(name, scale):
    p = _paper(name, scale)
    out = st.kkt_solve_structured(p)
    ref = oracle.kkt_solve(p, want_S=True)
    K = dense_K(p)
    kappa = np.linalg.cond(K)
    err = np.max(np.abs(out["x"] - ref["x"])) / np.max(np.abs(ref["x"]))
    assert err <= max(1e-12, 1e3 * kappa * EPS), (err, kappa)
    assert oracle.backward_error(p, out["x"]) <= 1e-13
    assert np.allclose(out["t"], ref["t"], rtol=1e-10, atol=1e-12 * np.abs(ref["t"]).max())
    # S negative definite: all n_C pivots negative (the coupling variables are multipliers)
    assert list(out["inertia_s"]) == [0, p.nC, 0]
