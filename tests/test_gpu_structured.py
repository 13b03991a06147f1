"""The structured S of the paper's cumulative coupling on the GPU
(kkt_options.structured_s = 2; Sec. 4.3, eqs. LocalSchurBs, LocalSchurBs3,
GlobalSchur) against the oracle (oracle/structured.py and the dense-S oracle).

* S_d and S_o element by element against the oracle's block vectors, within
  10 kappa(A_i) eps of max|S| (both sides form A_i^{-1} E by backward-stable
  solves; the blocks inherit the blocks' conditioning);
* the solution: eta <= 1e-10 by the oracle's K x, and element by element
  within 10 kappa(K) max(eta, eps) of the oracle's x;
* the inertia of K (N nP, N nD + nC, 0) from the pivots of the FP64-accurate
  factors (the TF32 mode factors the periods in FP32, whose pivot signs are
  not relied on, and may fall back to the FP64 factor);
* B values that break the repetition are reported by the next solve.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem
from oracle import structured as ost
from tests.kkt_dense import block_dense, dense_K

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _paper(name, scale=1.0):
    return make_problem(CONFIGS[name], coupling="paper", own_period_scale=scale)


def _run(p, prec, want_blocks=True, **opts):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    h = B.kkt_analyze(p, B.kkt_default_options(prec, structured_s=2, **opts))
    try:
        dev = torch.device("cuda:0")
        B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                     np.ascontiguousarray(p.c_vals))
        x = np.empty(p.nK)
        B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
        info = B.kkt_get_info(h)
        blocks = None
        if want_blocks:
            ns = p.nC // p.N
            Sd = torch.empty(p.N * ns * ns, dtype=torch.float64, device=dev)
            So = torch.empty(max(1, (p.N - 1) * ns * ns), dtype=torch.float64, device=dev)
            B.kkt_schur_blocks(h, Sd, So)
            torch.cuda.synchronize()
            # column-major blocks: transpose to (row, column)
            Sd = Sd.cpu().numpy().reshape(p.N, ns, ns).transpose(0, 2, 1)
            So = So.cpu().numpy()[:(p.N - 1) * ns * ns].reshape(p.N - 1, ns, ns).transpose(0, 2, 1)
            blocks = (Sd, So)
    finally:
        B.kkt_destroy(h)
    return x, info, blocks


def _expected_inertia(p):
    return [p.N * p.nP, p.N * (p.nA - p.nP) + p.nC, 0]


CASES = [("tiny", 1.0), ("small", 1.0), ("small", 0.5), ("grid30_n24", 1.0), ("grid30_n24", 0.5)]


@pytest.mark.parametrize("prec", ["fp64", "tf32", "f64emu"])
@pytest.mark.parametrize("name,scale", CASES)
def test_structured_matches_oracle(name, scale, prec):
    p = _paper(name, scale)
    # the FP32 period factors of the TF32 mode: GMRES refinement to 1e-13, so
    # that the forward-error bound below means something at kappa(K) ~ 1e11
    tight = {"refine_mode": 1, "refine_tol": 1e-13, "max_refine": 20} if prec == "tf32" else {}
    x, info, (Sd, So) = _run(p, prec, **tight)
    assert info["schur_block"] == p.nC // p.N
    Sd_ref, So_ref = ost.global_blocks(p)
    # the lower triangles of the diagonal blocks (the factor reads no more), all of S_o
    lower = np.tril(np.ones(Sd.shape[1:], dtype=bool))
    kappa_a = max(np.linalg.cond(block_dense(p, i)) for i in range(p.N))
    scale_s = max(np.abs(Sd_ref).max(), np.abs(So_ref).max() if So_ref.size else 0.0)
    tol = 10.0 * kappa_a * EPS * scale_s
    assert np.max(np.abs((Sd - Sd_ref)[:, lower])) <= tol
    if So_ref.size:
        assert np.max(np.abs(So - So_ref)) <= tol
    # the solution
    ref = oracle.kkt_solve(p)
    eta = oracle.backward_error(p, x)
    eta_ref = oracle.backward_error(p, ref["x"])
    assert eta <= (1e-13 if tight else 1e-10), eta
    kappa = np.linalg.cond(dense_K(p))
    err = np.max(np.abs(x - ref["x"])) / np.max(np.abs(ref["x"]))
    assert err <= 10.0 * kappa * max(eta, eta_ref, EPS), (err, kappa)
    if prec != "tf32" or info["fell_back_fp64"]:
        assert [info["n_pos"], info["n_neg"], info["n_zero"]] == _expected_inertia(p)
    if prec != "tf32":
        assert info["fell_back_fp64"] == 0


@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_structured_agrees_with_the_dense_path(name):
    """The same system through the dense S (structured_s = 0) and the block
    vectors: both solutions within the conditioning bound of each other."""
    from tests.test_gpu_parity import gpu_solve

    p = _paper(name, 0.5)
    xs, _, _ = _run(p, "fp64", want_blocks=False)
    xd, _ = gpu_solve(p, "fp64")
    kappa = np.linalg.cond(dense_K(p))
    eta = max(oracle.backward_error(p, xs), oracle.backward_error(p, xd), EPS)
    assert np.max(np.abs(xs - xd)) / np.max(np.abs(xd)) <= 10.0 * kappa * eta


def test_structured_reports_values_that_do_not_repeat():
    """A value of B in a later period that differs from the others breaks the
    structure: the next solve returns KKT_ERR_INVALID; a factor of proper
    values clears it."""
    _torch()
    from paper_1907_05420_gb300 import binding as B

    p = _paper("small", 1.0)
    ns = p.nC // p.N
    q = int(np.flatnonzero((np.asarray(p.b_col) // ns) == p.N - 1)[0])  # block 0, last period
    bad = p.b_vals.copy()
    bad[q] *= 2.0
    h = B.kkt_analyze(p, B.kkt_default_options("fp64", structured_s=2))
    try:
        x = np.empty(p.nK)
        B.kkt_factor(h, np.ascontiguousarray(p.a_vals), bad, np.ascontiguousarray(p.c_vals))
        with pytest.raises(B.KKTError) as ei:
            B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
        assert ei.value.status == 1
        B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                     np.ascontiguousarray(p.c_vals))
        B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
        assert oracle.backward_error(p, x) <= 1e-10
    finally:
        B.kkt_destroy(h)


def test_structured_split_api_is_refused():
    _torch()
    from paper_1907_05420_gb300 import binding as B

    p = _paper("small", 1.0)
    h = B.kkt_analyze(p, B.kkt_default_options("fp64", structured_s=2))
    try:
        with pytest.raises(B.KKTError) as ei:
            B.kkt_factor_blocks(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                                np.ascontiguousarray(p.c_vals))
        assert ei.value.status == 1
    finally:
        B.kkt_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_structured_grid2383_n96_paper(prec):
    """The full-size paper workload (n_C = 9,600 in 96 periods of 100), which
    the dense-S analysis cannot take: eta and inertia at any size, and the
    first diagonal and subdiagonal blocks against the oracle's, which need only
    the first two block solves."""
    p = _paper("grid2383_n96")
    x, info, (Sd, So) = _run(p, prec)
    assert oracle.backward_error(p, x) <= 1e-10
    if prec == "fp64" or info["fell_back_fp64"]:
        assert [info["n_pos"], info["n_neg"], info["n_zero"]] == _expected_inertia(p)
    ns, Y, Z = ost.cumulative_split(p)
    S11_0, S10_0, S00_0 = ost.local_blocks(p, 0, Y, Z)
    S11_1, S10_1, _ = ost.local_blocks(p, 1, Y, Z)
    c = np.asarray(p.c_vals)
    ref = {"Sd0": np.diag(c[:ns]) + S11_0, "So0": S10_0, "Sd1": np.diag(c[ns:2 * ns]) + S11_1 + S00_0,
           "So1": S10_1 + S00_0}
    got = {"Sd0": Sd[0], "So0": So[0], "Sd1": Sd[1], "So1": So[1]}
    lower = np.tril(np.ones((ns, ns), dtype=bool))
    for key, r in ref.items():
        g = got[key]
        m = lower if key.startswith("Sd") else np.ones_like(lower)
        rel = np.max(np.abs((g - r)[m])) / np.abs(r).max()
        assert rel <= 1e-6, (key, rel)
    # S is negative definite, so is every diagonal block
    assert np.all(np.linalg.eigvalsh(Sd[0]) < 0) and np.all(np.linalg.eigvalsh(Sd[-1]) < 0)
