"""Non-finite values never pass the refinement's convergence test.

The normwise backward error eta = ||r-Kx||_inf / (||K||_inf ||x||_inf + ||r||_inf)
is meaningless when any of its norms is NaN or Inf: an Inf in x alone would make
eta = 0.  The norms on the device keep NaN, and kkt_solve returns
KKT_ERR_NONFINITE instead of KKT_OK whenever the values of K, the right-hand
side or the final iterate are not finite.  The faults are made on the host: a
NaN planted in one value of A, an Inf in the right-hand side, one block of A
set to zero (every pivot of that block is then an exact zero and its factor
holds 0/0).  Afterwards the same handle, refactored with the original values,
solves to eta <= 1e-10 again: a bad input leaves no state behind.
"""
import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem

pytestmark = pytest.mark.gpu

KKT_ERR_NONFINITE = 9


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _solve_status(B, h, a, b, c, r):
    """(status, x) of kkt_factor + kkt_solve on host arrays."""
    B.kkt_factor(h, np.ascontiguousarray(a), np.ascontiguousarray(b), np.ascontiguousarray(c))
    x = np.empty(r.size)
    try:
        B.kkt_solve(h, np.ascontiguousarray(r), x)
        return 0, x
    except B.KKTError as e:
        return e.status, x


def _good_solve_after(B, p, h):
    st, x = _solve_status(B, h, p.a_vals, p.b_vals, p.c_vals, p.rhs)
    assert st == 0
    assert oracle.backward_error(p, x) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_nan_in_a_values_is_reported(name, prec):
    _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS[name])
    h = B.kkt_analyze(p, B.kkt_default_options(prec))
    try:
        a = np.array(p.a_vals, dtype=np.float64, copy=True).reshape(p.N, -1)
        a[1, a.shape[1] // 2] = np.nan
        st, _ = _solve_status(B, h, a, p.b_vals, p.c_vals, p.rhs)
        assert st == KKT_ERR_NONFINITE
        assert np.isnan(B.kkt_get_info(h)["rel_residual"])
        _good_solve_after(B, p, h)
    finally:
        B.kkt_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_inf_in_rhs_is_reported(prec):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["grid30_n24"])
    h = B.kkt_analyze(p, B.kkt_default_options(prec))
    try:
        dev = torch.device("cuda:0")
        up = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
        r = np.array(p.rhs, copy=True)
        r[3] = np.inf
        B.kkt_factor(h, up(p.a_vals), up(p.b_vals), up(p.c_vals))
        x = torch.empty(p.nK, dtype=torch.float64, device=dev)
        with pytest.raises(B.KKTError) as ei:
            B.kkt_solve(h, up(r), x)
        assert ei.value.status == KKT_ERR_NONFINITE
        # an Inf in the coupling rows' right-hand side too
        r = np.array(p.rhs, copy=True)
        r[-1] = -np.inf
        with pytest.raises(B.KKTError) as ei:
            B.kkt_solve(h, up(r), x)
        assert ei.value.status == KKT_ERR_NONFINITE
        _good_solve_after(B, p, h)
    finally:
        B.kkt_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_all_zero_block_is_reported(name, prec):
    _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS[name])
    h = B.kkt_analyze(p, B.kkt_default_options(prec))
    try:
        a = np.array(p.a_vals, dtype=np.float64, copy=True).reshape(p.N, -1)
        a[2, :] = 0.0
        st, _ = _solve_status(B, h, a, p.b_vals, p.c_vals, p.rhs)
        assert st != 0
        assert st == KKT_ERR_NONFINITE
        assert B.kkt_get_info(h)["n_zero"] >= p.nA  # every pivot of block 2
        _good_solve_after(B, p, h)
    finally:
        B.kkt_destroy(h)


def test_batch_reports_the_nonfinite_system():
    """kkt_batch_factor_solve passes the status of a bad system through and
    solves the others."""
    _torch()
    from paper_1907_05420_gb300 import binding as B

    probs = [make_problem(CONFIGS[n]) for n in ("small", "grid30_n24", "small")]
    hs = [B.kkt_analyze(q) for q in probs]
    try:
        a = [np.array(q.a_vals, dtype=np.float64, copy=True).reshape(-1) for q in probs]
        a[1][5] = np.nan
        xs = [np.empty(q.nK) for q in probs]
        with pytest.raises(B.KKTError) as ei:
            B.kkt_batch_factor_solve(hs, a, [np.ascontiguousarray(q.b_vals) for q in probs],
                                     [np.ascontiguousarray(q.c_vals) for q in probs],
                                     [np.ascontiguousarray(q.rhs) for q in probs], xs, streams=2)
        assert ei.value.status == KKT_ERR_NONFINITE
        for i in (0, 2):
            assert oracle.backward_error(probs[i], xs[i]) <= 1e-10
    finally:
        for h in hs:
            B.kkt_destroy(h)
