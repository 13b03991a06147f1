"""Slack elimination on the GPU (Sec. 2) through the C ABI.

* kkt_slack_reduce / kkt_slack_recover against the oracle (oracle/slack.py)
  element by element: both compute every entry with one IEEE operation
  sequence (round to nearest, no fused multiply-adds), so the results are
  bitwise equal; also in place (a_vals = a_base, c_vals = c_base);
* end to end: reduce on the GPU, kkt_factor + kkt_solve of the reduced K,
  recover on the GPU, against the unreduced Newton system of eq. SCOPFhessian
  solved densely by LAPACK, within 10 kappa(M) max(eta, eps).
"""
import numpy as np
import pytest

from gen import CONFIGS, GridSpec, make_ipm_state, make_problem
from oracle import slack as oslack

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
CASES = {
    "tiny_L4": (CONFIGS["tiny"], 4),
    "small_L10": (CONFIGS["small"], 10),
    "grid30_L40": (CONFIGS["grid30_n24"], 40),
    "grid30_L0": (CONFIGS["grid30_n24"], 0),
    "st20_L26": (GridSpec(20, 26, 4, 3, 6, 1e-4, 1e4, 5, "st20"), 26),
}


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _dev_state(torch, st):
    up = lambda v: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to("cuda:0")  # noqa: E731
    return {k: up(getattr(st, k)) for k in ("x", "z", "s", "y", "la", "le", "lcd", "lb", "lf")}, up


@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("case", sorted(CASES))
def test_slack_kernels_equal_the_oracle(case, in_place):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    spec, L = CASES[case]
    p = make_problem(spec, flow_limits=L)
    st = make_ipm_state(p, 23)
    a_ref, c_ref, r_ref = oslack.slack_reduce(p, st)
    rng = np.random.default_rng(5)
    dsol = rng.standard_normal(p.nK) * 10.0 ** rng.uniform(-3, 3, p.nK)
    ds_ref, dz_ref, dy_ref = oslack.slack_recover(p, st, dsol)
    h = B.kkt_analyze(p)
    sl = B.Slack(h, p.ineq_rows)
    try:
        ds_, up = _dev_state(torch, st)
        a_base, c_base = up(st.a_base), up(st.c_base)
        a_out = a_base if in_place else torch.full_like(a_base, float("nan"))
        c_out = c_base if in_place else torch.full_like(c_base, float("nan"))
        rhs = torch.full((p.nK,), float("nan"), dtype=torch.float64, device="cuda:0")
        sl.reduce(ds_, a_base, c_base, a_out, c_out, rhs)
        ds = torch.full((p.N * L,), float("nan"), dtype=torch.float64, device="cuda:0")
        dy = torch.full_like(ds, float("nan"))
        dz = torch.full((p.N * p.nP + p.nC,), float("nan"), dtype=torch.float64, device="cuda:0")
        sl.recover(ds_, up(dsol), ds, dz, dy)
        torch.cuda.synchronize()
    finally:
        sl.close()
        B.kkt_destroy(h)
    assert np.array_equal(a_out.cpu().numpy().reshape(p.N, -1), a_ref)
    assert np.array_equal(c_out.cpu().numpy(), c_ref)
    assert np.array_equal(rhs.cpu().numpy(), r_ref)
    assert np.array_equal(ds.cpu().numpy(), ds_ref)
    assert np.array_equal(dz.cpu().numpy(), dz_ref)
    assert np.array_equal(dy.cpu().numpy(), dy_ref)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
@pytest.mark.parametrize("case", ["small_L10", "grid30_L40", "st20_L26"])
def test_slack_elimination_end_to_end(case, prec):
    """One Newton step of the barrier method through the reduced K."""
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    spec, L = CASES[case]
    p = make_problem(spec, flow_limits=L)
    st = make_ipm_state(p, 29)
    h = B.kkt_analyze(p, B.kkt_default_options(prec))
    sl = B.Slack(h, p.ineq_rows)
    try:
        dst, up = _dev_state(torch, st)
        a = up(st.a_base)
        c = up(st.c_base)
        rhs = torch.empty(p.nK, dtype=torch.float64, device="cuda:0")
        sl.reduce(dst, a, c, a, c, rhs)  # in place, as an interior-point loop would
        B.kkt_factor(h, a, up(p.b_vals), c)
        x = torch.empty_like(rhs)
        B.kkt_solve(h, rhs, x)
        ds = torch.empty(p.N * L, dtype=torch.float64, device="cuda:0")
        dy = torch.empty_like(ds)
        dz = torch.empty(p.N * p.nP + p.nC, dtype=torch.float64, device="cuda:0")
        sl.recover(dst, x, ds, dz, dy)
        torch.cuda.synchronize()
        eta = B.kkt_get_info(h)["rel_residual"]
    finally:
        sl.close()
        B.kkt_destroy(h)
    assert eta <= 1e-10
    M, r, ix = oslack.unreduced_system(p, st)
    full = np.linalg.solve(M, r)
    xh = x.cpu().numpy()
    N, nP, nA, nC = p.N, p.nP, p.nA, p.nC
    blocks = xh[:N * nA].reshape(N, nA)
    ineq = np.asarray(p.ineq_rows)
    eqr = np.setdiff1d(np.arange(nP, nA), ineq)
    got = np.concatenate([blocks[:, :nP].reshape(-1), xh[N * nA:], ds.cpu().numpy(),
                          blocks[:, eqr].reshape(-1), blocks[:, ineq].reshape(-1), dz.cpu().numpy(),
                          dy.cpu().numpy()])
    kappa = np.linalg.cond(M)
    err = np.max(np.abs(got - full)) / np.max(np.abs(full))
    assert err <= 10 * kappa * max(eta, EPS), (err, kappa)
