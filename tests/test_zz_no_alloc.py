"""kkt_solve_noalloc: the solve entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc while they solve, e.g. a
serving process that gives all device memory to its own pool at start-up and
must stay inside that budget, or a latency-critical loop that cannot take the
device-wide synchronization an allocation may imply.  Its work vectors live in
one file-scope device array shared by every call.

Checked here through the C ABI: two calls in a row give the same solution as
kkt_solve (the existing entry point) within the parity tolerance of the other
GPU tests, 10 * kappa(K) * max(eta, eps) relative to ||x||_inf; a second
system reuses the shared array correctly; an oversized system is rejected.
The file is named so that pytest collects it last.
"""
import types

import numpy as np
import pytest

import oracle
from gen import CONFIGS, GridSpec, make_problem
from tests.kkt_dense import dense_K

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _factored(p, torch, B, opt=None):
    dev = torch.device("cuda:0")
    h = B.kkt_analyze(p, opt)
    a = torch.from_numpy(np.ascontiguousarray(p.a_vals)).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(p.b_vals)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(p.c_vals)).to(dev)
    B.kkt_factor(h, a, b, c)
    r = torch.from_numpy(np.ascontiguousarray(p.rhs)).to(dev)
    return h, r


@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_noalloc_matches_kkt_solve_on_two_calls(name):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS[name])
    h, r = _factored(p, torch, B)
    try:
        x_ref = torch.empty_like(r)
        B.kkt_solve(h, r, x_ref)
        outs = []
        for _ in range(2):
            x = torch.full_like(r, float("nan"))
            B.kkt_solve_noalloc(h, r, x)
            torch.cuda.synchronize()
            outs.append(x.cpu().numpy())
    finally:
        B.kkt_destroy(h)
    x_ref = x_ref.cpu().numpy()
    kappa = np.linalg.cond(dense_K(p))
    eta_ref = oracle.backward_error(p, x_ref)
    for x in outs:
        eta = oracle.backward_error(p, x)
        tol = 10.0 * kappa * max(eta, eta_ref, EPS)
        err = np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref))
        assert err <= tol, (err, tol)
        assert eta <= 1e-10


# Cases where the work-vector path departs most from kkt_solve's kernels: a
# dense tail whose factor was scattered back into the panels (FP64 and
# emulated-FP64 updates, augmented by the coupling rows), the envelope-limited
# factor of S, the emulated-FP64 factor of S, and the structured S of the
# paper's cumulative coupling.
AUG14 = GridSpec(14, 18, 3, 2, 4, 1e-6, 1e6, 102, "aug14")
CASES = {
    "aug14_tail_fp64": (AUG14, "fp64", {"dense_tail": 1}),
    "aug14_tail_emulated": (AUG14, "f64emu", {"dense_tail": 2}),
    "grid30_structured_s": (CONFIGS["grid30_n24"], "fp64", {"structured_s": 1}),
    "grid30_f64emu": (CONFIGS["grid30_n24"], "f64emu", {}),
    "grid30_paper_structured": (CONFIGS["grid30_n24"], "f64emu", {"structured_s": 2}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_kkt_solve_tail_structured_emulated(case):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    spec, prec, kw = CASES[case]
    p = make_problem(spec, coupling="paper") if kw.get("structured_s") == 2 else make_problem(spec)
    h, r = _factored(p, torch, B, B.kkt_default_options(prec, **kw))
    try:
        info = B.kkt_get_info(h)
        if "dense_tail" in kw:
            assert info["dense_tail_cols"] > 0 and info["tail_augmented"] == 1
        x_ref = torch.empty_like(r)
        B.kkt_solve(h, r, x_ref)
        outs = []
        for _ in range(2):
            x = torch.full_like(r, float("nan"))
            B.kkt_solve_noalloc(h, r, x)
            torch.cuda.synchronize()
            outs.append(x.cpu().numpy())
    finally:
        B.kkt_destroy(h)
    x_ref = x_ref.cpu().numpy()
    kappa = np.linalg.cond(dense_K(p))
    eta_ref = oracle.backward_error(p, x_ref)
    assert np.array_equal(outs[0], outs[1])
    for x in outs:
        eta = oracle.backward_error(p, x)
        assert eta <= 1e-10, eta
        tol = 10.0 * kappa * max(eta, eta_ref, EPS)
        err = np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref))
        assert err <= tol, (err, tol)


def test_noalloc_second_system_reuses_the_shared_array():
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p1 = make_problem(CONFIGS["grid30_n24"])
    p2 = make_problem(CONFIGS["small"])
    h1, r1 = _factored(p1, torch, B)
    h2, r2 = _factored(p2, torch, B)
    try:
        xs = []
        for h, r in ((h1, r1), (h2, r2), (h1, r1)):
            x = torch.empty_like(r)
            B.kkt_solve_noalloc(h, r, x)
            torch.cuda.synchronize()
            xs.append(x.cpu().numpy())
    finally:
        B.kkt_destroy(h1)
        B.kkt_destroy(h2)
    assert np.array_equal(xs[0], xs[2])
    assert oracle.backward_error(p2, xs[1]) <= 1e-10


def test_noalloc_rejects_a_system_beyond_the_static_array():
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    N, nA = 40, 60000  # N * nA = 2.4e6 doubles > 2^21
    p = types.SimpleNamespace(
        N=N, nA=nA, nP=nA, nC=0, c_kind=0,
        a_rowptr=np.arange(nA + 1, dtype=np.int32), a_col=np.arange(nA, dtype=np.int32),
        a_vals=np.ones((N, nA)), b_blockptr=np.zeros(N + 1, np.int32),
        b_row=np.zeros(0, np.int32), b_col=np.zeros(0, np.int32), b_vals=np.zeros(0),
        c_vals=np.zeros(0), rhs=np.ones(N * nA))
    h, r = _factored(p, torch, B)
    try:
        x = torch.empty_like(r)
        with pytest.raises(B.KKTError) as ei:
            B.kkt_solve_noalloc(h, r, x)
        assert ei.value.status == 1
        assert "static array" in str(ei.value)
    finally:
        B.kkt_destroy(h)
