"""kkt_solve with the refinement loop on the device (device_refine: one CUDA
graph, the loop a WHILE conditional node, the convergence test a one-thread
kernel) against the host loop on the same factorization: the same solution
bit for bit, the same number of steps, eta and fallback, over modes that take
no step, several steps, and the FP64 fallback; repeated solves replay the
graph, also after a fallback to the FP64-accurate factor of S and after a
new factor; a NaN in the right-hand side is reported as without it."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _solves(p, prec, rhs_list, **opts):
    from paper_1907_05420_gb300 import binding as B

    out = {}
    for dev in (0, 1):
        h = B.kkt_analyze(p, B.kkt_default_options(prec, device_refine=dev, **opts))
        try:
            B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                         np.ascontiguousarray(p.c_vals))
            res = []
            # a second factor after the solves: a TF32 handle that fell back to the
            # FP64-accurate factor of S returns to its FP32 one (the other graph)
            for refactor in (False, True):
                if refactor:
                    B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                                 np.ascontiguousarray(p.c_vals))
                for r in rhs_list:
                    x = np.empty(p.nK)
                    B.kkt_solve(h, np.ascontiguousarray(r), x, allow_not_converged=True)
                    info = B.kkt_get_info(h)
                    res.append((x, info["refine_steps"], info["rel_residual"], info["fell_back_fp64"]))
        finally:
            B.kkt_destroy(h)
        out[dev] = res
    return out


CASES = [
    ("grid30_n24", "fp64", {}, None),
    ("grid2383_n6", "tf32", {"refine_tol": 1e-13}, None),
    ("grid2383_n6", "bf16", {"refine_tol": 1e-13}, None),
    ("grid30_n24", "tf32", {"structured_s": 2}, "paper"),
]


@pytest.mark.parametrize("name,prec,opts,coupling", CASES)
def test_device_loop_equals_host_loop(name, prec, opts, coupling):
    _torch()
    if name == "grid2383_n6":
        spec = replace(CONFIGS["grid2383_n96"], n_per=6)
    else:
        spec = CONFIGS[name]
    p = make_problem(spec, coupling=coupling) if coupling else make_problem(spec)
    rng = np.random.default_rng(5)
    rhs = [p.rhs, rng.standard_normal(p.nK), p.rhs]
    out = _solves(p, prec, rhs, **opts)
    for (xh, sh, eh, fh), (xd, sd, ed, fd) in zip(out[0], out[1]):
        assert np.array_equal(xh, xd)
        assert (sh, fh) == (sd, fd)
        assert eh == ed
    if prec == "bf16":
        assert out[1][0][3] == 1  # the loop stopped above 1e-13 and the FP64 fallback took over
    for x, _, _, _ in out[1]:
        assert np.all(np.isfinite(x))
    assert oracle.backward_error(p, out[1][0][0]) <= opts.get("refine_tol", 1e-10)


def test_device_loop_reports_a_nan_right_hand_side():
    _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["small"])
    r = p.rhs.copy()
    r[3] = np.nan
    h = B.kkt_analyze(p, B.kkt_default_options("fp64", device_refine=1))
    try:
        B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                     np.ascontiguousarray(p.c_vals))
        x = np.empty(p.nK)
        with pytest.raises(B.KKTError) as ei:
            B.kkt_solve(h, r, x)
        assert ei.value.status == 9
        B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)  # the handle still solves
        assert oracle.backward_error(p, x) <= 1e-10
    finally:
        B.kkt_destroy(h)
