"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Criteria (FP64 mode):
* inertia: bit-exact against (N*nP + nC, N*(nA-nP), 0);
* normwise backward error eta = ||r-Kx||_inf/(||K||_inf ||x||_inf + ||r||_inf)
  evaluated by the oracle's FP64 K x: <= 1e-10 (the solver's stated target);
* element by element against the oracle's x: both are backward-stable
  solutions, so |x_gpu - x_oracle|_inf <= kappa(K) * (eta_gpu + eta_oracle)
  * ||x||_inf up to a modest constant.  Where kappa(K) is computable (dense
  K up to a few thousand rows) the test uses 10 * kappa * max(eta, eps).
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, GridSpec, make_problem, reseed_barrier
from tests.kkt_dense import dense_K

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_solve(p, prec="fp64", device_arrays=False, **opts):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    opt = B.kkt_default_options(prec, **opts)
    h = B.kkt_analyze(p, opt)
    try:
        if device_arrays:
            dev = torch.device("cuda:0")
            a = torch.from_numpy(np.ascontiguousarray(p.a_vals)).to(dev)
            b = torch.from_numpy(np.ascontiguousarray(p.b_vals)).to(dev)
            c = torch.from_numpy(np.ascontiguousarray(p.c_vals)).to(dev)
            r = torch.from_numpy(np.ascontiguousarray(p.rhs)).to(dev)
            x = torch.empty_like(r)
            B.kkt_factor(h, a, b, c)
            B.kkt_solve(h, r, x)
            xs = x.cpu().numpy()
        else:
            B.kkt_factor(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                         np.ascontiguousarray(p.c_vals))
            xs = np.empty(p.nK)
            B.kkt_solve(h, np.ascontiguousarray(p.rhs), xs)
        info = B.kkt_get_info(h)
    finally:
        B.kkt_destroy(h)
    return xs, info


def expected_inertia(p):
    return [p.N * p.nP + p.nC, p.N * (p.nA - p.nP), 0]


def check_against_oracle(p, x, info, kappa=None, eta_max=1e-10, inertia=True):
    ref = oracle.kkt_solve(p)
    eta = oracle.backward_error(p, x)
    eta_ref = oracle.backward_error(p, ref["x"])
    if inertia:
        assert [info["n_pos"], info["n_neg"], info["n_zero"]] == expected_inertia(p)
    assert list(ref["inertia"]) == expected_inertia(p)
    assert eta <= eta_max, eta
    err = np.max(np.abs(x - ref["x"])) / np.max(np.abs(ref["x"]))
    if kappa is not None:
        tol = 10.0 * kappa * max(eta, eta_ref, EPS)
        assert err <= tol, (err, tol)
    return eta, err


@pytest.mark.parametrize("name", ["tiny", "small", "grid30_n24"])
def test_fp64_matches_oracle(name):
    p = make_problem(CONFIGS[name])
    x, info = gpu_solve(p)
    kappa = np.linalg.cond(dense_K(p))
    check_against_oracle(p, x, info, kappa)
    assert info["n_perturbed"] == 0


def test_fp64_device_arrays():
    p = make_problem(CONFIGS["grid30_n24"])
    x, info = gpu_solve(p, device_arrays=True)
    xh, _ = gpu_solve(p, device_arrays=False)
    assert np.array_equal(x, xh)  # same kernels, same order: bitwise equal
    check_against_oracle(p, x, info, np.linalg.cond(dense_K(p)))


def test_fp64_2383_bus_grid_short_horizon():
    spec = replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6")
    p = make_problem(spec)
    x, info = gpu_solve(p)
    eta, err = check_against_oracle(p, x, info)
    print(f"eta={eta:.2e} err={err:.2e} steps={info['refine_steps']}")
    assert info["n_perturbed"] == 0


def test_zero_coupling_values():
    p = make_problem(CONFIGS["small"], zero_b=True)
    x, info = gpu_solve(p)
    check_against_oracle(p, x, info, np.linalg.cond(dense_K(p)))
    g = p.N * p.nA
    assert np.allclose(x[g:], p.rhs[g:] / p.c_vals, rtol=1e-13)


def test_single_block_without_coupling():
    p = make_problem(CONFIGS["small"])
    q = replace(p, N=1, nC=0, a_vals=p.a_vals[:1].copy(),
                b_blockptr=np.zeros(2, np.int32), b_row=np.zeros(0, np.int32),
                b_col=np.zeros(0, np.int32), b_vals=np.zeros(0), c_vals=np.zeros(0),
                rhs=p.rhs[: p.nA].copy())
    x, info = gpu_solve(q)
    check_against_oracle(q, x, info, np.linalg.cond(dense_K(q)))


def test_refactor_same_handle_new_values():
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["grid30_n24"])
    q = reseed_barrier(p, 77)
    h = B.kkt_analyze(p)
    try:
        out = []
        for prob in (p, q, p):
            B.kkt_factor(h, np.ascontiguousarray(prob.a_vals), prob.b_vals, prob.c_vals)
            x = np.empty(prob.nK)
            B.kkt_solve(h, prob.rhs, x)
            out.append((x, B.kkt_get_info(h)))
    finally:
        B.kkt_destroy(h)
    for prob, (x, info) in zip((p, q, p), out):
        check_against_oracle(prob, x, info, np.linalg.cond(dense_K(prob)))
    assert np.array_equal(out[0][0], out[2][0])
    del torch


def test_full_size_2383_bus_96_periods_backward_error():
    """The benchmarked workload: properties that hold at any size."""
    p = make_problem(CONFIGS["grid2383_n96"])
    x, info = gpu_solve(p)
    assert [info["n_pos"], info["n_neg"], info["n_zero"]] == expected_inertia(p)
    assert oracle.backward_error(p, x) <= 1e-10


AUG_SPECS = {  # grids whose dense tail lies wholly inside the reach of the coupling rows
    "aug14": GridSpec(14, 18, 3, 2, 4, 1e-6, 1e6, 102, "aug14"),
    "aug15": GridSpec(15, 19, 3, 2, 4, 1e-6, 1e6, 103, "aug15"),
}


@pytest.mark.parametrize("name", ["tiny", "grid30_n24", "aug14", "aug15", "grid2383_n6"])
def test_dense_tail_modes(name):
    """The dense tail factors the top of the tree as one triangle per block
    (mode 1: FP64 updates; mode 2: emulated-FP64 tensor-core updates); in every
    mode the solution meets the oracle's criteria and the pivot signs
    (inertia) are the expected ones."""
    spec = (replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6") if name == "grid2383_n6"
            else AUG_SPECS.get(name) or CONFIGS[name])
    p = make_problem(spec)
    kappa = np.linalg.cond(dense_K(p)) if p.nK <= 4000 else None
    for mode in (0, 1, 2):
        x, info = gpu_solve(p, dense_tail=mode)
        assert (info["dense_tail_cols"] > 0) == (mode > 0)
        check_against_oracle(p, x, info, kappa)
        assert info["n_perturbed"] == 0
        if name == "grid2383_n6" and mode:
            assert info["dense_tail_cols"] >= 400
        assert info["tail_augmented"] == (1 if mode else 0)


@pytest.mark.parametrize("prec", ["tf32", "f64emu", "fp64"])
def test_default_tail(prec):
    """Every mode takes an augmented dense tail by default (emulated-FP64
    updates in the reduced modes, FP64 on the CUDA cores in the FP64 mode)."""
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    x, info = gpu_solve(p, prec)
    assert info["dense_tail_cols"] >= 400 and info["tail_augmented"] == 1
    assert info["tail_ratio"] == 1.5
    assert oracle.backward_error(p, x) <= 1e-10


def test_autotuned_tail():
    """The autotuner times the distinct tails of its candidate ratios and keeps
    one of them; the solution is as accurate."""
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    x, info = gpu_solve(p, "tf32", autotune=1)
    assert info["autotune_candidates"] >= 2
    assert info["tail_ratio"] in (1.0, 1.25, 1.5, 2.0, 3.0)
    assert oracle.backward_error(p, x) <= 1e-10


def test_explicit_tail_ratio():
    """A set tail_ratio fixes the cost ratio (the autotuner is skipped); a larger
    ratio gives a tail at least as long, and the CPU inspection library, which
    runs the same rule, reports the same tail for the FP64 mode."""
    from test_symbolic import analyze

    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    cols = []
    for r in (1.0, 3.0):
        x, info = gpu_solve(p, "tf32", tail_ratio=r, autotune=1)
        assert info["tail_ratio"] == r and info["autotune_candidates"] == 0
        assert oracle.backward_error(p, x) <= 1e-10
        cols.append(info["dense_tail_cols"])
    assert cols[1] >= cols[0] > 0
    _, info = gpu_solve(p, "fp64")
    a = analyze(p)
    assert info["dense_tail_cols"] == a["n"] - a["tail_col"]


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_graph_replay_matches_direct_launches(prec):
    """The factor's launch sequence is captured once as a CUDA graph and
    replayed: each replay (with new values) gives bitwise the result of the
    same sequence launched directly."""
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    q = reseed_barrier(p, 91)
    out = {}
    for graphs in (0, 1):
        h = B.kkt_analyze(p, B.kkt_default_options(prec, use_graphs=graphs))
        try:
            xs = []
            for prob in (p, q, p):
                B.kkt_factor(h, np.ascontiguousarray(prob.a_vals), prob.b_vals, prob.c_vals)
                x = np.empty(prob.nK)
                B.kkt_solve(h, prob.rhs, x)
                xs.append(x)
            out[graphs] = (xs, B.kkt_get_info(h))
        finally:
            B.kkt_destroy(h)
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[1][0][0], out[1][0][2])
    # the launch count covers the replayed kernels too
    assert out[1][1]["n_launches"] == out[0][1]["n_launches"]
    for prob, x in zip((p, q), out[1][0][:2]):
        assert oracle.backward_error(prob, x) <= 1e-10
    del torch


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_early_solve_matches(prec):
    """With early_solve the first application's front half runs on another
    stream beside the dense factor of S: the same kernels in the same order
    per stream, so bitwise the same solution."""
    _torch()
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    x0, _ = gpu_solve(p, prec, early_solve=0)
    x1, _ = gpu_solve(p, prec, early_solve=1)
    assert np.array_equal(x0, x1)
    x2, _ = gpu_solve(p, prec, early_solve=1, device_arrays=True)
    assert np.array_equal(x0, x2)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_full_size_2383_bus_96_periods_reduced_modes(prec):
    """The reduced-precision factors of S at full size: eta by the oracle's
    residual after GMRES refinement to 1e-12, and the inertia of K from
    kkt_factor_inertia, which recounts the pivot signs of S on an
    FP64-accurate factor when the reduced-precision ones disagree (one TF32
    pivot sign of this S is wrong)."""
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["grid2383_n96"])
    h = B.kkt_analyze(p, B.kkt_default_options(prec, refine_mode=1, refine_tol=1e-12, max_refine=20))
    try:
        res = B.kkt_factor_inertia(h, np.ascontiguousarray(p.a_vals), np.ascontiguousarray(p.b_vals),
                                   np.ascontiguousarray(p.c_vals))
        assert res["trials"] == 1 and res["delta_w"] == 0.0
        info = B.kkt_get_info(h)
        assert [info["n_pos"], info["n_neg"], info["n_zero"]] == expected_inertia(p)
        x = np.empty(p.nK)
        B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
        assert oracle.backward_error(p, x) <= 1e-12
    finally:
        B.kkt_destroy(h)
    del torch
