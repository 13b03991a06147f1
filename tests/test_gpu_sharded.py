"""The steps of Algorithm 1 one at a time on the GPU, and the sharded data
flow with every shard on one GPU.

* kkt_factor_blocks + kkt_factor_schur is kkt_factor split in two: the same
  kernels in the same order, so the solution is bitwise the same;
* kkt_solve_front + kkt_solve_coupling + kkt_solve_back is one application of
  the factorization, bitwise that of kkt_solve without a refinement step;
* sharded.solve_in_process runs Algorithm 1's reduce and broadcast over 2 and
  3 shards held by one GPU (GpuShard: the C ABI) and meets the oracle's
  parity bound;
* the TF32 factor of S with 256-wide outer panels (S of order >= 512, dense
  mode) is as close to the FP64-accurate factor as the 64-wide TF32 factor
  (the structured mode, whose envelope is the whole matrix for a dense C).
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem, make_scopf
from tests.kkt_dense import dense_K

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")


@pytest.mark.parametrize("prec", ["fp64", "tf32", "f64emu"])
def test_split_factor_equals_kkt_factor(prec):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    a, b, c, r = (_dev(torch, v) for v in (p.a_vals, p.b_vals, p.c_vals, p.rhs))
    xs = []
    for split in (False, True):
        h = B.kkt_analyze(p, B.kkt_default_options(prec, use_graphs=0))
        try:
            x = torch.empty_like(r)
            if split:
                B.kkt_factor_blocks(h, a, b, c)
                with pytest.raises(B.KKTError) as ei:
                    B.kkt_solve(h, r, x)  # S is not factored yet
                assert ei.value.status == 8
                B.kkt_factor_schur(h)
            else:
                B.kkt_factor(h, a, b, c)
            B.kkt_solve(h, r, x)
            xs.append(x.cpu().numpy())
        finally:
            B.kkt_destroy(h)
    assert np.array_equal(xs[0], xs[1])
    assert oracle.backward_error(p, xs[1]) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_front_coupling_back_is_one_application(prec):
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["grid30_n24"])
    a, b, c, r = (_dev(torch, v) for v in (p.a_vals, p.b_vals, p.c_vals, p.rhs))
    h = B.kkt_analyze(p, B.kkt_default_options(prec, refine_tol=1e300))
    try:
        B.kkt_factor(h, a, b, c)
        x1 = torch.empty_like(r)
        B.kkt_solve(h, r, x1)  # refine_tol 1e300: no refinement step
        assert B.kkt_get_info(h)["refine_steps"] == 0
        t = torch.empty(p.nC, dtype=torch.float64, device="cuda:0")
        xg = torch.empty_like(t)
        x2 = torch.empty_like(r)
        with pytest.raises(B.KKTError):
            B.kkt_solve_back(h, xg, x2)  # no front half yet
        B.kkt_solve_front(h, r, t)
        B.kkt_solve_coupling(h, t, xg)
        B.kkt_solve_back(h, xg, x2)
        # the residual and the norms of the refinement pieces
        rho = torch.empty_like(r)
        B.kkt_residual(h, r, x2, rho)
        rs = torch.empty_like(r)
        B.kkt_abs_rowsums(h, rs)
        knorm = B.kkt_norm_inf(h, rs)
        rn = B.kkt_norm_inf(h, rho)
        xn = B.kkt_norm_inf(h, x2)
        torch.cuda.synchronize()
    finally:
        B.kkt_destroy(h)
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    xh = x2.cpu().numpy()
    rho = rho.cpu().numpy()
    res = p.rhs - oracle.kkt_matvec(p, xh)
    # the two residuals differ by the rounding of K x only
    bound = 64 * EPS * (oracle.kkt_norm_inf(p) * np.max(np.abs(xh)) + np.max(np.abs(p.rhs)))
    assert np.max(np.abs(rho - res)) <= bound
    assert knorm == pytest.approx(oracle.kkt_norm_inf(p), rel=1e-14)
    assert np.allclose(rs.cpu().numpy(), np.abs(dense_K(p)).sum(axis=1), rtol=1e-14, atol=0)
    assert xn == np.max(np.abs(xh)) and rn == np.max(np.abs(rho))


def test_norm_inf_keeps_nan_and_accumulate():
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = make_problem(CONFIGS["small"])
    h = B.kkt_analyze(p)
    try:
        v = torch.arange(1000, dtype=torch.float64, device="cuda:0") - 700.0
        assert B.kkt_norm_inf(h, v) == 700.0
        v[333] = float("nan")
        assert np.isnan(B.kkt_norm_inf(h, v))
        dst = torch.zeros(5 * 7, dtype=torch.float64, device="cuda:0")
        src = torch.arange(3 * 2, dtype=torch.float64, device="cuda:0") + 1.0
        B.kkt_accumulate(dst.data_ptr() + 8 * (1 + 2 * 5), 5, src, 3, 3, 2)  # a 3 x 2 block at (1, 2)
        B.kkt_accumulate(dst.data_ptr() + 8 * (1 + 2 * 5), 5, src, 3, 3, 2)
        got = dst.cpu().numpy().reshape(7, 5).T  # column-major 5 x 7
        want = np.zeros((5, 7))
        want[1:4, 2:4] = 2.0 * np.arange(1, 7).reshape(2, 3).T
        assert np.array_equal(got, want)
    finally:
        B.kkt_destroy(h)


@pytest.mark.parametrize("name,nshards,prec", [("grid30_n24", 2, "fp64"), ("grid30_n24", 3, "tf32"),
                                               ("grid30_n24", 4, "f64emu"), ("paper30", 2, "fp64"),
                                               ("scopf30", 2, "fp64"), ("grid2383_n6", 3, "tf32")])
def test_in_process_shards_match_the_oracle(name, nshards, prec):
    _torch()
    from paper_1907_05420_gb300 import binding as B
    from paper_1907_05420_gb300.sharded import GpuShard, solve_in_process

    if name == "paper30":
        p = make_problem(CONFIGS["grid30_n24"], coupling="paper")
    elif name == "scopf30":
        p = make_scopf(CONFIGS["grid30_n24"], 3)
    elif name == "grid2383_n6":
        p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6, name="grid2383_n6"))
    else:
        p = make_problem(CONFIGS[name])
    shards = []

    def backend(sub):
        shards.append(GpuShard(sub, B.kkt_default_options(prec)))
        return shards[-1]

    try:
        x, eta_dev, steps = solve_in_process(p, nshards, backend)
    finally:
        for s in shards:
            s.close()
    assert len(shards) == nshards
    eta = oracle.backward_error(p, x)
    assert eta <= 1e-10, (eta, eta_dev, steps)
    assert eta_dev <= 1e-10
    if p.nK <= 4000:
        ref = oracle.kkt_solve(p)
        kappa = np.linalg.cond(dense_K(p))
        err = np.max(np.abs(x - ref["x"])) / np.max(np.abs(ref["x"]))
        assert err <= 10 * kappa * max(eta, oracle.backward_error(p, ref["x"]), EPS), err


def _dense_c_system(nC, seed):
    """One 2 x 2 quasidefinite block, no coupling entries, and a dense SPD C of
    order nC with eigenvalues log-uniform in [1, 1e3]: S = C, so the factor of
    S is a plain dense LDL^T of a well-conditioned matrix."""
    import types

    rng = np.random.Generator(np.random.PCG64(seed))
    Q, _ = np.linalg.qr(rng.standard_normal((nC, nC)))
    C = (Q * np.exp(rng.uniform(0.0, np.log(1e3), nC))) @ Q.T
    C = 0.5 * (C + C.T)
    return types.SimpleNamespace(
        N=1, nA=2, nP=1, nC=nC, nK=2 + nC, c_kind=1,
        a_rowptr=np.array([0, 1, 3], np.int32), a_col=np.array([0, 0, 1], np.int32),
        a_vals=np.array([[1.0, 1.0, -1e-8]]), b_blockptr=np.zeros(2, np.int32),
        b_row=np.zeros(0, np.int32), b_col=np.zeros(0, np.int32), b_vals=np.zeros(0),
        c_vals=np.ascontiguousarray(C.reshape(-1)), rhs=rng.standard_normal(2 + nC))


@pytest.mark.parametrize("case", ["scopf2383", "dense_c_1100", "dense_c_2000"])
def test_tf32_wide_factor_matches_the_64_wide_one(case):
    """The factor of S from 256-wide outer panels (TF32, S of order >= 512) is
    as close to the FP64-accurate factor as the 64-wide one (the structured
    mode, whose envelope is the whole matrix for a dense C): S of the SCOPF
    workload (order 652, a mild barrier so that the FP32 factors stay
    comparable) and dense S of order 1,100 and 2,000 (ragged last panels;
    tile rows of up to 8 tiles per CTA)."""
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    if case == "scopf2383":
        p = make_scopf(replace(CONFIGS["grid2383_n96"], bar_lo=1e-2, bar_hi=1e2, name="scopf2383_mild"), 2)
    else:
        p = _dense_c_system(int(case.split("_")[-1]), 7)
    assert p.nC >= 512 and p.c_kind == 1
    a, b, c, r = (_dev(torch, v) for v in (p.a_vals, p.b_vals, p.c_vals, p.rhs))
    F = {}
    xs = {}
    for key, prec, st in (("wide", "tf32", 0), ("w64", "tf32", 1), ("f64", "f64emu", 0)):
        h = B.kkt_analyze(p, B.kkt_default_options(prec, structured_s=st))
        try:
            B.kkt_factor(h, a, b, c)
            out = torch.empty(p.nC * p.nC, dtype=torch.float64, device="cuda:0")
            B.kkt_schur_factor_copy(h, out)
            x = torch.empty_like(r)
            B.kkt_solve(h, r, x)
            info = B.kkt_get_info(h)
            F[key] = np.tril(out.cpu().numpy().reshape(p.nC, p.nC).T)
            xs[key] = (x.cpu().numpy(), info)
        finally:
            B.kkt_destroy(h)
    scale = np.max(np.abs(F["f64"]))
    e_wide = np.max(np.abs(F["wide"] - F["f64"])) / scale
    e_64 = np.max(np.abs(F["w64"] - F["f64"])) / scale
    assert e_wide <= 4.0 * max(e_64, 1e-6), (e_wide, e_64)
    assert e_wide <= 1e-2, e_wide
    for key in ("wide", "w64"):
        x, info = xs[key]
        assert oracle.backward_error(p, x) <= 1e-10
        assert info["fell_back_fp64"] == 0, key


@pytest.mark.parametrize("case", ["dense_c_1100", "dense_c_2000"])
def test_emulated_wide_factor_matches_fp64(case):
    """The emulated-FP64 factor of S with 256-wide outer panels (balanced
    digits, K = 256 per epilogue) against the FP64 factor on the CUDA cores
    and the 64-wide emulated factor (structured mode, full envelope), on a
    well-conditioned dense S: all three are FP64-accurate, so they agree to a
    few units of FP64 rounding times the growth of the factorization."""
    torch = _torch()
    from paper_1907_05420_gb300 import binding as B

    p = _dense_c_system(int(case.split("_")[-1]), 11)
    a, b, c, r = (_dev(torch, v) for v in (p.a_vals, p.b_vals, p.c_vals, p.rhs))
    F = {}
    for key, prec, st in (("wide", "f64emu", 0), ("w64", "f64emu", 1), ("f64", "fp64", 0)):
        h = B.kkt_analyze(p, B.kkt_default_options(prec, structured_s=st))
        try:
            B.kkt_factor(h, a, b, c)
            out = torch.empty(p.nC * p.nC, dtype=torch.float64, device="cuda:0")
            B.kkt_schur_factor_copy(h, out)
            x = torch.empty_like(r)
            B.kkt_solve(h, r, x)
            F[key] = np.tril(out.cpu().numpy().reshape(p.nC, p.nC).T)
            assert oracle.backward_error(p, x.cpu().numpy()) <= 1e-14
            info = B.kkt_get_info(h)
            assert [info["n_pos"], info["n_neg"], info["n_zero"]] == [p.nP + p.nC, p.nA - p.nP, 0]
        finally:
            B.kkt_destroy(h)
    scale = np.max(np.abs(F["f64"]))
    assert np.max(np.abs(F["wide"] - F["f64"])) <= 1e-11 * scale
    assert np.max(np.abs(F["wide"] - F["w64"])) <= 1e-11 * scale
