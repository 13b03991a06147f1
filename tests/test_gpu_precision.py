"""Precision modes of the dense factor of S against the oracle.

KKT_F64_EMULATED factors S FP64-accurately with the trailing update on the BF16
tensor cores (exact digit-slice products); it must meet the same parity bar as
KKT_FP64.  KKT_TF32 / KKT_BF16 factor S in FP32 on the tensor cores; FP64
refinement on K either converges or falls back to the FP64-accurate factor, so
every mode must reach eta <= 1e-10.  The inertia must be exact whenever the
factor of S in use is FP64-accurate (FP64, emulated FP64, or after the
fallback); an FP32 factor of an ill-conditioned S may flip pivot signs.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem
from tests.kkt_dense import dense_K
from tests.test_gpu_parity import check_against_oracle, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64emu", "tf32", "bf16"])
@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_precision_modes_small(name, prec):
    p = make_problem(CONFIGS[name])
    x, info = gpu_solve(p, prec)
    exact_s = prec == "f64emu" or info["fell_back_fp64"]
    check_against_oracle(p, x, info, np.linalg.cond(dense_K(p)), inertia=exact_s)
    if prec == "f64emu":
        assert info["refine_steps"] <= 1


@pytest.mark.parametrize("prec", ["f64emu", "tf32", "bf16"])
def test_precision_modes_2383_bus_short_horizon(prec):
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6))
    x, info = gpu_solve(p, prec)
    exact_s = prec == "f64emu" or info["fell_back_fp64"]
    eta, err = check_against_oracle(p, x, info, inertia=exact_s)
    print(f"{prec}: eta={eta:.2e} err={err:.2e} steps={info['refine_steps']} "
          f"fallback={info['fell_back_fp64']}")


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_reduced_contraction_falls_back_to_fp64_schur(prec):
    """TF32/BF16 contraction on the tensor cores: refinement either converges or
    the fallback rebuilds S from an FP64 contraction; eta <= 1e-10 either way."""
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6))
    x, info = gpu_solve(p, prec, reduced_contraction=1)
    exact_s = bool(info["fell_back_fp64"])
    eta, err = check_against_oracle(p, x, info, inertia=exact_s)
    print(f"{prec}+tc-contraction: eta={eta:.2e} steps={info['refine_steps']} fallback={info['fell_back_fp64']}")
    g = make_problem(CONFIGS["grid30_n24"])
    xg, ig = gpu_solve(g, prec, reduced_contraction=1)
    check_against_oracle(g, xg, ig, np.linalg.cond(dense_K(g)), inertia=bool(ig["fell_back_fp64"]))


def test_emulated_factor_matches_fp64_factor_solution():
    """The emulated FP64 update of S reproduces the FP64 path to near FP64
    accuracy (same block factors); with the emulated dense tail of the block
    factors as well, the backward error stays at the FP64 level."""
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=8))
    x64, _ = gpu_solve(p, "fp64")
    xe, info = gpu_solve(p, "f64emu", dense_tail=0)
    assert oracle.backward_error(p, xe) <= 1e-14
    assert np.max(np.abs(xe - x64)) / np.max(np.abs(x64)) <= 1e-6
    xt, info_t = gpu_solve(p, "f64emu")
    assert info_t["dense_tail_cols"] > 0
    assert oracle.backward_error(p, xt) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "tf32", "f64emu"])
def test_structured_s_equals_dense(prec):
    """The envelope-limited factor only skips exact zeros: bitwise the dense
    result with the same panel width.  The dense TF32 and emulated-FP64
    factors of an S of order >= 512 take 256-wide outer panels instead (one
    accumulation over K = 256 where the structured factor adds four 64-wide
    products), so there the two agree to rounding and both meet the parity
    criterion (the emulated one at the FP64 level)."""
    for p in (make_problem(CONFIGS["grid30_n24"]), make_problem(replace(CONFIGS["grid2383_n96"], n_per=6))):
        xd, infd = gpu_solve(p, prec)
        xs, infs = gpu_solve(p, prec, structured_s=1)
        if prec in ("tf32", "f64emu") and p.nC >= 512:
            assert oracle.backward_error(p, xd) <= (1e-10 if prec == "tf32" else 1e-14)
        else:
            assert np.array_equal(xd, xs)
            assert [infd["n_pos"], infd["n_neg"]] == [infs["n_pos"], infs["n_neg"]]
        assert oracle.backward_error(p, xs) <= 1e-10


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("name", ["small", "grid30_n24"])
def test_gmres_refinement_matches_oracle(name, prec):
    """GMRES refinement (refine_mode 1) meets the same parity bar as the plain
    iteration: eta <= 1e-10 and the oracle's solution within 10 kappa max(eta, eps)."""
    p = make_problem(CONFIGS[name])
    x, info = gpu_solve(p, prec, refine_mode=1)
    check_against_oracle(p, x, info, np.linalg.cond(dense_K(p)), inertia=bool(info["fell_back_fp64"]))


def test_gmres_refinement_reaches_a_tight_tolerance_without_fallback():
    """On the 2,383-bus grid over 6 periods the plain iteration with the TF32
    factor of S stalls above 1e-13 and falls back to the FP64-accurate factor;
    GMRES refinement with the same factor reaches it (8 applications measured),
    and two solves give bitwise the same solution."""
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6))
    xs = []
    for _ in range(2):
        x, info = gpu_solve(p, "tf32", refine_mode=1, refine_tol=1e-13, max_refine=12)
        assert info["fell_back_fp64"] == 0
        assert info["rel_residual"] <= 1e-13
        assert oracle.backward_error(p, x) <= 1e-13
        xs.append(x)
    assert np.array_equal(xs[0], xs[1])
    x0, info0 = gpu_solve(p, "tf32", refine_mode=0, refine_tol=1e-13, max_refine=12)
    assert info0["fell_back_fp64"] == 1 and oracle.backward_error(p, x0) <= 1e-13


def test_refinement_after_the_fallback_has_its_own_budget():
    """BF16 GMRES that uses the whole step budget falls back to the
    FP64-accurate factor of S; the refinement on that factor then has
    max_refine steps of its own, so the solve still meets the tolerance (on the
    9,241-bus system it had none left and stopped at 5.6e-9)."""
    p = make_problem(replace(CONFIGS["grid2383_n96"], n_per=6))
    x, info = gpu_solve(p, "bf16", refine_mode=1, max_refine=2, refine_tol=1e-13)
    assert info["fell_back_fp64"] == 1
    assert oracle.backward_error(p, x) <= 1e-13
    assert info["refine_steps"] <= 2 + 1 + 2
