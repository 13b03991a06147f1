"""Host-side logic of bench.py that runs without a GPU: the bounded CPU
baseline sample."""
import pytest

import bench
from gen import CONFIGS, make_problem


def test_cpu_baseline_full_solve_when_small(monkeypatch):
    p = make_problem(CONFIGS["grid30_n24"])
    fields, out = bench.cpu_baseline_sample("grid30_n24", p, 1e5)
    assert out is not None and fields["value"] > 0 and fields["kind"] == "oracle"
    assert fields["sample"].startswith("1 full solve")


def test_cpu_baseline_sampled_and_scaled_when_large(monkeypatch):
    """Above the work budget the oracle solves the first N' periods, N' the
    largest horizon within the budget, and the rate is scaled by the ratio of
    the estimated work."""
    p = make_problem(CONFIGS["grid30_n24"])
    block, ns = 1e5, p.nC // p.N
    est = lambda n: n * block + (n * ns) ** 3 / 3.0  # noqa: E731
    monkeypatch.setattr(bench, "CPU_SAMPLE_FLOPS", est(9) + 1.0)
    fields, out = bench.cpu_baseline_sample("grid30_n24", p, block)
    assert out is None
    assert "first 9 of 24 periods" in fields["sample"]
    assert f"x{est(24) / est(9):.1f}" in fields["sample"]
    assert fields["value"] > 0
