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


@pytest.mark.parametrize("workload", ["grid30_n24", "grid30_n24_paper", "scopf30_c8"])
def test_reference_arm_prints_the_contract_line(workload):
    """bench.py --impl reference runs the oracle on the host and prints one
    JSON line with the keys the measurement contract asks for."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", workload],
                       capture_output=True, text=True, check=True, timeout=600)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith(workload + ":")
