"""Named workloads: the MPOPF configurations, their variant with the paper's
own cumulative coupling, and SCOPF instances on the same synthetic grids.

    <config>            make_problem(CONFIGS[config])
    <config>_paper      make_problem(CONFIGS[config], coupling="paper")
    scopf<buses>_c<k>   make_scopf on the grid of the configuration with that
                        bus count, with k line contingencies (k + 1 blocks)

This module only names inputs; it contains nothing of the Schur method.
"""
from __future__ import annotations

import re

from .mpopf import CONFIGS, GridSpec, KKTProblem, make_problem
from .scopf import make_scopf

_SCOPF = re.compile(r"^scopf(\d+)_c(\d+)$")


def _grid_of(buses: int) -> GridSpec:
    for spec in CONFIGS.values():
        if spec.n_bus == buses:
            return spec
    raise KeyError(f"no configuration with {buses} buses")


def is_workload(name: str) -> bool:
    try:
        workload_spec(name)
        return True
    except KeyError:
        return False


def workload_spec(name: str):
    """(kind, spec, extra) of a named workload; KeyError if unknown."""
    if name in CONFIGS:
        return "mpopf", CONFIGS[name], None
    if name.endswith("_paper") and name[:-6] in CONFIGS:
        return "paper", CONFIGS[name[:-6]], None
    m = _SCOPF.match(name)
    if m:
        return "scopf", _grid_of(int(m.group(1))), int(m.group(2))
    raise KeyError(name)


def build_workload(name: str) -> KKTProblem:
    kind, spec, extra = workload_spec(name)
    if kind == "mpopf":
        return make_problem(spec)
    if kind == "paper":
        return make_problem(spec, coupling="paper")
    return make_scopf(spec, extra)


def describe_workload(name: str) -> str:
    kind, g, extra = workload_spec(name)
    grid = f"synthetic {g.n_bus:,}-bus grid, {g.n_line:,} lines, {g.n_gen:,} generators"
    if kind == "scopf":
        return f"{name}: SCOPF on the {grid}; {extra} line contingencies ({extra + 1} blocks)"
    p = f"{grid}, {g.n_stor:,} storage units, N={g.n_per} periods"
    if kind == "paper":
        return f"{name}: {p}; the paper's cumulative coupling (C = 0)"
    return f"{name}: {p}; blocks nA={g.n_a:,}; S {g.n_c:,} x {g.n_c:,}"
