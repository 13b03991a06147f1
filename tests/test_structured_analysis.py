"""kkt_analyze with structured_s = 2 refuses patterns without the cumulative
structure (Sec. 4.3: block i's coupling columns zero before period i and the
same for every later period; C diagonal).  The refusal comes from the host
analysis before any device call, so these run without a GPU."""
from dataclasses import replace

import numpy as np
import pytest

from gen import CONFIGS, make_problem


def _analyze(p):
    from paper_1907_05420_gb300 import binding as B

    try:
        B.load()
    except OSError as e:  # the CUDA runtime library itself is missing
        pytest.skip(f"cannot load libkkt_schur.so here: {e}")
    with pytest.raises(B.KKTError) as ei:
        B.kkt_analyze(p, B.kkt_default_options("fp64", structured_s=2))
    assert ei.value.status == 1
    return str(ei.value)


def _paper():
    return make_problem(CONFIGS["small"], coupling="paper")


def test_adjacent_coupling_is_refused():
    msg = _analyze(make_problem(CONFIGS["small"]))
    assert "period" in msg


def test_dense_c_is_refused():
    p = _paper()
    c = np.diag(np.asarray(p.c_vals, dtype=np.float64)).reshape(-1)
    assert "diagonal C" in _analyze(replace(p, c_kind=1, c_vals=c))


def test_entry_before_its_block_is_refused():
    p = _paper()
    ns = p.nC // p.N
    bp = np.asarray(p.b_blockptr)
    cols = np.asarray(p.b_col).copy()
    q = int(bp[2])          # first entry of block 2 lies in period 2; move it to period 1
    cols[q] -= ns
    assert "earlier period" in _analyze(replace(p, b_col=cols))


def test_later_periods_with_different_patterns_are_refused():
    p = _paper()
    ns = p.nC // p.N
    bp = np.asarray(p.b_blockptr)
    rows, cols, vals = (np.asarray(a) for a in (p.b_row, p.b_col, p.b_vals))
    # drop block 0's entries in its last period for one row
    keep = np.ones(len(rows), dtype=bool)
    drop = np.flatnonzero((np.arange(len(rows)) < bp[1]) & (cols // ns == p.N - 1))[0]
    keep[drop] = False
    nbp = bp.copy()
    nbp[1:] -= 1
    p2 = replace(p, b_row=rows[keep], b_col=cols[keep], b_vals=vals[keep], b_blockptr=nbp.astype(np.int32))
    assert "differs" in _analyze(p2)


def test_nc_not_a_multiple_of_n_is_refused():
    p = _paper()
    assert "multiple of N" in _analyze(replace(p, nC=p.nC + 1, c_vals=np.append(p.c_vals, 1.0)))
