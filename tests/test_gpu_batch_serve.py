"""Batching and serving: every result is the same alone and in the mix.

The kernels write every entry in a fixed order, so a system solved inside a
batch or among concurrent server requests must give bitwise the same x as the
same system solved alone; each is also checked against the oracle's residual.
"""
import numpy as np
import pytest

import oracle
from gen import GridSpec, make_problem, reseed_barrier

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _mix(count, seed0=500):
    rng = np.random.default_rng(seed0)
    probs = []
    for k in range(count):
        nb = int(rng.integers(30, 160))
        spec = GridSpec(nb, int(1.3 * nb), max(1, nb // 7), max(1, nb // 15),
                        int(rng.choice([6, 12, 24])), 1e-6, 1e6, seed0 + k, f"m{k}")
        probs.append(make_problem(spec))
    return probs


def _alone(B, h, p):
    B.kkt_factor(h, np.ascontiguousarray(p.a_vals), p.b_vals, p.c_vals)
    x = np.empty(p.nK)
    B.kkt_solve(h, np.ascontiguousarray(p.rhs), x)
    return x


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_batch_equals_alone(prec):
    _torch()
    from paper_1907_05420_gb300 import binding as B

    probs = _mix(6)
    hs = [B.kkt_analyze(p, B.kkt_default_options(prec)) for p in probs]
    try:
        alone = [_alone(B, h, p) for h, p in zip(hs, probs)]
        xs = [np.empty(p.nK) for p in probs]
        st = B.kkt_batch_factor_solve(hs, [np.ascontiguousarray(p.a_vals) for p in probs],
                                      [p.b_vals for p in probs], [p.c_vals for p in probs],
                                      [np.ascontiguousarray(p.rhs) for p in probs], xs, streams=4)
    finally:
        for h in hs:
            B.kkt_destroy(h)
    assert st == [0] * len(probs)
    for p, xa, xb in zip(probs, alone, xs):
        assert np.array_equal(xa, xb)
        assert oracle.backward_error(p, xb) <= 1e-10


def test_server_request_equals_alone_in_a_mix():
    _torch()
    from paper_1907_05420_gb300 import binding as B

    base = _mix(3, seed0=900)
    # each pattern is requested three times: the instance and two re-solves with
    # fresh barrier diagonals and right-hand sides
    reqs = []
    for i, p in enumerate(base):
        reqs += [(i, p), (i, reseed_barrier(p, 77 + i)), (i, reseed_barrier(p, 177 + i))]
    hs = [B.kkt_analyze(p) for p in base]
    srv = B.KKTServer(slots=3)
    try:
        outs = []
        ids = []
        for i, p in reqs:
            x = np.empty(p.nK)
            outs.append(x)
            ids.append(srv.submit(hs[i], np.ascontiguousarray(p.a_vals), p.b_vals, p.c_vals,
                                  np.ascontiguousarray(p.rhs), x))
        lats = []
        for rid in ids:
            st, lat = srv.wait(rid)
            assert st == 0
            lats.append(lat)
        srv.close()
        alone = [_alone(B, hs[i], p) for i, p in reqs]
    finally:
        srv.close()
        for h in hs:
            B.kkt_destroy(h)
    assert all(lat > 0 for lat in lats)
    for (i, p), xs, xa in zip(reqs, outs, alone):
        assert np.array_equal(xs, xa)
        assert oracle.backward_error(p, xs) <= 1e-10


def test_server_budget_below_one_handle_still_progresses():
    _torch()
    from paper_1907_05420_gb300 import binding as B

    probs = _mix(2, seed0=1300)
    hs = [B.kkt_analyze(p) for p in probs]
    srv = B.KKTServer(slots=2, device_budget_bytes=1)
    try:
        xs = [np.empty(p.nK) for p in probs]
        ids = [srv.submit(h, np.ascontiguousarray(p.a_vals), p.b_vals, p.c_vals,
                          np.ascontiguousarray(p.rhs), x) for h, p, x in zip(hs, probs, xs)]
        for rid in ids:
            assert srv.wait(rid)[0] == 0
    finally:
        srv.close()
        for h in hs:
            B.kkt_destroy(h)
    for p, x in zip(probs, xs):
        assert oracle.backward_error(p, x) <= 1e-10


@pytest.mark.parametrize("reserve", ["none", "all"])
def test_server_pattern_cache_equals_alone(reserve):
    """Requests that name patterns: the server analyses each key at its first
    request and re-solves later requests on the resident handle.  With no
    reserve nothing is evicted; with a reserve larger than the device every new
    analysis first evicts the idle handles, so repeated keys are analysed
    again.  Either way each result is bitwise the standalone solve."""
    _torch()
    from paper_1907_05420_gb300 import binding as B

    base = _mix(4, seed0=1700)
    reqs = []
    for rep in range(2):
        for i, p in enumerate(base):
            reqs.append((i, p if rep == 0 else reseed_barrier(p, 300 + i)))
    srv = B.KKTServer(slots=3)
    srv.set_cache(B.kkt_default_options("tf32"), 0 if reserve == "none" else 1 << 62)
    pats = [B.make_pattern(p) for p in base]
    try:
        outs, ids = [], []
        for i, p in reqs:
            x = np.empty(p.nK)
            outs.append(x)
            ids.append(srv.submit_pattern(i, p, np.ascontiguousarray(p.a_vals), p.b_vals, p.c_vals,
                                          np.ascontiguousarray(p.rhs), x, pattern=pats[i]))
        for rid in ids:
            assert srv.wait(rid)[0] == 0
        info = srv.cache_info()
    finally:
        srv.close()
    if reserve == "none":
        assert info["analyses"] == len(base) and info["evictions"] == 0 and info["resident"] == len(base)
    else:
        assert info["evictions"] > 0 and info["analyses"] >= len(base)
    alone = []
    for i, p in reqs:
        h = B.kkt_analyze(base[i], B.kkt_default_options("tf32"))
        try:
            alone.append(_alone(B, h, p))
        finally:
            B.kkt_destroy(h)
    for (i, p), xs, xa in zip(reqs, outs, alone):
        assert np.array_equal(xs, xa)
        assert oracle.backward_error(p, xs) <= 1e-10
