"""Host logic of the analysis phase (Sec. 4.1, 4.2): ordering, supernodes,
update maps, coupling reach and the envelope of S, checked on the CPU.

The analysis that kkt_analyze runs before it uploads anything is exposed by
the host-only inspection library (include/kkt_symbolic.h).  Its outputs are
pinned here against brute force (graph elimination on small blocks) and
against the oracle's independent symbolic and numeric factorizations.
"""
import ctypes as C
import functools

import numpy as np
import pytest

import oracle
from gen import CONFIGS, GridSpec, make_problem, make_scopf


@functools.lru_cache(maxsize=None)
def _lib():
    from paper_1907_05420_gb300 import build as lib_build

    L = C.CDLL(lib_build.build_symbolic())
    i32p, f64p = C.POINTER(C.c_int32), C.POINTER(C.c_double)
    L.kkt_symbolic_create.argtypes = [C.c_int32, C.c_int32, i32p, i32p, f64p, C.c_int32, C.c_int32,
                                      i32p, i32p, i32p, C.c_int32]
    L.kkt_symbolic_create.restype = C.c_void_p
    L.kkt_symbolic_get.argtypes = [C.c_void_p, C.c_char_p, C.POINTER(C.c_int64)]
    L.kkt_symbolic_get.restype = C.c_int64
    L.kkt_symbolic_destroy.argtypes = [C.c_void_p]
    L.kkt_symbolic_destroy.restype = None
    L.kkt_symbolic_error.argtypes = []
    L.kkt_symbolic_error.restype = C.c_char_p
    L.kkt_symbolic_choose_tail.argtypes = [C.c_void_p, C.c_double, C.c_int64]
    L.kkt_symbolic_choose_tail.restype = C.c_int32
    return L


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def analyze(p, hint=True, tails=None):
    """All arrays of the analysis of problem p, as a dict of int64 arrays.
    tails: optional list of (ratio, max_bytes); the tail is re-chosen with each
    and the resulting tail sizes are returned under "tails"."""
    L = _lib()
    rp = np.ascontiguousarray(p.a_rowptr, dtype=np.int32)
    col = np.ascontiguousarray(p.a_col, dtype=np.int32)
    bbp = np.ascontiguousarray(p.b_blockptr, dtype=np.int32)
    brow = np.ascontiguousarray(p.b_row, dtype=np.int32)
    bcol = np.ascontiguousarray(p.b_col, dtype=np.int32)
    hv = np.ascontiguousarray(np.asarray(p.a_vals).reshape(p.N, -1)[0], dtype=np.float64)
    h = L.kkt_symbolic_create(p.nA, p.nP, _ptr(rp, C.c_int32), _ptr(col, C.c_int32),
                              _ptr(hv, C.c_double) if hint else None, p.N, p.nC,
                              _ptr(bbp, C.c_int32), _ptr(brow, C.c_int32), _ptr(bcol, C.c_int32),
                              int(p.c_kind))
    assert h, L.kkt_symbolic_error().decode()
    out = {}
    try:
        if tails:
            out["tails"] = [int(L.kkt_symbolic_choose_tail(h, float(r), int(b))) for r, b in tails]
        for name in ("perm partner sn_first sn_rowptr sn_rows sn_valoff sn_parent sn_level a_map "
                     "upd_ptr upd_src upd_r0 upd_r1 upd_reloff upd_rel E e_t wpos sn_wrow s_key "
                     "panel_rend jlo jhi colcount upd_ntail tail_wrow wt_ptr wt_idx stats").split():
            n = L.kkt_symbolic_get(h, name.encode(), None)
            assert n >= 0, name
            a = np.zeros(n, dtype=np.int64)
            L.kkt_symbolic_get(h, name.encode(), _ptr(a, C.c_int64))
            out[name] = a
    finally:
        L.kkt_symbolic_destroy(h)
    st = out.pop("stats")
    out.update(n=int(st[0]), nsuper=int(st[1]), nlevels=int(st[2]), panel_total=int(st[3]),
               nnzL=int(st[4]), k=int(st[5]), nw=int(st[6]), tail_sn=int(st[7]), tail_col=int(st[8]),
               nw_before_tail=int(st[9]))
    return out


def _storage_spec(seed=5):
    # a few storage units, so M_i couples neighbouring periods through B
    return GridSpec(20, 26, 4, 3, 6, 1e-6, 1e6, seed, "st20")


def _aug_spec(seed=102, nb=14):
    # a block whose dense tail lies in the reach of the coupling rows
    return GridSpec(nb, nb + 4, 3, 2, 4, 1e-6, 1e6, seed, f"aug{seed}")


PROBLEMS = {
    "aug14": lambda: make_problem(_aug_spec()),
    "tiny": lambda: make_problem(CONFIGS["tiny"]),
    "small": lambda: make_problem(CONFIGS["small"]),
    "grid30_n24": lambda: make_problem(CONFIGS["grid30_n24"]),
    "storage20": lambda: make_problem(_storage_spec()),
    # the paper's cumulative coupling: every period's storage rows reach the
    # energy constraints of all later periods, so S is dense
    "paper20": lambda: make_problem(_storage_spec(), coupling="paper"),
    # security-constrained: scenario blocks, PV-bus coupling, dense C
    "scopf14": lambda: make_scopf(GridSpec(14, 20, 5, 0, 1, 1e-4, 1e4, 5, "scopf14"), 4),
}


@functools.lru_cache(maxsize=None)
def _case(name):
    p = PROBLEMS[name]()
    return p, analyze(p)


def _sym_adj(n, rowptr, col):
    adj = [set() for _ in range(n)]
    for r in range(n):
        for q in range(rowptr[r], rowptr[r + 1]):
            c = int(col[q])
            if c != r:
                adj[r].add(c)
                adj[c].add(r)
    return adj


def _fill_pattern(p, perm):
    """Strictly-lower pattern of L, per column of the permuted matrix, by
    eliminating vertices of the graph of A one at a time (brute force)."""
    n = p.nA
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    adj = _sym_adj(n, p.a_rowptr, p.a_col)
    g = [set(int(iperm[v]) for v in adj[perm[k]]) for k in range(n)]
    pat = []
    for k in range(n):
        later = {j for j in g[k] if j > k}
        pat.append(later)
        for a in later:
            g[a] |= later - {a}
    return pat


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_perm_is_permutation_with_partners_first(name):
    p, s = _case(name)
    perm = s["perm"]
    assert sorted(perm.tolist()) == list(range(p.nA))
    iperm = np.empty(p.nA, dtype=np.int64)
    iperm[perm] = np.arange(p.nA)
    partner = s["partner"]
    assert len(partner) == p.nA and np.all(partner[:p.nP] == -1)
    adj = _sym_adj(p.nA, p.a_rowptr, p.a_col)
    paired = 0
    for r in range(p.nP, p.nA):
        q = int(partner[r])
        if q < 0:
            continue
        paired += 1
        assert q < p.nP and q in adj[r]           # a primal neighbour of the multiplier
        assert iperm[q] < iperm[r]                 # the partner is eliminated first
    assert paired > 0


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_nnz_l_matches_oracle_symbolic(name):
    p, s = _case(name)
    perm = s["perm"].astype(np.int32)
    assert s["nnzL"] == oracle.nnz_l(p.nA, p.a_rowptr, p.a_col, perm)


@pytest.mark.parametrize("name", ["tiny", "small", "grid30_n24", "storage20"])
def test_supernode_rows_are_union_of_column_patterns(name):
    p, s = _case(name)
    pat = _fill_pattern(p, s["perm"])
    assert s["nnzL"] == sum(len(x) for x in pat)
    first, rp, rows = s["sn_first"], s["sn_rowptr"], s["sn_rows"]
    assert first[0] == 0 and first[-1] == p.nA and np.all(np.diff(first) >= 1)
    assert np.all(np.diff(first) <= 32)
    for q in range(s["nsuper"]):
        cols = set(range(first[q], first[q + 1]))
        want = set(cols)
        for j in cols:
            want |= pat[j]
        got = rows[rp[q]:rp[q + 1]].tolist()
        assert got == sorted(want)
        assert got[:len(cols)] == sorted(cols)


@pytest.mark.parametrize("name", ["tiny", "small", "grid30_n24", "storage20"])
def test_column_counts_match_brute_force(name):
    p, s = _case(name)
    pat = _fill_pattern(p, s["perm"])
    assert s["colcount"].tolist() == [len(x) for x in pat]


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_dense_tail_is_the_longest_cheap_suffix(name):
    """The dense tail: a suffix of the supernodes closed under the parent, whose
    dense flops nT^3/3 are at most 1.5 times the exact sparse flops of its
    columns; the longest such suffix that fits the memory cap is taken."""
    p, s = _case(name)
    first, rp, rows, par = s["sn_first"], s["sn_rowptr"], s["sn_rows"], s["sn_parent"]
    ns, n, t0, tc = s["nsuper"], p.nA, s["tail_sn"], s["tail_col"]
    assert tc == (first[t0] if t0 < ns else n)
    cc = s["colcount"].astype(float)
    fl = cc * (cc + 3)

    def ok(t):
        nT = n - first[t]
        return nT >= 16 and p.N * nT * nT * 8 <= 24 << 30 and nT ** 3 / 3.0 <= 1.5 * fl[first[t]:].sum()

    cands = [t for t in range(ns) if ok(t)]
    assert t0 == (min(cands) if cands else ns)
    for q in range(t0, ns):
        assert rows[rp[q]:rp[q + 1]].min() >= tc        # every row is a tail column
        assert par[q] == -1 or par[q] >= t0               # closed under the parent
    # update lists: the updates from outside the tail come first
    up, src, nt = s["upd_ptr"], s["upd_src"], s["upd_ntail"]
    for q in range(ns):
        lst = src[up[q]:up[q + 1]]
        assert np.all(lst[:nt[q]] < t0) and np.all(lst[nt[q]:] >= t0)


def _rule_tail(p, s, ratio, cap):
    """The tail rule evaluated directly: the longest suffix with
    nT^3/3 <= ratio * sparse flops, nT >= 16 and N nT^2 8 bytes <= cap."""
    first, ns, n = s["sn_first"], s["nsuper"], p.nA
    cc = s["colcount"].astype(float)
    fl = cc * (cc + 3)
    ok = [t for t in range(ns) if n - first[t] >= 16 and p.N * (n - first[t]) ** 2 * 8 <= cap
          and (n - first[t]) ** 3 / 3.0 <= ratio * fl[first[t]:].sum()]
    return n - first[min(ok)] if ok else 0


@pytest.mark.parametrize("name", ["aug14", "grid30_n24", "storage20"])
def test_tail_ratio_and_cap(name):
    """kkt_symbolic_choose_tail (the tail_ratio option and the per-mode byte
    caps) follows the rule for every ratio and cap, and a larger ratio or cap
    never shortens the tail."""
    p, _ = _case(name)
    caps = [24 << 30, 96 << 30, p.N * 20 * 20 * 8]
    grid = [(r, c) for c in caps for r in (1.0, 1.25, 1.5, 2.0, 3.0)]
    s = analyze(p, tails=grid)
    for (r, c), nT in zip(grid, s["tails"]):
        assert nT == _rule_tail(p, s, r, c), (r, c)
    t = dict(zip(grid, s["tails"]))
    for c in caps:
        assert all(t[(a, c)] <= t[(b, c)] for a, b in zip((1.0, 1.25, 1.5, 2.0), (1.25, 1.5, 2.0, 3.0)))
    assert all(t[(r, caps[2])] <= t[(r, caps[0])] <= t[(r, caps[1])] for r in (1.0, 1.5, 3.0))


def test_tail_sizes_of_the_9241_bus_grid():
    """On the 9,241-bus grid over 168 periods the 24 GiB cap of the FP64 tail
    binds (4,369 columns), while the 96 GiB cap of the tensor-core tail lets the
    rule take 7,009 (r = 1.25) or 7,447 (r = 1.5) columns."""
    p = make_problem(CONFIGS["grid9241_n168"])
    s = analyze(p, tails=[(1.5, 24 << 30), (1.25, 96 << 30), (1.5, 96 << 30)])
    assert s["tails"] == [4369, 7009, 7447]


def test_dense_tail_present_on_meshed_grids():
    import dataclasses

    p = make_problem(dataclasses.replace(CONFIGS["grid2383_n96"], n_per=2))
    s = analyze(p)
    nT = p.nA - s["tail_col"]
    cc = s["colcount"].astype(float)
    fl = cc * (cc + 3)
    assert 400 <= nT <= 2000
    assert fl[s["tail_col"]:].sum() >= 0.8 * fl.sum()   # the tail holds most of the work


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_supernodal_tree_levels_and_panels(name):
    p, s = _case(name)
    first, rp, rows, par, lvl = s["sn_first"], s["sn_rowptr"], s["sn_rows"], s["sn_parent"], s["sn_level"]
    col_sn = np.repeat(np.arange(s["nsuper"]), np.diff(first))
    off = s["sn_valoff"]
    for q in range(s["nsuper"]):
        w = first[q + 1] - first[q]
        m = rp[q + 1] - rp[q]
        assert off[q + 1] - off[q] == m * w
        # parent = supernode of the first row below the diagonal block
        if m > w:
            assert par[q] == col_sn[rows[rp[q] + w]]
            assert lvl[par[q]] > lvl[q]
        else:
            assert par[q] == -1
    assert off[-1] == s["panel_total"]
    leaves = set(range(s["nsuper"])) - set(par[par >= 0].tolist())
    assert all(lvl[q] == 0 for q in leaves)
    assert s["nlevels"] == lvl.max() + 1


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_a_map_places_each_entry_in_its_panel(name):
    p, s = _case(name)
    n = p.nA
    iperm = np.empty(n, dtype=np.int64)
    iperm[s["perm"]] = np.arange(n)
    first, rp, rows, off = s["sn_first"], s["sn_rowptr"], s["sn_rows"], s["sn_valoff"]
    col_sn = np.repeat(np.arange(s["nsuper"]), np.diff(first))
    amap = s["a_map"]
    assert len(amap) == p.nnzA
    for r in range(n):
        for q in range(p.a_rowptr[r], p.a_rowptr[r + 1]):
            a, b = iperm[r], iperm[p.a_col[q]]
            row, c = max(a, b), min(a, b)
            sn = col_sn[c]
            pos = int(np.searchsorted(rows[rp[sn]:rp[sn + 1]], row))
            assert rows[rp[sn] + pos] == row
            m = rp[sn + 1] - rp[sn]
            assert amap[q] == off[sn] + (c - first[sn]) * m + pos
    assert len(np.unique(amap)) == len(amap)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_update_lists_are_exact(name):
    p, s = _case(name)
    first, rp, rows = s["sn_first"], s["sn_rowptr"], s["sn_rows"]
    up, src, r0, r1, roff, rel = (s[k] for k in ("upd_ptr", "upd_src", "upd_r0", "upd_r1",
                                                  "upd_reloff", "upd_rel"))
    for q in range(s["nsuper"]):
        lo, hi = first[q], first[q + 1]
        srows = rows[rp[q]:rp[q + 1]]
        want = {}
        for d in range(q):
            drows = rows[rp[d]:rp[d + 1]]
            w = first[d + 1] - first[d]
            inside = [i for i in range(w, len(drows)) if lo <= drows[i] < hi]
            if inside:
                want[d] = (inside[0], inside[-1] + 1)
        got = {}
        for u in range(up[q], up[q + 1]):
            d = int(src[u])
            got[d] = (int(r0[u]), int(r1[u]))
            drows = rows[rp[d]:rp[d + 1]]
            for i in range(r0[u], len(drows)):
                assert srows[rel[roff[u] + i - r0[u]]] == drows[i]
        assert got == want


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_coupling_rows_and_reach(name):
    p, s = _case(name)
    E = s["E"]
    assert E.tolist() == sorted(set(np.asarray(p.b_row).tolist()))
    assert s["k"] == len(E)
    assert np.array_equal(E[s["e_t"]], np.asarray(p.b_row))
    iperm = np.empty(p.nA, dtype=np.int64)
    iperm[s["perm"]] = np.arange(p.nA)
    first, par = s["sn_first"], s["sn_parent"]
    col_sn = np.repeat(np.arange(s["nsuper"]), np.diff(first))
    reach = set()
    for r in E.tolist():
        q = int(col_sn[iperm[r]])
        while q >= 0 and q not in reach:
            reach.add(q)
            q = int(par[q])
    assert set(np.nonzero(s["sn_wrow"] >= 0)[0].tolist()) == reach
    assert s["nw"] == sum(first[q + 1] - first[q] for q in reach)
    # each unit right-hand side sits on E's own row inside W
    for t, r in enumerate(E.tolist()):
        q = int(col_sn[iperm[r]])
        assert s["wpos"][t] == s["sn_wrow"][q] + iperm[r] - first[q]


@pytest.mark.parametrize("name", ["tiny", "small", "grid30_n24", "storage20"])
def test_s_keys_cover_oracle_schur_complement(name):
    p, s = _case(name)
    S = oracle.kkt_solve(p, want_S=True)["S"]
    nC = p.nC
    keys = set(s["s_key"].tolist())
    assert np.all(np.diff(s["s_key"]) > 0)
    for key in keys:
        c1, c2 = divmod(key, nC)
        assert c1 >= c2
    nz = np.argwhere(np.tril(S, -1) != 0)
    for c1, c2 in nz:
        assert c1 * nC + c2 in keys
    # every structural pair is a real term: with generic values none cancels
    diag_off = {c * nC + c for c in range(nC)}
    assert len(keys - diag_off) == len(nz)


@pytest.mark.parametrize("name", ["tiny", "small", "grid30_n24", "storage20"])
def test_envelope_bounds_the_factor_of_s(name):
    p, s = _case(name)
    S = oracle.kkt_solve(p, want_S=True)["S"]
    nC, NB = p.nC, 64
    F, _ = oracle.dense_ldlt(S)
    Lnz = np.tril(F, -1) != 0
    nbk = (nC + NB - 1) // NB
    rend, jlo, jhi = s["panel_rend"], s["jlo"], s["jhi"]
    assert len(rend) == len(jlo) == len(jhi) == nbk
    for pb in range(nbk):
        c0, c1 = pb * NB, min(nC, pb * NB + NB)
        rr = np.nonzero(Lnz[:, c0:c1].any(axis=1))[0]
        assert rr.size == 0 or rr.max() < rend[pb]
        assert rend[pb] >= c1 and jhi[pb] == -(-rend[pb] // NB)
        rows_nz = np.nonzero(Lnz[c0:c1].any(axis=0))[0]
        assert rows_nz.size == 0 or rows_nz.min() // NB >= jlo[pb]
        assert jlo[pb] <= pb < jhi[pb]


def test_envelope_of_dense_c_is_full():
    p = make_problem(CONFIGS["tiny"])
    p.c_kind = 1
    p.c_vals = np.diag(np.asarray(p.c_vals, dtype=np.float64))
    s = analyze(p)
    nbk = (p.nC + 63) // 64
    assert s["jlo"].tolist() == [0] * nbk
    assert s["panel_rend"].tolist() == [p.nC] * nbk


def test_no_hint_still_orders_every_row():
    p = make_problem(CONFIGS["small"])
    s = analyze(p, hint=False)
    assert sorted(s["perm"].tolist()) == list(range(p.nA))
    assert s["nnzL"] == oracle.nnz_l(p.nA, p.a_rowptr, p.a_col, s["perm"].astype(np.int32))


def test_malformed_pattern_is_rejected():
    p = make_problem(CONFIGS["tiny"])
    bad = np.array(p.a_col, dtype=np.int32).copy()
    bad[0] = p.nA + 5
    p.a_col = bad
    L = _lib()
    rp = np.ascontiguousarray(p.a_rowptr, dtype=np.int32)
    bbp = np.ascontiguousarray(p.b_blockptr, dtype=np.int32)
    brow = np.ascontiguousarray(p.b_row, dtype=np.int32)
    bcol = np.ascontiguousarray(p.b_col, dtype=np.int32)
    h = L.kkt_symbolic_create(p.nA, p.nP, _ptr(rp, C.c_int32), _ptr(bad, C.c_int32), None, p.N, p.nC,
                              _ptr(bbp, C.c_int32), _ptr(brow, C.c_int32), _ptr(bcol, C.c_int32), 0)
    assert not h
    assert L.kkt_symbolic_error()


def test_full_size_block_pattern():
    # the 2383-bus block at two periods: the block pattern is that of the full workload
    import dataclasses

    p = make_problem(dataclasses.replace(CONFIGS["grid2383_n96"], n_per=2))
    s = analyze(p)
    assert s["nnzL"] == oracle.nnz_l(p.nA, p.a_rowptr, p.a_col, s["perm"].astype(np.int32))
    first, par, lvl = s["sn_first"], s["sn_parent"], s["sn_level"]
    assert np.all(np.diff(first) <= 32)
    kids = par >= 0
    assert np.all(lvl[par[kids]] > lvl[kids])
    assert np.all(par[kids] > np.nonzero(kids)[0])
    assert len(np.unique(s["a_map"])) == p.nnzA
    assert s["E"].tolist() == sorted(set(np.asarray(p.b_row).tolist()))


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_tail_w_rows(name):
    """The augmented tail needs the tail's W rows after all others: W rows are
    numbered in supernode order over the reach of E, so the rows outside the
    tail are the first nw_before_tail, and every tail column in the reach maps
    to its own W row."""
    p, s = _case(name)
    t0, tc, n = s["tail_sn"], s["tail_col"], p.nA
    first, wrow = s["sn_first"], s["sn_wrow"]
    nT = n - tc
    assert s["nw_before_tail"] == sum(first[q + 1] - first[q] for q in range(t0) if wrow[q] >= 0)
    tw = s["tail_wrow"]
    assert len(tw) == nT
    for q in range(t0, s["nsuper"]):
        for j in range(first[q], first[q + 1]):
            assert tw[j - tc] == (wrow[q] + j - first[q] if wrow[q] >= 0 else -1)
    rows = tw[tw >= 0]
    assert np.all(rows >= s["nw_before_tail"]) and len(set(rows.tolist())) == len(rows)
    assert len(rows) == s["nw"] - s["nw_before_tail"]


@pytest.mark.parametrize("name", ["aug14", "tiny", "small", "grid30_n24", "storage20"])
def test_w_column_sets_match_the_structure_of_l_inverse(name):
    """Column t of W = L^{-1} P^T e_{E_t} is structurally nonzero exactly on the
    rows reachable from E_t's pivot in the graph of L; a supernode carries
    column t when one of its columns is reachable.  Checked with the fill
    pattern from brute-force elimination."""
    p, s = _case(name)
    pat = _fill_pattern(p, s["perm"])
    iperm = np.empty(p.nA, dtype=np.int64)
    iperm[s["perm"]] = np.arange(p.nA)
    first = s["sn_first"]
    col_sn = np.repeat(np.arange(s["nsuper"]), np.diff(first))
    want = [set() for _ in range(s["nsuper"])]
    for t, r in enumerate(s["E"].tolist()):
        seen, stack = set(), [int(iperm[r])]
        while stack:
            j = stack.pop()
            if j in seen:
                continue
            seen.add(j)
            stack.extend(pat[j])
        for j in seen:
            want[col_sn[j]].add(t)
    ptr, idx = s["wt_ptr"], s["wt_idx"]
    for q in range(s["nsuper"]):
        got = idx[ptr[q]:ptr[q + 1]].tolist()
        assert got == sorted(want[q])
        assert (len(got) > 0) == (s["sn_wrow"][q] >= 0)
