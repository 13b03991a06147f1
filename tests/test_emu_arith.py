"""The exact arithmetic of the emulated-FP64 tensor-core update, on the CPU.

The update (Sec. 4.2's dense factor, run as 28 digit products per tile on the
BF16 tensor cores) depends on helper arithmetic that must be exact or
correctly rounded: the base-256 digits of each FP64 operand, the read-out of
the FP32 digit-product levels without conversion instructions, and the FP64
bit pattern of -W 2^e.  The helpers compile for the host as well
(csrc/emu_arith.cuh); here they are built with g++ and compared, on random and
edge-case inputs, with exact rational arithmetic (fractions.Fraction, whose
conversion to float rounds correctly) and numpy.
"""
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    d = tmp_path_factory.mktemp("emu")
    exe = str(d / "emu_arith_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_1907_05420_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "emu_arith_check.cpp"), "-o", exe], check=True)

    def run(mode, data, out_dtype):
        src, dst = str(d / f"{mode}.in"), str(d / f"{mode}.out")
        if data is not None:
            np.ascontiguousarray(data).tofile(src)
        subprocess.run([exe, mode, src if data is not None else "-", dst], check=True)
        return np.fromfile(dst, dtype=out_dtype)

    return run


def test_exact_f2i(prog):
    """Integer-valued FP32 numbers below 2^30 (the digit-product levels are
    below 2^24) come back exactly."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.integers(-2**24, 2**24 + 1, 200_000),
                        rng.integers(-2**30 + 1, 2**30, 20_000) // 64 * 64,
                        np.arange(-600, 601), [2**24, -2**24, 2**23 + 1, -(2**23 + 1), 128, -128, 384]])
    xf = x.astype(np.float32)
    assert np.all(xf.astype(np.float64) == x)  # the inputs are exact FP32 integers
    got = prog("f2i", xf, np.int32)
    assert np.array_equal(got.astype(np.int64), x.astype(np.int64))


def test_round_f2ll(prog):
    """Round to nearest, ties to even, of FP32 numbers below 2^37 (the folded
    low levels reach about 2^33), ties included."""
    rng = np.random.default_rng(2)
    parts = [rng.standard_normal(100_000) * s for s in (1.0, 1e3, 1e6, 1e9, 2.0**36)]
    ties = np.arange(-2000, 2000) + 0.5
    big_ties = (np.arange(-300, 300) * 65536.0 + 32768.0)
    x = np.concatenate(parts + [ties, big_ties]).astype(np.float32)
    x = x[np.abs(x.astype(np.float64)) < 2.0**37]
    got = prog("f2ll", x, np.int64)
    want = np.rint(x.astype(np.float64)).astype(np.int64)
    assert np.array_equal(got, want)


def test_neg_scaled_rounds_once(prog):
    """-W 2^e as FP64 bits: the correctly rounded value of the exact product,
    normal, subnormal, underflowing to zero or overflowing to infinity."""
    rng = np.random.default_rng(3)
    n = 60_000
    bits = rng.integers(0, 63, n)
    W = np.array([int(rng.integers(0, 2**int(b))) if b else 0 for b in bits], dtype=np.int64)
    W[rng.random(n) < 0.5] *= -1
    e = np.where(rng.random(n) < 0.6, rng.integers(-200, 200, n), rng.integers(-1200, 1100, n))
    edge_W = [1, 3, 2**53 + 1, 2**53 + 3, 2**62 + 2**9, 2**62 + 2**9 + 1, 2**63 - 1]
    edge_e = [-1074, -1075, -1076, -1100, -1130, -1136, -1137, -1138, 0, 900, 960, 961, 962, 1000]
    EW = np.array([s * w for w in edge_W for _ in edge_e for s in (1, -1)], dtype=np.int64)
    Ee = np.array([x for _ in edge_W for x in edge_e for _ in (1, -1)], dtype=np.int64)
    W = np.concatenate([W, EW])
    e = np.concatenate([e, Ee])
    got = prog("neg", np.stack([W, e], axis=1).astype(np.int64), np.float64)
    for w, s, g in zip(W.tolist(), e.tolist(), got.tolist()):
        v = Fraction(-w) * Fraction(2) ** s
        try:
            want = float(v)
        except OverflowError:
            want = float("inf") if v > 0 else float("-inf")
        assert g == want, (w, s, g, want)


def test_digits_are_the_truncated_scaled_magnitude(prog):
    """q = trunc(|v| 2^(56 - e)) for |v| < 2^e: normal and subnormal v, the
    bound taken from the exponent of v or from a larger one."""
    rng = np.random.default_rng(4)
    n = 20_000
    v = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, n)
    v = np.concatenate([v, [5e-324, -5e-324, 2.2250738585072014e-308, -1.5e-310, 0.0, -0.0, 1.0, -1.0,
                            0.9999999999999999, 1.7976931348623157e308]])
    ex = np.array([np.frexp(x)[1] if x != 0 else 0 for x in v], dtype=np.int64)  # |v| < 2^ex
    ex = ex + rng.integers(0, 3, len(v))  # a looser bound drops low digits
    data = np.stack([v.view(np.int64), ex], axis=1)
    out = prog("digits", data, np.int64).reshape(-1, 2)
    for x, s, (q, sg) in zip(v.tolist(), ex.tolist(), out.tolist()):
        want = int(abs(Fraction(x)) * Fraction(2) ** (56 - s))
        assert q == want, (x, s, q, want)
        assert sg == (-1 if np.signbit(x) else 1)


def test_pow2_exponent(prog):
    k = np.arange(-1074, 1024)
    s = np.array([float(Fraction(2) ** int(i)) for i in k])
    got = prog("pow2", s, np.int64)
    assert np.array_equal(got, k)


def test_bf16_table(prog):
    """The BF16 patterns of the byte values are those of the exact FP32
    numbers with the low 16 bits dropped."""
    got = prog("bf16", None, np.uint32)
    want = np.arange(256, dtype=np.float32).view(np.uint32) >> 16
    assert np.array_equal(got, want)


@pytest.mark.parametrize("jsplit", [1, 4])
def test_tile_runs_cover_the_lower_triangle_once(prog, jsplit):
    """The tasks of the emulated update (runs of at most 8 tiles of one tile
    row) cover every 128 x 64 tile holding part of the lower triangle exactly
    once; the first jsplit tile columns (jmode 1: the next panel's 64 or 256
    columns) and the rest (jmode 2) split the full set (jmode 0) between them."""
    ms = list(range(1, 3000, 37)) + [64, 127, 128, 129, 192, 255, 256, 1024, 7409]
    trip = []
    for m in ms:
        TI, TJ = -(-m // 128), -(-m // 64)
        for jmode in (0, 1, 2):
            trip.append((TI, TJ, jmode, jsplit))
    out = prog("tasks", np.array(trip, dtype=np.int64), np.int64).tolist()
    pos = 0
    sets = {}
    for TI, TJ, jmode, _ in trip:
        cnt = out[pos]
        pos += 1
        tiles = []
        for _ in range(cnt):
            I, j0, j1 = out[pos:pos + 3]
            pos += 3
            assert 0 <= I < TI and 0 <= j0 < j1 <= TJ and j1 - j0 <= 8
            tiles += [(I, J) for J in range(j0, j1)]
        assert len(tiles) == len(set(tiles))
        sets[(TI, TJ, jmode)] = set(tiles)
    assert pos == len(out)
    for m in ms:
        TI, TJ = -(-m // 128), -(-m // 64)
        want = {(I, J) for I in range(TI) for J in range(TJ) if J <= 2 * I + 1}
        assert sets[(TI, TJ, 0)] == want
        assert sets[(TI, TJ, 1)] == {t for t in want if t[1] < jsplit}
        assert sets[(TI, TJ, 2)] == {t for t in want if t[1] >= jsplit}


def test_balanced_digits(prog):
    """q < 2^55 rebalanced into 7 base-256 digits: the digits add up to q
    exactly, the lower six lie in [-128, 127] and the top one in [0, 128], so
    every product of two digits is at most 2^14 and 4 K = 256-term sums of
    them stay at most 2^24 (exact in FP32)."""
    rng = np.random.default_rng(6)
    q = np.concatenate([rng.integers(0, 2**55, 200_000, dtype=np.int64),
                        np.array([0, 1, 127, 128, 255, 256, 2**55 - 1, 2**55 - 2**48, 0x7F7F7F7F7F7F7F,
                                  0x7F80808080808080 >> 8, 0x80808080808080 >> 1], dtype=np.int64)])
    q = q[q < 2**55]
    d = prog("balanced", q, np.int64).reshape(-1, 7)
    w = np.array([256 ** (6 - s) for s in range(7)], dtype=object)
    assert all(sum(int(x) * int(y) for x, y in zip(row, w)) == int(v) for row, v in zip(d[:5000], q[:5000]))
    # all rows: compare in two exact int64 halves
    lo = d[:, 4:] @ np.array([65536, 256, 1], dtype=np.int64)
    hi = d[:, :4] @ np.array([2**24, 2**16, 2**8, 1], dtype=np.int64)
    assert np.array_equal(hi * 2**24 + lo, q)
    assert d[:, 1:].min() >= -128 and d[:, 1:].max() <= 127
    assert d[:, 0].min() >= 0 and d[:, 0].max() <= 128
