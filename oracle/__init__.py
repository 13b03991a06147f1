"""CPU oracle for the block-arrowhead KKT Schur-complement solve.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark use it.  The library's product path never imports it.

Every routine is a plain FP64 CPU implementation (oracle.c) of the quantity
the paper defines:

* ``min_degree``          -- fill-reducing ordering of A_i's pattern
                             (minimum degree on the explicit elimination graph);
* ``ldlt_dense``          -- A = P L D L^T P^T, 1x1 pivots (block factorization, Algorithm 1);
* ``sparse_solve``        -- A^{-1} b from that factor;
* ``sparse_solve_multi``  -- A^{-1} B for several columns, one factorization;
* ``dense_ldlt``          -- S = L_s D_s L_s^T, no pivoting (dense factor of S, Algorithm 1);
* ``kkt_solve``           -- eqs. SCform, SCsolve, SCsolve1 in sequence,
                             S by one full solve per nonzero column of B_i
                             ("backsolve", Sec. 4.2);
* ``kkt_matvec`` / ``kkt_norm_inf`` / ``backward_error`` -- K x, ||K||_inf and
  the normwise backward error eta = ||r - Kx||_inf / (||K||_inf ||x||_inf + ||r||_inf).

Parity pins: see tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class OracleError(RuntimeError):
    pass


_ERR = {-1: "invalid input", -2: "out of memory", -3: "zero pivot"}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_min_degree.argtypes = [C.c_int32, _i32p, _i32p, _i32p]
        L.orc_min_degree.restype = C.c_int
        L.orc_min_degree_ex.argtypes = [C.c_int32, _i32p, _i32p, C.c_int32, _i32p]
        L.orc_min_degree_ex.restype = C.c_int
        L.orc_nnz_l.argtypes = [C.c_int32, _i32p, _i32p, _i32p]
        L.orc_nnz_l.restype = C.c_int64
        L.orc_ldlt_dense.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, _f64p, _f64p]
        L.orc_ldlt_dense.restype = C.c_int
        L.orc_sparse_solve.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, _f64p, _f64p]
        L.orc_sparse_solve.restype = C.c_int
        L.orc_sparse_solve_multi.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _i32p, C.c_int32, _f64p, _f64p]
        L.orc_sparse_solve_multi.restype = C.c_int
        L.orc_dense_ldlt.argtypes = [C.c_int64, _f64p, _i64p]
        L.orc_dense_ldlt.restype = C.c_int
        L.orc_dense_ldlt_solve.argtypes = [C.c_int64, _f64p, _f64p]
        L.orc_dense_ldlt_solve.restype = C.c_int
        common = [C.c_int32, C.c_int32, C.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p,
                  _f64p, C.c_int32, _f64p]
        L.orc_kkt_matvec.argtypes = common + [_f64p, _f64p]
        L.orc_kkt_matvec.restype = C.c_int
        L.orc_kkt_norm_inf.argtypes = common
        L.orc_kkt_norm_inf.restype = C.c_double
        L.orc_kkt_solve.argtypes = common + [_f64p, _i32p, _f64p, C.c_void_p, C.c_void_p, _i64p,
                                             C.c_int32]
        L.orc_kkt_solve.restype = C.c_int
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise OracleError(_ERR.get(rc, f"error {rc}"))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def min_degree(n, rowptr, col, n_primal=None) -> np.ndarray:
    """Minimum-degree elimination order (perm[k] = node eliminated k-th).

    With n_primal given, a node >= n_primal (a multiplier row of A_i) becomes
    eligible only once all its original neighbours < n_primal (the primal
    variables it constrains) are eliminated.  In exact arithmetic any order
    factors a quasidefinite A_i with 1x1 pivots; in FP64 this order keeps the
    -1e-8 multiplier diagonal from being used as a pivot before its primal
    neighbours have been folded in, which avoids growth of order 1/1e-8.
    """
    perm = np.empty(n, dtype=np.int32)
    npr = n if n_primal is None else int(n_primal)
    _check(lib().orc_min_degree_ex(n, _i32(rowptr), _i32(col), npr, perm))
    return perm


def nnz_l(n, rowptr, col, perm) -> int:
    r = int(lib().orc_nnz_l(n, _i32(rowptr), _i32(col), _i32(perm)))
    if r < 0:
        _check(r)
    return r


def ldlt_dense(n, rowptr, col, vals, perm):
    """Dense copies of L (unit lower, permuted order) and D."""
    L = np.empty((n, n))
    D = np.empty(n)
    _check(lib().orc_ldlt_dense(n, _i32(rowptr), _i32(col), _f64(vals), _i32(perm), L, D))
    return L, D


def sparse_solve(n, rowptr, col, vals, perm, b):
    x = np.empty(n)
    _check(lib().orc_sparse_solve(n, _i32(rowptr), _i32(col), _f64(vals), _i32(perm), _f64(b), x))
    return x


def sparse_solve_multi(n, rowptr, col, vals, perm, B):
    """X = A^{-1} B for the columns of the n x m array B (one factorization)."""
    Bc = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(n, -1))
    m = Bc.shape[1]
    flat = np.ascontiguousarray(Bc.T).reshape(-1)
    X = np.empty(n * m)
    _check(lib().orc_sparse_solve_multi(n, _i32(rowptr), _i32(col), _f64(vals), _i32(perm), m, flat, X))
    return X.reshape(m, n).T.copy()


def dense_ldlt(S):
    """In-place-style dense LDL^T: returns (F, inertia) with L in the strict
    lower triangle of F and D on its diagonal."""
    F = np.array(S, dtype=np.float64, order="C", copy=True)
    inertia = np.zeros(3, dtype=np.int64)
    _check(lib().orc_dense_ldlt(F.shape[0], F, inertia))
    return F, inertia


def dense_ldlt_solve(F, b):
    x = _f64(b).copy()
    _check(lib().orc_dense_ldlt_solve(F.shape[0], _f64(F), x))
    return x


def _common(p):
    c_vals = _f64(p.c_vals).reshape(-1)
    return (p.N, p.nA, p.nC, _i32(p.a_rowptr), _i32(p.a_col), _f64(p.a_vals).reshape(-1),
            _i32(p.b_blockptr), _i32(p.b_row), _i32(p.b_col), _f64(p.b_vals), int(p.c_kind),
            c_vals)


def kkt_matvec(p, x):
    y = np.empty(p.nK)
    _check(lib().orc_kkt_matvec(*_common(p), _f64(x), y))
    return y


def kkt_norm_inf(p) -> float:
    return float(lib().orc_kkt_norm_inf(*_common(p)))


def backward_error(p, x, rhs=None) -> float:
    """eta = ||r - Kx||_inf / (||K||_inf ||x||_inf + ||r||_inf)."""
    r = p.rhs if rhs is None else rhs
    res = r - kkt_matvec(p, x)
    return float(np.max(np.abs(res)) /
                 (kkt_norm_inf(p) * np.max(np.abs(x)) + np.max(np.abs(r))))


def kkt_solve(p, perm=None, *, want_S=False, nthreads=0, rhs=None):
    """Solve K x = rhs by the Schur-complement method.

    Returns dict(x, inertia, perm, S (if want_S), t (if want_S)).
    """
    if perm is None:
        perm = min_degree(p.nA, p.a_rowptr, p.a_col, p.nP)
    r = _f64(p.rhs if rhs is None else rhs)
    x = np.empty(p.nK)
    inertia = np.zeros(3, dtype=np.int64)
    S = np.empty((p.nC, p.nC)) if want_S else None
    t = np.empty(p.nC) if want_S else None
    _check(lib().orc_kkt_solve(
        *_common(p), r, _i32(perm), x,
        S.ctypes.data if want_S else None, t.ctypes.data if want_S else None,
        inertia, int(nthreads)))
    out = {"x": x, "inertia": inertia, "perm": perm}
    if want_S:
        out["S"] = S
        out["t"] = t
    return out


def lib_path() -> str:
    return os.path.abspath(_build.LIB)
