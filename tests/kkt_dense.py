"""Test helpers: dense assembly of small arrowhead systems.

Only used on tiny inputs, as an independent cross-check (numpy LAPACK LU,
eigvalsh) of the oracle.
"""
import numpy as np
import scipy.sparse as sp


def block_dense(p, i):
    A = sp.csr_matrix((p.a_vals[i], p.a_col, p.a_rowptr), shape=(p.nA, p.nA)).toarray()
    return A + A.T - np.diag(np.diag(A))


def lower_dense(rowptr, col, vals, n):
    A = sp.csr_matrix((vals, col, rowptr), shape=(n, n)).toarray()
    return A + A.T - np.diag(np.diag(A))


def b_dense(p, i):
    B = np.zeros((p.nA, p.nC))
    for q in range(p.b_blockptr[i], p.b_blockptr[i + 1]):
        B[p.b_row[q], p.b_col[q]] += p.b_vals[q]
    return B


def c_dense(p):
    if p.c_kind == 0:
        return np.diag(p.c_vals)
    return np.asarray(p.c_vals, dtype=np.float64).reshape(p.nC, p.nC)


def dense_K(p):
    nK = p.nK
    K = np.zeros((nK, nK))
    g = p.N * p.nA
    for i in range(p.N):
        s = slice(i * p.nA, (i + 1) * p.nA)
        K[s, s] = block_dense(p, i)
        B = b_dense(p, i)
        K[s, g:] = B
        K[g:, s] = B.T
    K[g:, g:] = c_dense(p)
    return K
