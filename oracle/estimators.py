"""Error estimator of the paper's multiplication benchmark, in FP64.

Test infrastructure only (see ``oracle/__init__``).

Sec. 5.1 measures the error of the formatted product with

    e_F(M) = ||M X||_F / ||X||_F,

X an N x 10 matrix of independent uniform entries, applied to M = A B - A (.) B: the exact
product of the two compressed matrices minus the formatted (masked) one.  M is never formed:
M X = A (B X) - C X with C = P_S(A B), three block-sparse times dense products.
"""
import math

import numpy as np

from . import product as _prod


def spmm(A, X):
    """A X for a BlockCSR A and a dense N x k X (column by column)."""
    X = np.asarray(X, dtype=np.float64)
    return np.stack([_prod.spmv(A, X[:, j]) for j in range(X.shape[1])], axis=1)


def ef(A, B, C, X):
    """e_F(A B - C) = ||A (B X) - C X||_F / ||X||_F."""
    M = spmm(A, spmm(B, X)) - spmm(C, X)
    return float(np.linalg.norm(M) / np.linalg.norm(X))


def ef_of(M, X):
    """e_F(M) for a BlockCSR M."""
    return float(np.linalg.norm(spmm(M, X)) / np.linalg.norm(X))


def frob(M):
    return math.sqrt(float(np.dot(M.val, M.val)))
