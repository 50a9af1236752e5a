"""S-format addition, norm estimate, and the two matrix-function drivers, in FP64.

Test infrastructure only (see ``oracle/__init__``).

  add            C = alpha A + beta B + gamma I on a common pattern (Sec. 4.1: addition of
                 matrices compressed on the same pattern).
  norm_estimate  largest eigenvalue by power iteration with Rayleigh quotients, 50 steps
                 (Sec. 5.3 estimates ||K^eta||_2 this way).  Reading: start vector all ones.
  sqrtm_ns       A^{1/2} by the coupled Newton-Schulz iteration (the paper computes A^{1/2}
                 by a contour integral with selected inversion, Sec. 4.4; this is the
                 product-only method: Y_0 = A/c, Z_0 = I, T_k = (3I - Z_k Y_k)/2,
                 Y_{k+1} = Y_k T_k, Z_{k+1} = T_k Z_k, X = sqrt(c) Y_K), every product masked
                 to S.  Reading: c = 1.01 * norm_estimate(A), frozen.  Optional residual
                 correction after the iteration (Newton's method for Y^2 = A/c with the
                 inverse of Y replaced by the coupled iterate Z ~ (A/c)^{-1/2}):
                 R = A/c - P_S(Y Y), Y <- Y + P_S(Z R)/2, repeated `refine` times
                 (``ns_refine``).
  expm_taylor    exp(sign * A) by the power series of Sec. 4.4, truncated at degree 8
                 (Sec. 5.3 finds stagnation after 8 terms), evaluated by Horner's rule on
                 X = sign*A/2^s, then s masked squarings.  Reading: s = max(0,
                 ceil(log2(lambda/theta))), theta = 0.5, lambda = norm_estimate(A); s = 0
                 gives the paper's plain truncated series.
"""
import math

import numpy as np

from . import product as _prod
from .sformat import BlockCSR


def add(A, B, alpha=1.0, beta=1.0, gamma=0.0):
    """alpha A + beta B + gamma I, all on A's pattern (B must share it)."""
    assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.colidx, B.colidx)
    C = A.like(alpha * A.val + beta * B.val)
    if gamma != 0.0:
        C.val = C.val + A.identity_like(gamma).val
    return C


def frob(A):
    return float(np.sqrt(np.dot(A.val, A.val)))


def norm_estimate(A, iters=50):
    x = np.ones(A.n) / math.sqrt(A.n)
    lam = 0.0
    for _ in range(iters):
        y = _prod.spmv(A, x)
        lam = float(np.dot(x, y))
        ny = math.sqrt(float(np.dot(y, y)))
        if ny == 0.0:
            return 0.0
        x = y / ny
    return lam


def sqrtm_ns(A, steps=25, c=None, return_history=False, nthreads=1, refine=0):
    """Returns X (and, with return_history, the list of (Y_k, Z_k) and c)."""
    if c is None:
        c = 1.01 * norm_estimate(A)
    Y = A.like(A.val / c)
    Z = A.identity_like(1.0)
    hist = []
    for _ in range(steps):
        hist.append((Y, Z))
        P = _prod.mul_masked(Z, Y, A, nthreads=nthreads)
        T = add(P, P, alpha=-0.5, beta=0.0, gamma=1.5)
        Yn = _prod.mul_masked(Y, T, A, nthreads=nthreads)
        Zn = _prod.mul_masked(T, Z, A, nthreads=nthreads)
        Y, Z = Yn, Zn
    Y = ns_refine(A.like(A.val / c), Y, Z, refine, nthreads=nthreads)
    X = A.like(math.sqrt(c) * Y.val)
    if return_history:
        return X, hist, c
    return X


def ns_refine(B, Y, Z, steps, nthreads=1):
    """Residual correction of an approximate square root Y of B with Z ~ B^{-1/2}: Newton's
    method for Y^2 = B, the correction E of (Y + E)^2 = B to first order being taken as
    Z R / 2 with R = B - Y Y (exact when Y, Z and R commute).  Every product masked to B's
    pattern:  R = B - P_S(Y Y),  Y <- Y + P_S(Z R)/2,  `steps` times."""
    for _ in range(steps):
        R = add(B, _prod.mul_masked(Y, Y, B, nthreads=nthreads), 1.0, -1.0)
        Y = add(Y, _prod.mul_masked(Z, R, B, nthreads=nthreads), 1.0, 0.5)
    return Y


def sqrt_residual(X, A, nthreads=1):
    """||P_S(X X) - A||_F / ||A||_F."""
    XX = _prod.mul_masked(X, X, A, nthreads=nthreads)
    return frob(add(XX, A, 1.0, -1.0)) / frob(A)


def exp_scaling(lam, theta=0.5):
    if lam <= theta:
        return 0
    return max(0, int(math.ceil(math.log2(lam / theta))))


def expm_taylor(A, sign=1.0, degree=8, s=None, nthreads=1):
    if s is None:
        s = exp_scaling(abs(norm_estimate(A)))
    X = A.like(sign * A.val / (2.0 ** s))
    E = add(X, X, alpha=1.0 / degree, beta=0.0, gamma=1.0)          # I + X/m
    for k in range(degree - 1, 0, -1):
        XE = _prod.mul_masked(X, E, A, nthreads=nthreads)
        E = add(XE, XE, alpha=1.0 / k, beta=0.0, gamma=1.0)         # I + X E / k
    for _ in range(s):
        E = _prod.mul_masked(E, E, A, nthreads=nthreads)
    return E
