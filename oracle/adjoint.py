"""Reverse mode of the masked product and of the masked Newton-Schulz iteration, in FP64.

Test infrastructure only (see ``oracle/__init__``).

For C = P_{S_C}(A B) with A on S_A and B on S_B, the adjoints are masked products too:
    dA = P_{S_A}(dC B^T),   dB = P_{S_B}(A^T dC).
The Newton-Schulz backward replays the forward of ``funm.sqrtm_ns`` in reverse with c
frozen; the loss used by the gradient checks is L = z^T X z with X = P_S(A^{1/2}) on S.
"""
import math

import numpy as np

from . import product as _prod
from .funm import add


def mul_masked_adjoint(dC, A, B, nthreads=1):
    dA = _prod.mul_masked(dC, B.transpose(), A, nthreads=nthreads)
    dB = _prod.mul_masked(A.transpose(), dC, B, nthreads=nthreads)
    return dA, dB


def _acc(X, Y):
    return X.like(X.val + Y.val)


def sqrtm_ns_backward(dX, hist, c, nthreads=1):
    """dL/dA on S for X = sqrtm_ns(A, ...), given dL/dX on S and the forward history."""
    S = dX
    dY = S.like(math.sqrt(c) * dX.val)
    dZ = S.like()
    for Y, Z in reversed(hist):
        P = _prod.mul_masked(Z, Y, S, nthreads=nthreads)
        T = add(P, P, alpha=-0.5, beta=0.0, gamma=1.5)
        # Y' = P_S(Y T),  Z' = P_S(T Z)
        dYk, dT1 = mul_masked_adjoint(dY, Y, T, nthreads)
        dT2, dZk = mul_masked_adjoint(dZ, T, Z, nthreads)
        dT = _acc(dT1, dT2)
        dP = dT.like(-0.5 * dT.val)                 # T = 1.5 I - 0.5 P
        dZp, dYp = mul_masked_adjoint(dP, Z, Y, nthreads)   # P = P_S(Z Y)
        dY = _acc(dYk, dYp)
        dZ = _acc(dZk, dZp)
    return dY.like(dY.val / c)


def quad_form(X, z):
    """z^T X z over the stored blocks of X."""
    tot = 0.0
    for k in range(X.nblocks):
        i, j = X.brow[k], X.colidx[k]
        zi = z[X.boff[i]:X.boff[i + 1]]
        zj = z[X.boff[j]:X.boff[j + 1]]
        tot += float(zi @ X.block(k) @ zj)
    return tot


def quad_form_grad(S, z):
    """dL/dX of L = z^T X z: the block (nu, nu') of S gets z_nu z_nu'^T."""
    G = S.like()
    for k in range(S.nblocks):
        i, j = S.brow[k], S.colidx[k]
        G.val[G.voff[k]:G.voff[k + 1]] = np.outer(z[S.boff[i]:S.boff[i + 1]],
                                                  z[S.boff[j]:S.boff[j + 1]]).ravel()
    return G
