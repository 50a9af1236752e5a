"""Samplet basis by the two-scale QR construction (Sec. 3.2: refinement relation, Eq. (QR),
Eq. (vanishingMomentsQR), leaf scaling distributions, Eq. (Wbasis); properties in
Thm. (waveletProperties)).  Dense transform T, so for small N only.

Test infrastructure only (see ``oracle/__init__``).

Readings of the paper (it fixes neither):
  * monomials x^alpha, |alpha| <= q, in graded order: total degree 0..q, and within a
    degree lexicographically with the first exponent largest first;
  * moments are taken in the cluster's local coordinates (x - c) / s with c the bounding
    box centre and s half its longest edge (s = 1 for a one-point box); this is a
    graded-triangular change of the polynomial basis, so the spans in Eq. (QR) and the
    vanishing-moment property are unchanged;
  * Householder QR with the reflector u = x - beta e1, beta = -sign(x_0) |x| (sign(0) = +1),
    and no reflector when the part of the column below the diagonal is zero;
  * a cluster keeps min(m_q, n_in) scaling functions (n_in = number of functions it
    receives from its sons, or its point count for a leaf) and n_in - min(m_q, n_in)
    samplets; the root also keeps its scaling functions as coordinates, ahead of its
    samplets;
  * coordinate order: clusters breadth first, and within a cluster the order of the
    columns of Q.
"""
from itertools import product as iproduct

import numpy as np


def monomial_exponents(d, q):
    """All alpha in N_0^d with |alpha| <= q, graded, first exponent largest first."""
    out = []
    for g in range(q + 1):
        degs = [a for a in iproduct(range(g + 1), repeat=d) if sum(a) == g]
        degs.sort(reverse=True)
        out.extend(degs)
    return np.array(out, dtype=np.int64).reshape(-1, d)


def m_q(d, q):
    """m_q = sum_{l=0}^q C(l+d-1, d-1), the dimension of P_q (Sec. 3.2)."""
    return len(monomial_exponents(d, q))


def monomials(y, exps):
    """[y_i^alpha]_{i, alpha} for local coordinates y (n x d)."""
    y = np.asarray(y, dtype=np.float64)
    out = np.ones((y.shape[0], exps.shape[0]))
    for k, a in enumerate(exps):
        for ax in range(y.shape[1]):
            if a[ax]:
                out[:, k] *= y[:, ax] ** a[ax]
    return out


def householder_qr(A):
    """Full QR, A = Q R with Q square orthogonal, by Householder reflections written out
    from the textbook definition (reflector convention in the module docstring).

    Pinned against numpy.linalg.qr(mode='complete') in tests/test_oracle_samplets.py.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    n, m = R.shape
    Q = np.eye(n)
    for k in range(min(n, m)):
        x = R[k:, k].copy()
        if x.size <= 1 or not np.any(x[1:] != 0.0):
            continue
        normx = np.sqrt(np.dot(x, x))
        beta = -normx if x[0] >= 0.0 else normx
        u = x
        u[0] -= beta
        u /= np.sqrt(np.dot(u, u))
        R[k:, :] -= 2.0 * np.outer(u, u @ R[k:, :])
        Q[:, k:] -= 2.0 * np.outer(Q[:, k:] @ u, u)
    return Q, R


class SampletBasis:
    """Result of ``samplet_basis``.

    T        dense N x N transform, rows = samplet coefficient vectors omega over the
             original point order (Eq. (coefficientVectorsOfWavelets)).
    bsize    rows of T owned by each cluster (root: scaling + samplets).
    boff     row offsets, bsize prefix sums.
    nscal    scaling functions kept by each cluster.
    Q        per-cluster two-scale matrices Q^nu of Eq. (QR).
    """

    def __init__(self, T, bsize, boff, nscal, Q):
        self.T = T
        self.bsize = bsize
        self.boff = boff
        self.nscal = nscal
        self.Q = Q


def samplet_basis(points, clusters, q):
    x = np.asarray(points, dtype=np.float64)
    n, d = x.shape
    exps = monomial_exponents(d, q)
    mq = exps.shape[0]
    nc = len(clusters)
    phi = [None] * nc     # |nu| x nscal weights of the scaling functions, in nu's point order
    sig = [None] * nc     # |nu| x nsamp weights of the samplets
    Qs = [None] * nc
    nscal = np.zeros(nc, dtype=np.int64)
    for c in reversed(clusters):
        npts = len(c.idx)
        if not c.sons:
            psi = np.eye(npts)                       # Dirac measures at the leaf's points
        else:
            blocks = [phi[s] for s in c.sons]
            rows = sum(b.shape[0] for b in blocks)
            cols = sum(b.shape[1] for b in blocks)
            psi = np.zeros((rows, cols))
            r0 = c0 = 0
            for b in blocks:
                psi[r0:r0 + b.shape[0], c0:c0 + b.shape[1]] = b
                r0 += b.shape[0]
                c0 += b.shape[1]
        centre = 0.5 * (c.bmin + c.bmax)
        half = 0.5 * float(np.max(c.bmax - c.bmin))
        if half <= 0.0:
            half = 1.0
        P = monomials((x[c.idx] - centre) / half, exps)   # |nu| x m_q
        Mt = psi.T @ P                                      # (M^nu)^T, n_in x m_q
        Q, _ = householder_qr(Mt)
        nin = psi.shape[1]
        ns = min(mq, nin)
        nscal[c.id] = ns
        Qs[c.id] = Q
        phi[c.id] = psi @ Q[:, :ns]
        sig[c.id] = psi @ Q[:, ns:]
    bsize = np.array([sig[c.id].shape[1] for c in clusters], dtype=np.int64)
    bsize[0] += nscal[0]
    boff = np.zeros(nc + 1, dtype=np.int64)
    boff[1:] = np.cumsum(bsize)
    assert boff[-1] == n
    T = np.zeros((n, n))
    for c in clusters:
        r = boff[c.id]
        if c.id == 0:
            T[r:r + nscal[0], c.idx] = phi[0].T
            r += nscal[0]
        k = sig[c.id].shape[1]
        T[r:r + k, c.idx] = sig[c.id].T
    return SampletBasis(T, bsize, boff, nscal, Qs)
