"""Pins of the oracle's selected inversion (Sec. 4.2, Eq. (blockInv)), of the elimination
game behind the factor's pattern, and of the contour-integral quadrature (Eq. (ContInt),
Sec. 4.4), each against something other than the oracle itself:

  * the Kac-Murdock-Szego matrix rho^|i-j|, whose inverse is tridiagonal in closed form;
  * the 2 x 2 block formula of Eq. (blockInv) (Schur complement of the leading block);
  * diagonal matrices under a shift;
  * the structure of a dense Cholesky factor of generic values (brute force) and two graphs
    whose fill is known by hand (an arrow and a path);
  * for the quadrature, the closed form at c_lo = c_hi (sn = sin, cn = cos, dn = 1,
    K(0) = pi/2), the scalar limit lambda^{-1/2} over the whole spectral interval, and the
    matrix square root through an eigendecomposition."""
import math

import numpy as np
import pytest

from oracle import contour, selinv
from oracle.sformat import BlockCSR
from tests.test_oracle_product import random_pattern


def full_pattern(nc):
    rowptr = np.arange(nc + 1, dtype=np.int64) * nc
    colidx = np.tile(np.arange(nc, dtype=np.int64), nc)
    return rowptr, colidx


def band_pattern(nc, w):
    rowptr, cols = [0], []
    for i in range(nc):
        js = [j for j in range(nc) if abs(i - j) <= w]
        cols.extend(js)
        rowptr.append(len(cols))
    return np.array(rowptr, dtype=np.int64), np.array(cols, dtype=np.int64)


def kms(n, rho):
    i = np.arange(n)
    return rho ** np.abs(i[:, None] - i[None, :])


def kms_inverse(n, rho):
    """Closed form: tridiagonal, 1/(1-rho^2) times (1+rho^2 inside, 1 at both ends, -rho
    off the diagonal)."""
    T = np.zeros((n, n))
    d = np.full(n, 1.0 + rho * rho)
    d[0] = d[-1] = 1.0
    T[np.diag_indices(n)] = d
    T[np.arange(n - 1), np.arange(1, n)] = -rho
    T[np.arange(1, n), np.arange(n - 1)] = -rho
    return T / (1.0 - rho * rho)


@pytest.mark.parametrize("rho", [0.3, 0.9])
def test_kms_inverse_closed_form(rho):
    bsize = np.array([3, 2, 4, 1, 3, 5])
    n = int(bsize.sum())
    want = kms_inverse(n, rho)
    rp, ci = full_pattern(len(bsize))
    A = BlockCSR.from_dense(kms(n, rho), bsize, rp, ci)
    Z = selinv.selected_inverse(A)
    np.testing.assert_allclose(Z.to_dense(), want, rtol=0, atol=1e-10 / (1 - rho * rho))
    # a block-tridiagonal matrix (the KMS matrix's blocks on that pattern) is a different
    # matrix: its selected inverse is P_S of its own inverse and holds no other blocks
    rp, ci = band_pattern(len(bsize), 1)
    Ab = BlockCSR.from_dense(kms(n, rho), bsize, rp, ci)
    Zb = selinv.selected_inverse(Ab)
    assert Zb.nblocks == Ab.nblocks
    np.testing.assert_allclose(Zb.to_dense() @ np.eye(n) * Ab.mask(),
                               np.linalg.inv(Ab.to_dense()) * Ab.mask(), rtol=0, atol=1e-10)


def test_block_inverse_formula():
    """Eq. (blockInv): A^{-1} from A11^{-1}, C = -A11^{-1} A12 and the Schur complement
    S = A22 + A12^T C."""
    rng = np.random.Generator(np.random.PCG64(3))
    bsize = np.array([4, 3, 5, 2])
    n = int(bsize.sum())
    G = rng.standard_normal((n, n))
    M = G @ G.T + n * np.eye(n)
    k = 7                                          # split after the first two clusters
    A11, A12, A22 = M[:k, :k], M[:k, k:], M[k:, k:]
    A11i = np.linalg.inv(A11)
    C = -A11i @ A12
    Si = np.linalg.inv(A22 + A12.T @ C)
    want = np.block([[A11i + C @ Si @ C.T, C @ Si], [Si @ C.T, Si]])
    Z = selinv.selected_inverse(BlockCSR.from_dense(M, bsize, *full_pattern(4)))
    np.testing.assert_allclose(Z.to_dense(), want, rtol=1e-12, atol=1e-14)


def test_inverse_columns_by_conjugate_gradients():
    """Columns of the KMS inverse (closed form) through the sparse CG route, with a shift."""
    bsize = np.array([3, 2, 4, 1, 3, 5])
    n = int(bsize.sum())
    rho = 0.6
    A = BlockCSR.from_dense(kms(n, rho), bsize, *full_pattern(len(bsize)))
    M = selinv.to_scipy(A)
    np.testing.assert_array_equal(M.toarray(), kms(n, rho))
    cols = [0, 5, n - 1]
    X = selinv.inverse_columns(M, 0.0, cols)
    np.testing.assert_allclose(X, kms_inverse(n, rho)[:, cols], rtol=0, atol=1e-10)
    Xs = selinv.inverse_columns(M, 0.5, cols)
    np.testing.assert_allclose(Xs, np.linalg.inv(kms(n, rho) + 0.5 * np.eye(n))[:, cols], rtol=0, atol=1e-10)


def test_diagonal_shift():
    bsize = np.array([2, 3])
    d = np.array([1.0, 2.0, 4.0, 0.5, 3.0])
    rp, ci = band_pattern(2, 0)
    A = BlockCSR.from_dense(np.diag(d), bsize, rp, ci)
    Z = selinv.selected_inverse(A, 0.25)
    np.testing.assert_allclose(np.diag(Z.to_dense()), 1.0 / (d + 0.25), rtol=1e-15)


def dense_factor_structure(bsize, rowptr, colidx, perm, seed):
    """Block structure of the Cholesky factor of a generic SPD matrix with the given block
    pattern, clusters in the order perm (brute force: factor and look at the blocks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = len(bsize)
    A = BlockCSR(bsize, rowptr, colidx)
    A.val[:] = rng.uniform(-1.0, 1.0, len(A.val))
    D = A.to_dense()
    D = D + D.T
    D += np.eye(D.shape[0]) * (np.abs(D).sum(axis=1).max() + 1.0)
    idx = np.concatenate([np.arange(A.boff[c], A.boff[c + 1]) for c in perm])
    Lf = np.linalg.cholesky(D[np.ix_(idx, idx)])
    off = np.zeros(nc + 1, dtype=np.int64)
    off[1:] = np.cumsum(bsize[np.asarray(perm)])
    struct = []
    for p in range(nc):
        s = []
        for q in range(p + 1, nc):
            blk = Lf[off[q]:off[q + 1], off[p]:off[p + 1]]
            if blk.size and np.abs(blk).max() > 1e-12:
                s.append(q)
        struct.append(s)
    return struct


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_block_fill_against_dense_cholesky(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = 14
    bsize = rng.integers(1, 4, size=nc)
    rp, ci = random_pattern(nc, 0.18, seed)
    # symmetrise the pattern
    M = np.zeros((nc, nc), dtype=bool)
    for r in range(nc):
        M[r, ci[rp[r]:rp[r + 1]]] = True
    M |= M.T
    rowptr = np.concatenate([[0], np.cumsum(M.sum(axis=1))]).astype(np.int64)
    colidx = np.concatenate([np.nonzero(M[r])[0] for r in range(nc)]).astype(np.int64)
    perm = rng.permutation(nc)
    got = selinv.block_fill(nc, rowptr, colidx, perm)
    want = dense_factor_structure(bsize, rowptr, colidx, perm, seed + 100)
    assert got == want


def test_block_fill_arrow_and_path():
    nc = 6                                         # cluster 0 is the hub of an arrow
    M = np.eye(nc, dtype=bool)
    M[0, :] = M[:, 0] = True
    rowptr = np.concatenate([[0], np.cumsum(M.sum(axis=1))]).astype(np.int64)
    colidx = np.concatenate([np.nonzero(M[r])[0] for r in range(nc)]).astype(np.int64)
    leaves_first = selinv.block_fill(nc, rowptr, colidx, [1, 2, 3, 4, 5, 0])
    assert leaves_first == [[5]] * 5 + [[]]        # no fill
    assert list(selinv.etree_levels(leaves_first)) == [0, 0, 0, 0, 0, 1]
    hub_first = selinv.block_fill(nc, rowptr, colidx, [0, 1, 2, 3, 4, 5])
    assert hub_first == [[1, 2, 3, 4, 5], [2, 3, 4, 5], [3, 4, 5], [4, 5], [5], []]   # a clique
    assert list(selinv.etree_levels(hub_first)) == [0, 1, 2, 3, 4, 5]
    path = np.eye(nc, dtype=bool) | np.eye(nc, k=1, dtype=bool) | np.eye(nc, k=-1, dtype=bool)
    rowptr = np.concatenate([[0], np.cumsum(path.sum(axis=1))]).astype(np.int64)
    colidx = np.concatenate([np.nonzero(path[r])[0] for r in range(nc)]).astype(np.int64)
    s = selinv.block_fill(nc, rowptr, colidx, [0, 5, 1, 4, 2, 3])  # both ends inward
    assert sum(len(x) for x in s) == nc - 1        # a path eliminated from its ends: no fill


# ---- Eq. (ContInt) --------------------------------------------------------------------


def test_nodes_closed_form_at_zero_parameter():
    """c_lo = c_hi = c: m = 0, K(0) = pi/2, sn = sin, cn = cos, dn = 1, so w_k^2 =
    c tan^2 t_k, weights sqrt(c) / (n cos^2 t_k), and the rule gives c^{-1/2} exactly."""
    c, n = 2.5, 5
    w2, wt = contour.nodes(c, c, n)
    t = (math.pi / 2) * (np.arange(1, n + 1) - 0.5) / n
    np.testing.assert_allclose(w2, c * np.tan(t) ** 2, rtol=1e-14)
    np.testing.assert_allclose(wt, math.sqrt(c) / (n * np.cos(t) ** 2), rtol=1e-14)
    assert abs(np.sum(wt / (c + w2)) - 1.0 / math.sqrt(c)) < 1e-15


@pytest.mark.parametrize("ratio", [1e2, 1e4, 1e6])
def test_scalar_limit_over_the_interval(ratio):
    """The rule converges to lambda^{-1/2} on all of [c_lo, c_hi] (geometric decrease in
    the number of nodes); a wrong constant in place of K(1 - c_lo/c_hi) does not."""
    lam = np.geomspace(1.0, ratio, 101)
    errs = []
    for n in (5, 10, 20, 40):
        w2, wt = contour.nodes(1.0, ratio, n)
        approx = (wt[None, :] / (lam[:, None] + w2[None, :])).sum(axis=1)
        errs.append(np.abs(approx * np.sqrt(lam) - 1.0).max())
    assert errs[-1] < 1e-12
    assert all(b < a for a, b in zip(errs[:2], errs[1:3]))
    assert errs[1] < 1e-4 if ratio <= 1e4 else errs[1] < 1e-3


def test_matrix_inverse_square_root_through_eigh():
    rng = np.random.Generator(np.random.PCG64(9))
    bsize = np.array([3, 4, 2, 5])
    n = int(bsize.sum())
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1e-3, 1.0, n)
    M = (Q * lam) @ Q.T
    rp, ci = full_pattern(4)
    A = BlockCSR.from_dense(M, bsize, rp, ci)
    Z = contour.invsqrt(A, 1e-3, 1.0, 40)
    want = (Q / np.sqrt(lam)) @ Q.T
    assert np.linalg.norm(Z.to_dense() - want) <= 1e-10 * np.linalg.norm(want)
    R = contour.sqrt(A, Z)
    np.testing.assert_allclose(R.to_dense() @ R.to_dense(), M, atol=1e-10)
