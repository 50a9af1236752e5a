"""The oracle's own block-CSR container for S-format matrices, and the compressed values
K^eta = P_S(T K T^T) (Sec. 3.3, Thm. (S-compression)) with the a-posteriori threshold of
Sec. 5.

Test infrastructure only (see ``oracle/__init__``).

Layout: clusters are block rows/columns; cluster nu owns rows boff[nu]:boff[nu+1]; block k
of row nu is (nu, colidx[k]) for rowptr[nu] <= k < rowptr[nu+1]; its entries are stored
row-major at val[voff[k]:voff[k+1]].

Threshold reading (the paper's a-posteriori pattern, Sec. 5, drops entries below tau; the
store keeps whole blocks): the decision is taken on the unordered pair, so that the kept
pattern of a symmetric matrix stays symmetric even where T K T^T is symmetric only up to
rounding.  With m(p, q) = max(|a_pq|, |a_qp|):
  * block (nu, nu') is kept iff nu = nu' or m >= tau for one of its entries;
  * entries with m < tau inside kept blocks are set to zero.
"""
import numpy as np


class BlockCSR:
    def __init__(self, bsize, rowptr, colidx, val=None):
        self.bsize = np.asarray(bsize, dtype=np.int64)
        self.boff = np.zeros(len(self.bsize) + 1, dtype=np.int64)
        self.boff[1:] = np.cumsum(self.bsize)
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.colidx = np.asarray(colidx, dtype=np.int64)
        nb = len(self.colidx)
        self.brow = np.repeat(np.arange(len(self.bsize)), np.diff(self.rowptr))
        sz = self.bsize[self.brow] * self.bsize[self.colidx]
        self.voff = np.zeros(nb + 1, dtype=np.int64)
        self.voff[1:] = np.cumsum(sz)
        if val is None:
            val = np.zeros(int(self.voff[-1]))
        self.val = np.asarray(val, dtype=np.float64)
        assert self.val.shape[0] == self.voff[-1]

    @property
    def n(self):
        return int(self.boff[-1])

    @property
    def nclusters(self):
        return len(self.bsize)

    @property
    def nblocks(self):
        return len(self.colidx)

    def like(self, val=None):
        return BlockCSR(self.bsize, self.rowptr, self.colidx, val)

    def block(self, k):
        i, j = self.brow[k], self.colidx[k]
        return self.val[self.voff[k]:self.voff[k + 1]].reshape(self.bsize[i], self.bsize[j])

    def find(self, i, j):
        """Block index of (i, j), or -1."""
        lo, hi = self.rowptr[i], self.rowptr[i + 1]
        pos = lo + np.searchsorted(self.colidx[lo:hi], j)
        if pos < hi and self.colidx[pos] == j:
            return int(pos)
        return -1

    def to_dense(self):
        A = np.zeros((self.n, self.n))
        for k in range(self.nblocks):
            i, j = self.brow[k], self.colidx[k]
            A[self.boff[i]:self.boff[i + 1], self.boff[j]:self.boff[j + 1]] = self.block(k)
        return A

    def mask(self):
        """Dense 0/1 mask of the pattern."""
        M = np.zeros((self.n, self.n))
        for k in range(self.nblocks):
            i, j = self.brow[k], self.colidx[k]
            M[self.boff[i]:self.boff[i + 1], self.boff[j]:self.boff[j + 1]] = 1.0
        return M

    @staticmethod
    def from_dense(D, bsize, rowptr, colidx):
        A = BlockCSR(bsize, rowptr, colidx)
        for k in range(A.nblocks):
            i, j = A.brow[k], A.colidx[k]
            A.val[A.voff[k]:A.voff[k + 1]] = \
                D[A.boff[i]:A.boff[i + 1], A.boff[j]:A.boff[j + 1]].ravel()
        return A

    def transpose(self):
        """B = A^T in the same format (pattern transposed, every block transposed)."""
        nc = self.nclusters
        cnt = np.bincount(self.colidx, minlength=nc)
        rowptr = np.zeros(nc + 1, dtype=np.int64)
        rowptr[1:] = np.cumsum(cnt)
        order = np.lexsort((self.brow, self.colidx))
        colidx = self.brow[order]
        B = BlockCSR(self.bsize, rowptr, colidx)
        for newk, k in enumerate(order):
            B.val[B.voff[newk]:B.voff[newk + 1]] = self.block(k).T.ravel()
        return B

    def identity_like(self, gamma=1.0):
        """gamma * I on this pattern (the pattern must hold the diagonal blocks)."""
        A = self.like()
        for i in range(self.nclusters):
            k = self.find(i, i)
            if self.bsize[i] == 0:
                continue
            assert k >= 0, "pattern lacks a diagonal block"
            A.val[A.voff[k]:A.voff[k + 1]] = (gamma * np.eye(self.bsize[i])).ravel()
        return A


def compress(Khat, bsize, rowptr, colidx, tau=0.0):
    """P_S(Khat) on the eta pattern, then the a-posteriori threshold (module docstring).

    Khat is the full samplet-coordinate matrix T K T^T (+ nugget).  Returns BlockCSR on
    the kept blocks.
    """
    bsize = np.asarray(bsize)
    boff = np.zeros(len(bsize) + 1, dtype=np.int64)
    boff[1:] = np.cumsum(bsize)
    nc = len(bsize)
    mag = np.abs(np.asarray(Khat, dtype=np.float64))
    mag = np.maximum(mag, mag.T)                 # m(p, q): the pair decides
    keep_rowptr = np.zeros(nc + 1, dtype=np.int64)
    keep_cols = []
    for i in range(nc):
        for k in range(rowptr[i], rowptr[i + 1]):
            j = colidx[k]
            blk = mag[boff[i]:boff[i + 1], boff[j]:boff[j + 1]]
            if i == j or np.any(blk >= tau):
                keep_cols.append(j)
        keep_rowptr[i + 1] = len(keep_cols)
    A = BlockCSR.from_dense(Khat, bsize, keep_rowptr, np.array(keep_cols, dtype=np.int64))
    if tau > 0.0:
        M = BlockCSR.from_dense(mag, bsize, keep_rowptr, np.array(keep_cols, dtype=np.int64))
        A.val[M.val < tau] = 0.0
    return A
