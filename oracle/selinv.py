"""Selected inversion on the compression pattern (Sec. 4.2 "Sparse selected inversion",
Eq. (blockInv)), in FP64.

Test infrastructure only (see ``oracle/__init__``).

The method factors A = L D L^T and then computes the entries of A^{-1} on the pattern of L
from the recurrences that follow from Eq. (blockInv); the pattern of L contains the pattern
of A, and the paper keeps the entries on the pattern of A (the compression pattern S).  Up
to rounding these are the entries of the exact inverse, so the oracle is that definition:

    selected_inverse(A, sigma) = P_S((A + sigma I)^{-1}),

the dense inverse of the shifted matrix restricted to the blocks of S.

For sizes where a dense inverse is out of reach, ``inverse_columns`` computes chosen columns
of (A + sigma I)^{-1} by conjugate gradients (scipy) on the sparse matrix, to be compared on
the entries of S in those columns.

``block_fill`` is the symbolic side: the block pattern of L when the clusters are eliminated
in a given order, by the elimination game (eliminating a block column joins all blocks that
are still to be eliminated and are adjacent to it into a clique), the textbook rule for the
structure of a Cholesky or LDL^T factor (no cancellation assumed).
"""
import numpy as np

from .sformat import BlockCSR


def selected_inverse(A, sigma=0.0):
    """P_S((A + sigma I)^{-1}) as a BlockCSR on A's pattern (A symmetric positive definite
    after the shift)."""
    D = A.to_dense()
    D[np.diag_indices_from(D)] += sigma
    Z = np.linalg.solve(D, np.eye(D.shape[0]))
    return BlockCSR.from_dense(Z, A.bsize, A.rowptr, A.colidx)


def to_scipy(A):
    """A as a scipy CSR matrix (entry level)."""
    import scipy.sparse as sp
    rows, cols, vals = [], [], []
    for k in range(A.nblocks):
        i, j = A.brow[k], A.colidx[k]
        bi, bj = A.bsize[i], A.bsize[j]
        if bi == 0 or bj == 0:
            continue
        r = np.repeat(np.arange(A.boff[i], A.boff[i + 1]), bj)
        c = np.tile(np.arange(A.boff[j], A.boff[j + 1]), bi)
        rows.append(r)
        cols.append(c)
        vals.append(A.val[A.voff[k]:A.voff[k + 1]])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(A.n, A.n))


def inverse_columns(M, sigma, cols, rtol=1e-13):
    """Columns ``cols`` of (M + sigma I)^{-1} for a sparse symmetric positive definite scipy
    matrix M, by conjugate gradients (dense array n x len(cols))."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n = M.shape[0]
    B = (M + sigma * sp.identity(n, format="csr")).tocsr()
    out = np.zeros((n, len(cols)))
    for t, c in enumerate(cols):
        e = np.zeros(n)
        e[c] = 1.0
        try:
            x, info = sla.cg(B, e, rtol=rtol, atol=0.0, maxiter=20 * n)
        except TypeError:  # scipy before 1.12 names the relative tolerance `tol`
            x, info = sla.cg(B, e, tol=rtol, atol=0.0, maxiter=20 * n)
        if info != 0:
            raise RuntimeError("conjugate gradients did not converge (info %d)" % info)
        out[:, t] = x
    return out


def block_fill(nclusters, rowptr, colidx, perm):
    """Column structures of the block factor L for the elimination order ``perm``
    (perm[p] = cluster eliminated p-th).  Returns ``struct``: struct[p] is the sorted list
    of positions q > p with L(q, p) != 0 (blocks below the diagonal, in position space).
    The pattern (rowptr, colidx) must be symmetric."""
    nc = int(nclusters)
    pos = np.empty(nc, dtype=np.int64)
    pos[np.asarray(perm, dtype=np.int64)] = np.arange(nc)
    adj = [set() for _ in range(nc)]
    for r in range(nc):
        for c in colidx[rowptr[r]:rowptr[r + 1]]:
            pr, pc = int(pos[r]), int(pos[int(c)])
            if pr != pc:
                adj[min(pr, pc)].add(max(pr, pc))
    struct = []
    for p in range(nc):
        s = sorted(adj[p])
        struct.append(s)
        # eliminating p joins its later neighbours into a clique; the first of them (the
        # parent in the elimination tree) carries the clique onward
        if s:
            adj[s[0]].update(s[1:])
    return struct


def etree_levels(struct):
    """Level of every position in the elimination tree (leaves 0, a parent one above its
    highest child); the parent of p is min(struct[p])."""
    nc = len(struct)
    lvl = np.zeros(nc, dtype=np.int64)
    for p in range(nc):
        if struct[p]:
            q = struct[p][0]
            lvl[q] = max(lvl[q], lvl[p] + 1)
    return lvl
