"""Input preparation for small N, end to end: points -> cluster tree -> samplet basis ->
pattern -> K^eta = P_S(T K T^T) (+ nugget) -> threshold (Sec. 3.2-3.3, Sec. 5).

Test infrastructure only (see ``oracle/__init__``).  Dense in N: for N up to a few
thousand.

Reading of the kernel scaling: the benchmarks of Sec. 5 scale the kernel by 1/N; here
``scale`` multiplies K, the nugget mu is added after scaling (T (sK + mu I) T^T =
s T K T^T + mu I since T is orthogonal), and tau is absolute on the resulting entries.
"""
import numpy as np

from .kernels import kernel_matrix, kernel_matrix_dell
from .pattern import eta_pattern
from .samplets import samplet_basis
from .sformat import compress
from .tree import build_tree


class Compressed:
    def __init__(self, clusters, basis, rowptr, colidx, A, Khat):
        self.clusters = clusters
        self.basis = basis
        self.rowptr_eta = rowptr     # a-priori eta pattern
        self.colidx_eta = colidx
        self.A = A                   # BlockCSR after the threshold
        self.Khat = Khat             # dense T K T^T (+ mu I), before masking


def compress_kernel(points, nu, ell, q, leaf, eta, tau=0.0, scale=1.0, nugget=0.0):
    x = np.asarray(points, dtype=np.float64)
    clusters = build_tree(x, leaf)
    basis = samplet_basis(x, clusters, q)
    rowptr, colidx = eta_pattern(clusters, basis.bsize, eta)
    K = kernel_matrix(x, nu, ell, scale)
    Khat = basis.T @ K @ basis.T.T + nugget * np.eye(x.shape[0])
    A = compress(Khat, basis.bsize, rowptr, colidx, tau)
    return Compressed(clusters, basis, rowptr, colidx, A, Khat)


def dA_dell(points, basis, A, nu, ell, scale=1.0):
    """P_S(T dK/dell T^T) on A's pattern (the nugget does not depend on ell)."""
    from .sformat import BlockCSR
    dK = kernel_matrix_dell(np.asarray(points, dtype=np.float64), nu, ell, scale)
    D = basis.T @ dK @ basis.T.T
    return BlockCSR.from_dense(D, A.bsize, A.rowptr, A.colidx)
