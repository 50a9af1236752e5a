"""Host logic of the selected inversion (include/sselinv.h), no GPU needed: the elimination
order and the size of the factor against the oracle's elimination game (Sec. 4.2), and the
quadrature nodes of Eq. (ContInt) against scipy's elliptic functions (oracle.contour)."""
import numpy as np
import pytest

from oracle import contour, selinv as osel
from tests.test_oracle_product import random_pattern


@pytest.fixture(scope="module")
def si():
    from paper_2211_11681_gb300 import build
    build.build()
    from paper_2211_11681_gb300 import selinv
    return selinv


def symmetric_pattern(nc, density, seed):
    rp, ci = random_pattern(nc, density, seed)
    M = np.zeros((nc, nc), dtype=bool)
    for r in range(nc):
        M[r, ci[rp[r]:rp[r + 1]]] = True
    M |= M.T
    np.fill_diagonal(M, True)
    rowptr = np.concatenate([[0], np.cumsum(M.sum(axis=1))]).astype(np.int64)
    colidx = np.concatenate([np.nonzero(M[r])[0] for r in range(nc)]).astype(np.int64)
    return rowptr, colidx, M


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_order_against_the_elimination_game(si, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = 40
    bsize = rng.integers(0, 7, size=nc)                 # some empty clusters
    rowptr, colidx, M = symmetric_pattern(nc, 0.12, seed)
    perm, nl, levels = si.order(bsize, rowptr, colidx)
    assert sorted(perm.tolist()) == list(range(nc))
    m = int((bsize > 0).sum())
    assert all(bsize[perm[:m]] > 0) and all(bsize[perm[m:]] == 0)   # empty clusters last
    st = [[i for i in s if i < m] for s in osel.block_fill(nc, rowptr, colidx, perm)[:m]]
    assert nl == m + sum(len(s) for s in st)
    assert levels == int(osel.etree_levels(st).max()) + 1
    # minimum degree: the first cluster eliminated has the fewest non-empty neighbours
    ne = bsize > 0
    deg = [(M[c] & ne).sum() - 1 for c in range(nc)]
    assert deg[perm[0]] == min(deg[c] for c in range(nc) if ne[c])


def test_order_on_a_samplet_pattern(si):
    import workloads as W
    from oracle.pipeline import compress_kernel
    w = W.WORKLOADS["paper_mult_2d"]
    n = 1024
    c = compress_kernel(W.points(w, n), w.nu, w.ell, w.q, w.leaf, w.eta, W.tau_of(w, n), 1.0 / n, 0.0)
    A = c.A
    perm, nl, levels = si.order(A.bsize, A.rowptr, A.colidx)
    m = int((A.bsize > 0).sum())
    st = [[i for i in s if i < m] for s in osel.block_fill(A.nclusters, A.rowptr, A.colidx, perm)[:m]]
    assert nl == m + sum(len(s) for s in st)
    lower = (A.nblocks - A.nclusters) // 2 + A.nclusters
    assert lower <= nl + (A.nclusters - m)               # the factor holds S's lower part


def test_order_rejects_a_non_symmetric_pattern(si):
    from paper_2211_11681_gb300 import sformat as sf
    rowptr = np.array([0, 2, 3], dtype=np.int64)
    colidx = np.array([0, 1, 1], dtype=np.int64)          # (0,1) without (1,0)
    with pytest.raises(sf.SFormatError) as e:
        si.order(np.array([2, 3]), rowptr, colidx)
    assert e.value.status == sf.S_ERR_PATTERN


@pytest.mark.parametrize("c_lo,c_hi,n", [(1e-4, 1.0, 7), (1.0, 1.0, 5), (1e-6, 1.0, 12), (0.3, 2.0, 9)])
def test_contour_nodes_match_scipy(si, c_lo, c_hi, n):
    w2, wt = si.contour_nodes(c_lo, c_hi, n)
    v2, vt = contour.nodes(c_lo, c_hi, n)
    np.testing.assert_allclose(w2, v2, rtol=1e-12)
    np.testing.assert_allclose(wt, vt, rtol=1e-12)


def test_contour_nodes_reject_bad_intervals(si):
    from paper_2211_11681_gb300 import sformat as sf
    for args in [(0.0, 1.0, 7), (2.0, 1.0, 7), (1e-4, 1.0, 0)]:
        with pytest.raises(sf.SFormatError) as e:
            si.contour_nodes(*args)
        assert e.value.status == sf.S_ERR_ARG
