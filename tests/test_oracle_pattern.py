"""Pins of the oracle's compression pattern (Eq. (cutoff), Thm. (S-compression))."""
import numpy as np
import pytest

from oracle.pattern import eta_pattern
from oracle.samplets import samplet_basis
from oracle.tree import build_tree


def _pairs(rowptr, colidx):
    return {(i, int(colidx[k])) for i in range(len(rowptr) - 1) for k in range(rowptr[i], rowptr[i + 1])}


@pytest.mark.parametrize("eta", [0.5, 1.0, 1.25, 2.0])
def test_one_dimensional_point_set_definition(eta):
    # On the line a bounding box is the interval spanned by the cluster's points, so box
    # diam/dist equal the point-set diam/dist of Eq. (cutoff): brute force over points.
    rng = np.random.Generator(np.random.PCG64(int(eta * 100)))
    x = np.sort(rng.random(200))[:, None]
    cl = build_tree(x, 4)
    B = samplet_basis(x, cl, 1)
    rowptr, colidx = eta_pattern(cl, B.bsize, eta)
    got = _pairs(rowptr, colidx)
    want = set()
    for a in cl:
        for b in cl:
            if B.bsize[a.id] == 0 or B.bsize[b.id] == 0:
                continue
            pa, pb = x[a.idx, 0], x[b.idx, 0]
            dist = np.abs(pa[:, None] - pb[None, :]).min()
            diam = max(pa.max() - pa.min(), pb.max() - pb.min())
            if not dist >= eta * diam:          # admissible pairs are dropped
                want.add((a.id, b.id))
    assert got == want


def test_pattern_invariants():
    rng = np.random.Generator(np.random.PCG64(9))
    x = rng.random((2000, 3))
    cl = build_tree(x, 32)
    B = samplet_basis(x, cl, 3)
    rowptr, colidx = eta_pattern(cl, B.bsize, 1.0)
    P = _pairs(rowptr, colidx)
    assert all((j, i) in P for (i, j) in P)                              # symmetric
    assert all((c.id, c.id) in P for c in cl if B.bsize[c.id] > 0)       # diagonal kept
    assert all((0, c.id) in P for c in cl if B.bsize[c.id] > 0)          # root row full
    for i in range(len(cl)):
        assert np.all(np.diff(colidx[rowptr[i]:rowptr[i + 1]]) > 0)      # sorted
    # admissibility is inherited by sons (boxes of sons lie inside the parent's):
    # a kept pair of sons has a kept pair of parents
    for (i, j) in P:
        pi, pj = cl[i].parent, cl[j].parent
        if pi >= 0 and pj >= 0 and B.bsize[pi] > 0 and B.bsize[pj] > 0:
            assert (pi, pj) in P
    full_r, full_c = eta_pattern(cl, B.bsize, np.inf)
    nz = int(np.sum(B.bsize > 0))
    assert len(full_c) == nz * nz
