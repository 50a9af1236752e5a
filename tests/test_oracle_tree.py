"""Pins of the oracle's cluster tree (Def. cluster-tree, bounding-box lemma, Sec. 3.2)."""
import numpy as np
import pytest

import workloads as W
from oracle.tree import bbox_diam, bbox_dist, build_tree


@pytest.mark.parametrize("n,d,leaf", [(1000, 2, 16), (777, 3, 32), (64, 1, 1), (5, 2, 16)])
def test_tree_invariants(n, d, leaf):
    rng = np.random.Generator(np.random.PCG64(n))
    x = rng.random((n, d))
    cl = build_tree(x, leaf)
    assert sorted(cl[0].idx.tolist()) == list(range(n))
    for c in cl:
        pts = x[c.idx]
        np.testing.assert_array_equal(c.bmin, pts.min(axis=0))
        np.testing.assert_array_equal(c.bmax, pts.max(axis=0))
        if c.sons:
            a, b = (cl[s] for s in c.sons)
            # disjoint union, balanced, point list = sons' lists concatenated
            assert len(a.idx) == len(c.idx) // 2 and len(a.idx) + len(b.idx) == len(c.idx)
            np.testing.assert_array_equal(np.concatenate([a.idx, b.idx]), c.idx)
            assert a.level == b.level == c.level + 1
            # split along the longest edge: the sons are separated along that axis
            ax = int(np.argmax(c.bmax - c.bmin))
            assert x[a.idx, ax].max() <= x[b.idx, ax].min()
            assert len(c.idx) > leaf
        else:
            assert len(c.idx) <= leaf or n <= leaf
    # breadth-first numbering
    levels = [c.level for c in cl]
    assert levels == sorted(levels)


def test_box_geometry():
    class B:
        pass
    a, b = B(), B()
    a.bmin, a.bmax = np.array([0.0, 0.0]), np.array([1.0, 2.0])
    b.bmin, b.bmax = np.array([4.0, 6.0]), np.array([5.0, 7.0])
    assert bbox_diam(a) == pytest.approx(np.sqrt(5.0))
    assert bbox_dist(a, b) == pytest.approx(5.0)   # gaps 3 and 4
    assert bbox_dist(a, a) == 0.0


def test_workload_points_are_seeded():
    w = W.WORKLOADS["matern52_sphere"]
    p1 = W.points(w, 100)
    p2 = W.points(w, 100)
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_allclose(np.linalg.norm(p1, axis=1), 1.0, rtol=1e-14)
