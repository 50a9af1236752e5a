"""Cluster tree and bounding boxes (Sec. 3.2, Def. cluster-tree and the bounding-box
lemma).  Test infrastructure only (see ``oracle/__init__``).

Readings of the paper (it asks only for a balanced binary tree):
  * a cluster with more than ``leaf`` points is split; one with ``leaf`` or fewer is a leaf;
  * the split direction is the longest edge of the cluster's bounding box (lowest axis on
    ties); the points are ordered by that coordinate, ties by original index, and the
    first floor(|nu|/2) go to the first son;
  * clusters are numbered breadth first: level by level, first son before second son;
  * the point list of an internal cluster is its first son's list followed by its
    second son's list, so a son's weights sit in a contiguous slice of the parent's.
"""
import numpy as np


class Cluster:
    __slots__ = ("idx", "level", "parent", "sons", "bmin", "bmax", "id")

    def __init__(self, idx, level, parent):
        self.idx = idx          # original point indices, in this cluster's point order
        self.level = level
        self.parent = parent
        self.sons = []
        self.bmin = None
        self.bmax = None
        self.id = -1


def build_tree(points, leaf):
    """Return the list of clusters in breadth-first order.

    Each cluster carries its original point indices ``idx`` (point order as stated in the
    module docstring), ``level``, ``parent`` id, ``sons`` ids and bounding box
    ``bmin``/``bmax`` (the smallest axis-parallel box holding its points).
    """
    x = np.asarray(points, dtype=np.float64)
    n = x.shape[0]
    root = Cluster(np.arange(n, dtype=np.int64), 0, -1)
    order = [root]
    head = 0
    while head < len(order):
        c = order[head]
        c.id = head
        head += 1
        pts = x[c.idx]
        c.bmin = pts.min(axis=0)
        c.bmax = pts.max(axis=0)
        if len(c.idx) > leaf:
            edge = c.bmax - c.bmin
            dim = int(np.argmax(edge))            # first maximal axis
            perm = np.lexsort((c.idx, pts[:, dim]))  # by coordinate, ties by index
            srt = c.idx[perm]
            h = len(srt) // 2
            for part in (srt[:h], srt[h:]):
                s = Cluster(part, c.level + 1, c.id)
                order.append(s)
    for c in order:
        if c.parent >= 0:
            order[c.parent].sons.append(c.id)
    # point list of an internal cluster: sons' lists concatenated (first son first)
    for c in reversed(order):
        if c.sons:
            c.idx = np.concatenate([order[s].idx for s in c.sons])
    return order


def bbox_diam(c):
    """diam(nu): length of the diagonal of the bounding box."""
    return float(np.sqrt(np.sum((c.bmax - c.bmin) ** 2)))


def bbox_dist(c1, c2):
    """dist(nu, nu'): Euclidean distance between the two bounding boxes."""
    gap = np.maximum(0.0, np.maximum(c1.bmin - c2.bmax, c2.bmin - c1.bmax))
    return float(np.sqrt(np.sum(gap * gap)))
