"""Compression pattern S by eta-admissibility (Sec. 3.3, Thm. (S-compression),
Eq. (cutoff)), over all cluster pairs of T x T including pairs on different levels.

Test infrastructure only (see ``oracle/__init__``).

Readings: diam and dist are those of bounding boxes (bounding-box lemma, Sec. 3.2);
clusters that own no rows are left out; a pair is kept (non-admissible) iff
dist < eta * max(diam, diam'), so eta = inf keeps every pair.
"""
import numpy as np


def eta_pattern(clusters, bsize, eta):
    """Return (rowptr, colidx) of the block pattern, columns sorted, by brute force over
    every pair of clusters."""
    nc = len(clusters)
    bmin = np.array([c.bmin for c in clusters])
    bmax = np.array([c.bmax for c in clusters])
    diam = np.sqrt(np.sum((bmax - bmin) ** 2, axis=1))
    rowptr = np.zeros(nc + 1, dtype=np.int64)
    cols = []
    for i in range(nc):
        if bsize[i] > 0:
            gap = np.maximum(0.0, np.maximum(bmin[i] - bmax, bmin - bmax[i]))
            dist = np.sqrt(np.sum(gap * gap, axis=1))
            keep = (bsize > 0) & (dist < eta * np.maximum(diam[i], diam))
            js = np.nonzero(keep)[0]
        else:
            js = np.zeros(0, dtype=np.int64)
        cols.append(js)
        rowptr[i + 1] = rowptr[i] + len(js)
    colidx = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    return rowptr, colidx.astype(np.int64)
