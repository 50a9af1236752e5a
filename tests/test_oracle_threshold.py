"""Pins of the oracle's a-posteriori threshold (Sec. 5 drops the entries below tau; the
block store keeps a block iff it is diagonal or holds an entry at or above tau, decided on
the unordered pair {(nu, nu'), (nu', nu)}, and zeroes the sub-tau entries of kept blocks).

The matrices are written out by hand, so every kept block and every zeroed entry is known
without running the oracle.  Each case is built to fail under one plausible slip:
  * a decision on the ordered block only (the two halves of a pair straddle tau);
  * ">" written for ">=" (an entry equals tau exactly);
  * a dropped diagonal rule (a diagonal block lies entirely below tau);
  * entries below tau left in a kept block.
"""
import numpy as np

from oracle.sformat import compress

TAU = 1.0
BSIZE = np.array([2, 2, 2, 2])
BOFF = np.array([0, 2, 4, 6, 8])


def _full_pattern(nc):
    rowptr = np.arange(nc + 1, dtype=np.int64) * nc
    colidx = np.tile(np.arange(nc, dtype=np.int64), nc)
    return rowptr, colidx


def _set_block(K, i, j, blk):
    K[BOFF[i]:BOFF[i + 1], BOFF[j]:BOFF[j + 1]] = blk


def _khat():
    K = np.zeros((8, 8))
    # diagonal blocks: 0, 1 and 3 hold large entries; block (2,2) lies entirely below tau
    _set_block(K, 0, 0, [[5.0, 0.25], [0.25, 4.0]])
    _set_block(K, 1, 1, [[3.0, 0.0], [0.0, 3.0]])
    _set_block(K, 2, 2, [[0.5, 0.125], [0.125, 0.75]])
    _set_block(K, 3, 3, [[2.0, 1.5], [1.5, 2.0]])
    # pair {0,1}: symmetric up to rounding, the two halves straddle tau
    _set_block(K, 0, 1, [[1.0 + 2e-16, 0.5], [0.25, 0.125]])
    _set_block(K, 1, 0, [[1.0 - 2e-16, 0.25], [0.5, 0.125]])
    # pair {0,2}: one entry equals tau exactly (kept, since the rule is >=)
    _set_block(K, 0, 2, [[0.0, TAU], [0.5, 0.0]])
    _set_block(K, 2, 0, [[0.0, 0.5], [TAU, 0.0]])
    # pair {1,3}: every entry below tau (dropped)
    _set_block(K, 1, 3, [[0.5, 0.9], [0.25, 0.75]])
    _set_block(K, 3, 1, [[0.5, 0.25], [0.9, 0.75]])
    # pairs {0,3}, {1,2}, {2,3}: zero (dropped)
    return K


def _kept(A):
    return {(int(A.brow[k]), int(A.colidx[k])) for k in range(A.nblocks)}


def test_kept_blocks_decided_on_the_unordered_pair():
    rowptr, colidx = _full_pattern(4)
    A = compress(_khat(), BSIZE, rowptr, colidx, TAU)
    want = {(0, 0), (1, 1), (2, 2), (3, 3), (0, 1), (1, 0), (0, 2), (2, 0)}
    assert _kept(A) == want
    # the kept pattern is symmetric
    assert {(j, i) for (i, j) in _kept(A)} == _kept(A)


def test_sub_tau_entries_of_kept_blocks_are_zero():
    rowptr, colidx = _full_pattern(4)
    K = _khat()
    A = compress(K, BSIZE, rowptr, colidx, TAU)
    D = A.to_dense()
    # written out: every entry whose pair magnitude is below tau is zero, the rest unchanged
    want = np.zeros((8, 8))
    want[0, 0], want[1, 1] = 5.0, 4.0
    want[2, 2], want[3, 3] = 3.0, 3.0
    want[6:8, 6:8] = [[2.0, 1.5], [1.5, 2.0]]
    want[0, 2], want[2, 0] = 1.0 + 2e-16, 1.0 - 2e-16
    want[0, 5], want[5, 0] = TAU, TAU
    assert np.array_equal(D, want)
    # the below-tau diagonal block is kept as a block of zeros
    k = A.find(2, 2)
    assert k >= 0 and not np.any(A.block(k))


def test_tau_zero_keeps_the_whole_eta_pattern():
    rowptr, colidx = _full_pattern(4)
    K = _khat()
    A = compress(K, BSIZE, rowptr, colidx, 0.0)
    assert A.nblocks == 16
    assert np.array_equal(A.to_dense(), K)
