"""Selected inversion (Sec. 4.2, Eq. (blockInv)) and the contour-integral inverse square root
(Sec. 4.4, Eq. (ContInt)) on the GPU, through the C ABI, against the FP64 CPU oracle:

  * random symmetric block patterns with empty and ragged clusters, blocks up to 64 wide
    (output blocks split into several 512-entry work items), a single cluster, a full
    pattern (the factor a chain of supernodes);
  * the compressed exponential kernel matrix of the paper's benchmarks (uniform [0,1]^2,
    exp(-r)/N, q+1 = 4 vanishing moments, eta = 1.25, tau = 1e-5/N) plus a ridge mu I;
  * out = alpha P_S(Z) + beta out, the not-positive-definite record, the width limit;
  * Eq. (ContInt) with n = 7 nodes on the kernel matrix.

Tolerances.  Both sides are FP64 solves of the same matrix; their difference is bounded by
the condition number times a modest multiple of the unit roundoff: 1e-12 relative
(maximum entry) on the shifted random matrices (condition number at most 2R + 1, a few
hundred here),
1e-11 relative Frobenius at mu = 1e-2 (condition number about 1e2) and 1e-9 at mu = 1e-4
(about 1e4); the quadrature sums seven such inverses with positive weights: 1e-9."""
import numpy as np
import pytest

import workloads as W
from oracle import contour as ocon
from oracle import selinv as osel
from oracle.pipeline import compress_kernel
from oracle.sformat import BlockCSR
from tests.gpu_util import dev, host, pattern_of, rel_frob
from tests.test_gpu_product import drop_empty
from tests.test_selinv_host import symmetric_pattern

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_11681_gb300 import selinv, sformat
    return sformat, selinv


def random_spd(bsize, density, seed):
    """Symmetric values on a symmetric random pattern, and a shift sigma = R + 1, R the largest
    absolute row sum, so that the spectrum of A + sigma I lies in [1, 2R + 1] (Gershgorin)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rowptr, colidx, _ = symmetric_pattern(len(bsize), density, seed)
    A = BlockCSR(bsize, rowptr, colidx)
    A.val[:] = rng.uniform(-1.0, 1.0, len(A.val))
    D = A.to_dense()
    A = drop_empty(BlockCSR.from_dense(D + D.T, bsize, rowptr, colidx))   # no blocks of empty clusters
    sigma = float(np.abs(A.to_dense()).sum(axis=1).max()) + 1.0
    return A, sigma


def run(mods, A, sigma):
    sf, si = mods
    P = pattern_of(A)
    inv = si.SelInv(P)
    Z = dev(np.full(len(A.val), np.nan))
    inv.factor(dev(A.val), sigma)
    inv.invert(Z)
    inv.status()
    return inv, P, host(Z)


def max_rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_patterns(mods, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = rng.integers(0, 8, size=30)
    A, sigma = random_spd(bsize, 0.15, seed)
    inv, _, Z = run(mods, A, sigma)
    want = osel.selected_inverse(A, sigma).val
    assert max_rel(Z, want) <= 1e-12
    st = inv.stats()
    perm, nl, levels = mods[1].order(A.bsize, A.rowptr, A.colidx)
    assert st["l_blocks"] == nl and st["levels"] == levels
    assert st["flops_factor"] > 0 and st["flops_invert"] > 0


def test_wide_blocks_and_tiles(mods):
    bsize = np.array([64, 1, 40, 0, 23, 64, 7, 33, 2, 48])
    A, sigma = random_spd(bsize, 0.35, 11)
    _, _, Z = run(mods, A, sigma)
    assert max_rel(Z, osel.selected_inverse(A, sigma).val) <= 1e-12


def test_single_cluster_and_full_pattern(mods):
    A, sigma = random_spd(np.array([12]), 1.0, 5)
    _, _, Z = run(mods, A, sigma)
    assert max_rel(Z, osel.selected_inverse(A, sigma).val) <= 1e-12
    bsize = np.array([5, 3, 6, 4, 2, 5, 1, 6])
    A, sigma = random_spd(bsize, 1.0, 6)                  # every cluster pair: a dense chain
    inv, _, Z = run(mods, A, sigma)
    assert inv.stats()["levels"] == len(bsize)
    assert max_rel(Z, osel.selected_inverse(A, sigma).val) <= 1e-12


def test_alpha_beta_accumulation(mods):
    rng = np.random.Generator(np.random.PCG64(8))
    bsize = rng.integers(1, 6, size=20)
    A, sigma = random_spd(bsize, 0.2, 8)
    sf, si = mods
    inv = si.SelInv(pattern_of(A))
    prev = W.random_values(len(A.val), 3)
    out = dev(prev)
    inv.factor(dev(A.val), sigma)
    inv.invert(out, alpha=2.0, beta=0.5)
    inv.status()
    want = 2.0 * osel.selected_inverse(A, sigma).val + 0.5 * prev
    assert max_rel(host(out), want) <= 1e-12


def test_not_positive_definite_is_reported(mods):
    sf, si = mods
    bsize = np.array([3, 4, 2])
    A, _ = random_spd(bsize, 0.5, 4)
    inv = si.SelInv(pattern_of(A))
    inv.factor(dev(-A.identity_like().val), 0.0)        # -I: the first pivot is -1
    with pytest.raises(sf.SFormatError) as e:
        inv.status()
    assert e.value.status == sf.S_ERR_NOT_SPD
    inv.status()                                         # reported once, then cleared
    A2, sigma = random_spd(bsize, 0.5, 4)
    Z = dev(np.zeros(len(A2.val)))
    inv.factor(dev(A2.val), sigma)                       # the plan stays usable
    inv.invert(Z)
    inv.status()
    assert max_rel(host(Z), osel.selected_inverse(A2, sigma).val) <= 1e-12


def test_blocks_wider_than_64_are_refused(mods):
    sf, si = mods
    A, _ = random_spd(np.array([65, 3]), 1.0, 2)
    with pytest.raises(sf.SFormatError) as e:
        si.SelInv(pattern_of(A))
    assert e.value.status == sf.S_ERR_ARG


@pytest.fixture(scope="module")
def kmat():
    w = W.WORKLOADS["paper_mult_2d"]
    n = 2048
    c = compress_kernel(W.points(w, n), w.nu, w.ell, w.q, w.leaf, w.eta, W.tau_of(w, n), 1.0 / n, 0.0)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    return c.A, levels


@pytest.mark.parametrize("mu,tol", [(1e-2, 1e-11), (1e-4, 1e-9)])
def test_kernel_matrix_with_ridge(mods, kmat, mu, tol):
    A, levels = kmat
    sf, si = mods
    inv = si.SelInv(pattern_of(A, levels))
    Z = dev(np.zeros(len(A.val)))
    inv.factor(dev(A.val), mu)
    inv.invert(Z)
    inv.status()
    assert rel_frob(host(Z), osel.selected_inverse(A, mu).val) <= tol


def test_contour_inverse_square_root(mods, kmat):
    A, levels = kmat
    sf, si = mods
    mu = 1e-4
    B = A.like(A.val + A.identity_like(mu).val)          # K + mu I on S
    inv = si.SelInv(pattern_of(A, levels))
    Z = dev(np.zeros(len(A.val)))
    inv.invsqrt(dev(B.val), mu, 1.0, 7, Z)
    want = ocon.invsqrt(B, mu, 1.0, 7).val
    assert rel_frob(host(Z), want) <= 1e-9
