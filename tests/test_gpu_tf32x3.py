"""GPU parity of the split-TF32 tensor-core product (S_TF32X3, tcgen05) against the FP64
oracle, through the C ABI: forward and adjoint, general patterns, ragged and wide blocks
(several 32-row / 32-column slices and 24-wide lambda slices), symmetric reads.

Tolerances: each product keeps hi*hi + hi*lo + lo*hi of TF32-rounded parts, so the dropped
terms are below 3 * 2^-22 |x y| with random signs, and the sums accumulate in fp32.  On the
kernel-matrix pattern (N = 4096, sums of O(10^3) terms without strong cancellation) that is
the mixed-precision target 1e-6; uniform [-1, 1] values on random patterns cancel about
tenfold, hence the float-class bound 1e-5 used for the other float kernels there."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import product as oprod
from oracle.pipeline import compress_kernel
from tests.gpu_util import dev, host, pattern_of, rel_frob
from tests.test_gpu_product import drop_empty
from tests.test_oracle_product import random_bcsr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_11681_gb300 import sformat
    return sformat


@pytest.fixture(scope="module")
def c1():
    w = W.WORKLOADS["matern32_2d_4096"]
    c = compress_kernel(W.points(w), w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, w.scale, w.nugget)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    return c, levels


def test_c1_tf32x3(sf, c1):
    c, levels = c1
    A = c.A
    P = pattern_of(A, levels)
    want = oprod.mul_masked(A, A, A, nthreads=8).val
    dA = dev(A.val, "float32")
    for sym in (False, True):
        p = sf.Plan(P, P, P, "tf32x3")
        p.set_symmetric_a(sym)
        out = dev(np.full(len(A.val), np.nan), "float32")
        p.mul(dA, dA, out)
        got = host(out)
        assert np.isfinite(got).all()
        assert rel_frob(got, want) <= 1e-6, sym
        # the same plan again gives the same bits
        out2 = dev(np.zeros(len(A.val)), "float32")
        p.mul(dA, dA, out2)
        np.testing.assert_array_equal(host(out2), got)


@pytest.mark.parametrize("seed,bmax,n", [(1, 46, 30), (2, 46, 30), (3, 46, 30), (4, 97, 12)])
def test_tf32x3_general_patterns(sf, seed, bmax, n):
    # S_A != S_B != S_C, empty clusters, odd block sizes (4-byte copies), blocks wider than one
    # 32-wide panel slice and than one 24-wide lambda slice, up to the 96 limit
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = rng.integers(0, bmax, size=n)
    bsize[rng.integers(0, n, size=2)] = 0
    A = drop_empty(random_bcsr(bsize, 0.35, seed * 10))
    B = drop_empty(random_bcsr(bsize, 0.35, seed * 20, diag=False))
    Cp = drop_empty(random_bcsr(bsize, 0.4, seed * 30, diag=False))
    want = oprod.mul_masked(A, B, Cp).val
    pa, pb, pc = pattern_of(A), pattern_of(B), pattern_of(Cp)
    plan = sf.Plan(pa, pb, pc, "tf32x3")
    out = dev(np.full(len(Cp.val), np.nan), "float32")
    plan.mul(dev(A.val, "float32"), dev(B.val, "float32"), out)
    assert rel_frob(host(out), want) <= 1e-5
    dC = Cp.like(W.random_values(len(Cp.val), seed + 7))
    gA = dev(np.full(len(A.val), np.nan), "float32")
    gB = dev(np.full(len(B.val), np.nan), "float32")
    plan.adjoint(dev(dC.val, "float32"), dev(A.val, "float32"), dev(B.val, "float32"), gA, gB)
    wA, wB = oadj.mul_masked_adjoint(dC, A, B)
    assert rel_frob(host(gA), wA.val) <= 1e-5
    assert rel_frob(host(gB), wB.val) <= 1e-5


def test_tf32x3_limits(sf, c1):
    # blocks wider than 96 are refused at plan creation
    A = random_bcsr(np.array([97, 4, 6]), 1.0, 3)
    p = pattern_of(A)
    with pytest.raises(sf.SFormatError) as e:
        sf.Plan(p, p, p, "tf32x3")
    assert e.value.status == sf.S_ERR_ARG
    # a symmetric plan must be called with B = A
    c, levels = c1
    P = pattern_of(c.A, levels)
    plan = sf.Plan(P, P, P, "tf32x3")
    plan.set_symmetric_a(True)
    x = dev(c.A.val, "float32")
    y = dev(c.A.val, "float32")
    with pytest.raises(sf.SFormatError) as e2:
        plan.mul(x, y, dev(np.zeros(len(c.A.val)), "float32"))
    assert e2.value.status == sf.S_ERR_ARG
