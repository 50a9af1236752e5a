"""GPU parity of the masked product (Eq. (product)), its adjoint, S-format addition and the
norm estimate against the FP64 CPU oracle, through the C ABI, in double, double-float
(S_FP64_DF) and compensated float arithmetic.

Tolerances: FP64 results agree with the oracle to 1e-12 relative Frobenius error (the
summation order differs, each entry is a sum of at most a few thousand products of
O(1)-conditioned terms, so rounding stays near 1e-15 x sqrt(terms)); the FP32 product is
checked at 1e-5 (float rounding 6e-8 per operation times sqrt of the longest sum)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import funm as ofunm
from oracle import product as oprod
from oracle.pipeline import compress_kernel
from tests.gpu_util import dev, host, pattern_of, rel_frob
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
    x = W.points(w)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, w.scale, w.nugget)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    return c, levels


def test_c1_fp64_parity(sf, c1):
    c, levels = c1
    A = c.A
    P = pattern_of(A, levels)
    assert P.nnz == len(A.val) and P.nblocks == A.nblocks
    np.testing.assert_array_equal(P.block_offsets(), A.voff)
    plan = sf.Plan(P, P, P, "fp64")
    t, f = plan.stats()
    assert (t, f) == oprod.mul_count(A, A, A)
    assert plan.variant()["tile"] == 10            # 6- and 10-wide blocks: the 10-wide tiles
    dA = dev(A.val)
    dC = dev(np.full(len(A.val), np.nan))
    plan.mul(dA, dA, dC)
    want = oprod.mul_masked(A, A, A, nthreads=8).val
    got = host(dC)
    assert rel_frob(got, want) <= 1e-12
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # deterministic: a second run gives the same bits
    dC2 = dev(np.zeros(len(A.val)))
    plan.mul(dA, dA, dC2)
    np.testing.assert_array_equal(host(dC2), got)
    # double-float arithmetic (float pairs, ~2^-44 per term) meets the double bound too
    pdf = sf.Plan(P, P, P, "fp64_df")
    assert pdf.stats() == (t, f)
    dD = dev(np.full(len(A.val), np.nan))
    pdf.mul(dA, dA, dD)
    assert rel_frob(host(dD), want) <= 1e-12


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_general_patterns_and_ragged_tiles(sf, seed):
    # S_A != S_B != S_C, empty clusters, blocks wider than one 20x20 tile
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = rng.integers(0, 46, size=30)
    bsize[rng.integers(0, 30, size=3)] = 0
    A = random_bcsr(bsize, 0.3, seed * 10)
    B = random_bcsr(bsize, 0.35, seed * 20, diag=False)
    Cp = random_bcsr(bsize, 0.4, seed * 30, diag=False)
    # blocks touching empty clusters are not allowed in a pattern: drop them
    A, B, Cp = (drop_empty(X) for X in (A, B, Cp))
    pa, pb, pc = pattern_of(A), pattern_of(B), pattern_of(Cp)
    plan = sf.Plan(pa, pb, pc, "fp64")
    assert plan.stats() == oprod.mul_count(A, B, Cp)
    want = oprod.mul_masked(A, B, Cp).val
    for v in range(plan.num_variants()):       # tile edges 20 and 10
        plan.set_variant(v)
        out = dev(np.full(len(Cp.val), np.nan))
        plan.mul(dev(A.val), dev(B.val), out)
        assert rel_frob(host(out), want) <= 1e-12, v
    # FP32 arithmetic on the same values
    p32 = sf.Plan(pa, pb, pc, "fp32")
    o32 = dev(np.zeros(len(Cp.val)), "float32")
    p32.mul(dev(A.val, "float32"), dev(B.val, "float32"), o32)
    assert rel_frob(host(o32), want) <= 1e-5
    # double-float arithmetic, every kernel shape, forward and adjoint
    pdf = sf.Plan(pa, pb, pc, "fp64_df")
    for v in range(pdf.num_variants()):
        pdf.set_variant(v)
        odf = dev(np.full(len(Cp.val), np.nan))
        pdf.mul(dev(A.val), dev(B.val), odf)
        assert rel_frob(host(odf), want) <= 1e-12, v
    # adjoint
    dC = Cp.like(W.random_values(len(Cp.val), seed + 99))
    gA, gB = dev(np.zeros(len(A.val))), dev(np.zeros(len(B.val)))
    plan.adjoint(dev(dC.val), dev(A.val), dev(B.val), gA, gB)
    wA, wB = oadj.mul_masked_adjoint(dC, A, B)
    assert rel_frob(host(gA), wA.val) <= 1e-12
    assert rel_frob(host(gB), wB.val) <= 1e-12
    hA, hB = dev(np.zeros(len(A.val))), dev(np.zeros(len(B.val)))
    pdf.adjoint(dev(dC.val), dev(A.val), dev(B.val), hA, hB)
    assert rel_frob(host(hA), wA.val) <= 1e-12
    assert rel_frob(host(hB), wB.val) <= 1e-12


@pytest.mark.parametrize("seed", [5, 6])
def test_bf16x3_general_even_patterns(sf, seed):
    # even block sizes up to 44 (tiles and lambda slices with ragged ends, 4- and 8-byte copies);
    # uniform [-1, 1] values cancel about tenfold in these sums, so the float-class bound
    # of the random-pattern tests (1e-5) applies, as for the compensated float kernel
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = 2 * rng.integers(0, 23, size=28)
    A = drop_empty(random_bcsr(bsize, 0.35, seed * 10))
    B = drop_empty(random_bcsr(bsize, 0.35, seed * 20, diag=False))
    Cp = drop_empty(random_bcsr(bsize, 0.4, seed * 30, diag=False))
    want = oprod.mul_masked(A, B, Cp).val
    pa, pb, pc = pattern_of(A), pattern_of(B), pattern_of(Cp)
    plan = sf.Plan(pa, pb, pc, "bf16x3")
    out = dev(np.full(len(Cp.val), np.nan), "float32")
    plan.mul(dev(A.val, "float32"), dev(B.val, "float32"), out)
    assert rel_frob(host(out), want) <= 1e-5
    dC = Cp.like(W.random_values(len(Cp.val), seed + 7))
    gA, gB = dev(np.zeros(len(A.val)), "float32"), dev(np.zeros(len(B.val)), "float32")
    plan.adjoint(dev(dC.val, "float32"), dev(A.val, "float32"), dev(B.val, "float32"), gA, gB)
    wA, wB = oadj.mul_masked_adjoint(dC, A, B)
    assert rel_frob(host(gA), wA.val) <= 1e-5
    assert rel_frob(host(gB), wB.val) <= 1e-5


def test_bf16x3_rejects_odd_blocks(sf):
    A = random_bcsr(np.array([3, 4, 6]), 1.0, 3)
    p = pattern_of(A)
    with pytest.raises(sf.SFormatError) as e:
        sf.Plan(p, p, p, "bf16x3")
    assert e.value.status == sf.S_ERR_ARG


def drop_empty(X):
    from oracle.sformat import BlockCSR
    keep_rows, cols = [0], []
    for i in range(X.nclusters):
        for k in range(X.rowptr[i], X.rowptr[i + 1]):
            j = X.colidx[k]
            if X.bsize[i] > 0 and X.bsize[j] > 0:
                cols.append(j)
        keep_rows.append(len(cols))
    Y = BlockCSR(X.bsize, np.array(keep_rows), np.array(cols, dtype=np.int64))
    for k in range(Y.nblocks):
        kk = X.find(Y.brow[k], Y.colidx[k])
        Y.val[Y.voff[k]:Y.voff[k + 1]] = X.block(kk).ravel()
    return Y


def test_c1_fp32_error_and_add(sf, c1):
    c, levels = c1
    A = c.A
    P = pattern_of(A, levels)
    # split-bfloat16 tensor-core product (six cross products of three bf16 planes)
    want0 = oprod.mul_masked(A, A, A, nthreads=8).val
    for sym in (False, True):
        pb = sf.Plan(P, P, P, "bf16x3")
        pb.set_symmetric_a(sym)
        ob = dev(np.full(len(A.val), np.nan), "float32")
        pb.mul(dev(A.val, "float32"), dev(A.val, "float32"), ob)
        assert rel_frob(host(ob), want0) <= 1e-6
    plan = sf.Plan(P, P, P, "fp32")
    out = dev(np.zeros(len(A.val)), "float32")
    plan.mul(dev(A.val, "float32"), dev(A.val, "float32"), out)
    want = oprod.mul_masked(A, A, A, nthreads=8).val
    assert rel_frob(host(out), want) <= 1e-6          # the mixed-precision target
    # A is symmetric: reading A(nu, lambda) through the stored (lambda, nu) gives the same product
    for prec, tol in (("fp32", 1e-6), ("fp64", 1e-12)):
        ps = sf.Plan(P, P, P, prec)
        ps.set_symmetric_a(True)
        dt = "float32" if prec == "fp32" else "float64"
        o = dev(np.zeros(len(A.val)), dt)
        ps.mul(dev(A.val, dt), dev(A.val, dt), o)
        assert rel_frob(host(o), want) <= tol
    B = A.like(W.random_values(len(A.val), 5))
    C = dev(np.zeros(len(A.val)))
    sf.add(P, dev(A.val), dev(B.val), C, 0.75, -2.0, 0.5)
    np.testing.assert_allclose(host(C), ofunm.add(A, B, 0.75, -2.0, 0.5).val, rtol=1e-15, atol=1e-15)


def test_norm_estimate(sf, c1):
    c, levels = c1
    P = pattern_of(c.A, levels)
    lam = sf.norm_est(P, dev(c.A.val), 50)
    assert lam == pytest.approx(ofunm.norm_estimate(c.A), rel=1e-12)


def test_tree_mismatch_and_empty(sf, c1):
    c, levels = c1
    P = pattern_of(c.A, levels)
    Q = pattern_of(c.A, levels + 1)
    with pytest.raises(sf.SFormatError) as e:
        sf.Plan(P, Q, P)
    assert e.value.status == sf.S_ERR_MISMATCH
    # the symmetric flag checks the pattern
    from oracle.sformat import BlockCSR as _B
    asym = _B(c.A.bsize, np.array([0, 2] + [2] * (c.A.nclusters - 1)), np.array([0, 1]))
    pa = pattern_of(asym, levels)
    with pytest.raises(sf.SFormatError) as e2:
        sf.Plan(pa, pa, pa).set_symmetric_a(True)
    assert e2.value.status == sf.S_ERR_PATTERN
    # an empty output pattern is a valid, empty product
    from oracle.sformat import BlockCSR
    Z = BlockCSR(c.A.bsize, np.zeros(c.A.nclusters + 1, dtype=np.int64), np.zeros(0, dtype=np.int64))
    pz = pattern_of(Z, levels)
    plan = sf.Plan(P, P, pz)
    assert plan.stats() == (0, 0.0)
    d = dev(c.A.val)
    plan.mul(d, d, dev(np.zeros(1)))
