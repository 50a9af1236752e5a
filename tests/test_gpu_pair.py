"""A product of two different kernel matrices on three different patterns of one cluster
tree, C = P_{S_C}(K_A K_B) (Eq. (product) for general S_A, S_B, S_C, Thm. (product)):
K_A Matern-3/2 (ell = 0.2) on the eta = 1.25 pattern, K_B Matern-5/2 (ell = 0.1) on the
eta = 1.0 pattern, S_C the eta = 0.8 pattern; N = 4096 points in [0,1]^2, q = 2, leaf 16.

Parity against the FP64 oracle on shared inputs (oracle-built values uploaded): FP64 and
double-float within 1e-12 relative Frobenius, compensated float within 1e-6 (every kernel
shape), the adjoint in FP64 within 1e-12.  Then the same pipeline end to end from the
device builder (three builders on the same points give the same tree), checked against the
oracle product of the downloaded device values."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import product as oprod
from oracle.pattern import eta_pattern
from oracle.pipeline import compress_kernel
from oracle.sformat import BlockCSR
from tests.gpu_util import dev, host, pattern_of, rel_frob

pytestmark = pytest.mark.gpu
S = W.PAIR_2D


def points():
    w = W.Workload("pair", S["seed"], S["n"], S["d"], "cube", 0.0, 0.0, 0.0, S["q"], S["leaf"], 0.0, 0.0)
    return W.points(w)


@pytest.fixture(scope="module")
def pair():
    x = points()
    n = len(x)
    (nua, la, ea), (nub, lb, eb) = S["a"], S["b"]
    ca = compress_kernel(x, nua, la, S["q"], S["leaf"], ea, 0.0, 1.0 / n, S["nugget"])
    cb = compress_kernel(x, nub, lb, S["q"], S["leaf"], eb, 0.0, 1.0 / n, S["nugget"])
    rp, ci = eta_pattern(ca.clusters, ca.basis.bsize, S["c_eta"])
    Cp = BlockCSR(ca.A.bsize, rp, ci)
    levels = np.array([cl.level for cl in ca.clusters], dtype=np.int32)
    return ca.A, cb.A, Cp, levels


def test_three_different_patterns(pair):
    A, B, Cp, _ = pair
    sets = [{(int(X.brow[k]), int(X.colidx[k])) for k in range(X.nblocks)} for X in (A, B, Cp)]
    assert sets[2] < sets[1] < sets[0]          # smaller eta: fewer pairs, nested
    assert not np.allclose(A.val[:10], B.val[:10])


def test_pair_product_parity(pair):
    from paper_2211_11681_gb300 import sformat as sf
    A, B, Cp, levels = pair
    pa, pb, pc = (pattern_of(X, levels) for X in (A, B, Cp))
    want = oprod.mul_masked(A, B, Cp, nthreads=8).val
    for prec, dt, tol in (("fp64", "float64", 1e-12), ("fp64_df", "float64", 1e-12)):
        plan = sf.Plan(pa, pb, pc, prec)
        assert plan.stats() == oprod.mul_count(A, B, Cp)
        out = dev(np.full(len(Cp.val), np.nan), dt)
        plan.mul(dev(A.val, dt), dev(B.val, dt), out)
        assert rel_frob(host(out), want) <= tol, prec
    plan = sf.Plan(pa, pb, pc, "fp32")
    for v in range(plan.num_variants()):
        plan.set_variant(v)
        out = dev(np.full(len(Cp.val), np.nan), "float32")
        plan.mul(dev(A.val, "float32"), dev(B.val, "float32"), out)
        assert rel_frob(host(out), want) <= 1e-6, v
    # reverse mode on the three patterns
    dC = Cp.like(W.random_values(len(Cp.val), 17))
    wA, wB = oadj.mul_masked_adjoint(dC, A, B)
    p64 = sf.Plan(pa, pb, pc, "fp64")
    gA, gB = dev(np.zeros(len(A.val))), dev(np.zeros(len(B.val)))
    p64.adjoint(dev(dC.val), dev(A.val), dev(B.val), gA, gB)
    assert rel_frob(host(gA), wA.val) <= 1e-12
    assert rel_frob(host(gB), wB.val) <= 1e-12


def test_pair_pipeline_from_the_device_builder():
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    x = points()
    n = len(x)
    (nua, la, ea), (nub, lb, eb) = S["a"], S["b"]
    ba = Builder(x, S["leaf"], S["q"], ea)
    bb = Builder(x, S["leaf"], S["q"], eb)
    bc = Builder(x, S["leaf"], S["q"], S["c_eta"])
    np.testing.assert_array_equal(ba.block_offset, bc.block_offset)
    pa, va = ba.values(nua, la, 1.0 / n, S["nugget"], 0.0)
    pb, vb = bb.values(nub, lb, 1.0 / n, S["nugget"], 0.0)
    pc = sf.Pattern(bc.block_offset, bc.level, bc.rowptr, bc.colidx)
    plan = sf.Plan(pa, pb, pc, "fp64")
    out = dev(np.full(pc.nnz, np.nan))
    plan.mul(va, vb, out)
    bs = np.diff(ba.block_offset)
    A = BlockCSR(bs, ba.rowptr, ba.colidx.astype(np.int64), host(va))
    B = BlockCSR(bs, bb.rowptr, bb.colidx.astype(np.int64), host(vb))
    Cp = BlockCSR(bs, bc.rowptr, bc.colidx.astype(np.int64))
    want = oprod.mul_masked(A, B, Cp, nthreads=8).val
    assert rel_frob(host(out), want) <= 1e-12
    p32 = sf.Plan(pa, pb, pc, "fp32")
    o32 = dev(np.full(pc.nnz, np.nan), "float32")
    p32.mul(va.float(), vb.float(), o32)
    assert rel_frob(host(o32), want) <= 1e-6
