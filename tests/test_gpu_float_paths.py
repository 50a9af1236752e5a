"""GPU parity of the float paths against the FP64 CPU oracle, through the C ABI:

  * every float kernel shape of the autotuner, with A read as stored and through its
    transpose (s_plan_set_symmetric_a), on the benchmark's block shapes: N = 4096 points in
    [0,1]^3, Matern-1/2, ell = 0.1, q = 3 (20-wide interior blocks, up to 12-wide leaf
    blocks, a 40-wide root block), leaf 32, eta = 1.0, tau = 1e-8, kernel scaled by 1/N;
  * the float adjoint (s_mul_masked_adjoint with an S_FP32 plan) and float addition (s_add
    with S_FP32);
  * the time-out record of the split-TF32 and float plans, planted from the host (no device
    wait is made to run out).

Tolerances: 1e-6 relative Frobenius error on the compressed kernel matrices (the
compensated float kernel measures near 1e-7 there; inputs rounded to float alone give
~3e-8), 1e-5 on random values in [-1, 1] whose sums cancel about tenfold; float addition
within one float rounding of each term (6e-8 relative to the largest term)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import funm as ofunm
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
def c3d():
    w = W.WORKLOADS["matern12_3d_1m"]
    n = 4096
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, 1.0 / n, w.nugget)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    want = oprod.mul_masked(c.A, c.A, c.A, nthreads=8).val
    return c.A, levels, want


def test_block_shapes_of_the_workload(c3d):
    A, _, _ = c3d
    widths = set(int(b) for b in A.bsize)
    assert 20 in widths and max(widths) == 40 and min(w for w in widths if w > 0) < 20


@pytest.mark.parametrize("sym", [False, True])
def test_every_float_variant_on_20_wide_blocks(sf, c3d, sym):
    A, levels, want = c3d
    P = pattern_of(A, levels)
    plan = sf.Plan(P, P, P, "fp32")
    plan.set_symmetric_a(sym)
    dA = dev(A.val, "float32")
    for v in range(plan.num_variants()):
        plan.set_variant(v)
        out = dev(np.full(len(A.val), np.nan), "float32")
        plan.mul(dA, dA, out)
        assert rel_frob(host(out), want) <= 1e-6, (v, sym, plan.variant())
    # the autotuner's choice is one of them and stays selected
    shape = plan.autotune(dA, dA, dev(np.zeros(len(A.val)), "float32"))
    out = dev(np.full(len(A.val), np.nan), "float32")
    plan.mul(dA, dA, out)
    assert plan.variant() == shape
    assert rel_frob(host(out), want) <= 1e-6


def test_float_adjoint_on_kernel_matrix(sf, c3d):
    A, levels, _ = c3d
    P = pattern_of(A, levels)
    dC = A.like(A.val[::-1].copy())          # kernel-matrix magnitudes, no symmetry
    wA, wB = oadj.mul_masked_adjoint(dC, A, A)
    plan = sf.Plan(P, P, P, "fp32")
    gA, gB = dev(np.zeros(len(A.val)), "float32"), dev(np.zeros(len(A.val)), "float32")
    plan.adjoint(dev(dC.val, "float32"), dev(A.val, "float32"), dev(A.val, "float32"), gA, gB)
    assert rel_frob(host(gA), wA.val) <= 1e-6
    assert rel_frob(host(gB), wB.val) <= 1e-6


@pytest.mark.parametrize("seed", [7, 8])
def test_float_adjoint_general_patterns(sf, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = rng.integers(0, 46, size=30)
    A = drop_empty(random_bcsr(bsize, 0.3, seed * 10))
    B = drop_empty(random_bcsr(bsize, 0.35, seed * 20, diag=False))
    Cp = drop_empty(random_bcsr(bsize, 0.4, seed * 30, diag=False))
    dC = Cp.like(W.random_values(len(Cp.val), seed + 99))
    wA, wB = oadj.mul_masked_adjoint(dC, A, B)
    plan = sf.Plan(pattern_of(A), pattern_of(B), pattern_of(Cp), "fp32")
    gA, gB = dev(np.zeros(len(A.val)), "float32"), dev(np.zeros(len(B.val)), "float32")
    plan.adjoint(dev(dC.val, "float32"), dev(A.val, "float32"), dev(B.val, "float32"), gA, gB)
    assert rel_frob(host(gA), wA.val) <= 1e-5
    assert rel_frob(host(gB), wB.val) <= 1e-5
    # one side only
    hA = dev(np.zeros(len(A.val)), "float32")
    plan.adjoint(dev(dC.val, "float32"), None, dev(B.val, "float32"), hA, None)
    np.testing.assert_array_equal(host(hA), host(gA))


def test_float_add(sf, c3d):
    A, levels, _ = c3d
    P = pattern_of(A, levels)
    B = A.like(W.random_values(len(A.val), 5) * np.abs(A.val).max())
    a32, b32 = A.val.astype(np.float32).astype(np.float64), B.val.astype(np.float32).astype(np.float64)
    want = ofunm.add(A.like(a32), B.like(b32), 0.75, -2.0, 0.5).val
    C = dev(np.zeros(len(A.val)), "float32")
    sf.add(P, dev(A.val, "float32"), dev(B.val, "float32"), C, 0.75, -2.0, 0.5, prec="fp32")
    scale = 0.75 * np.abs(a32) + 2.0 * np.abs(b32) + 0.5
    assert np.all(np.abs(host(C) - want) <= 2 * 6e-8 * scale)
    # C aliasing A
    D = dev(A.val, "float32")
    sf.add(P, D, dev(B.val, "float32"), D, 0.75, -2.0, 0.5, prec="fp32")
    np.testing.assert_array_equal(host(D), host(C))


def test_tf32x3_timeout_record_planted_from_host(sf, c3d):
    A, levels, want = c3d
    P = pattern_of(A, levels)
    plan = sf.Plan(P, P, P, "tf32x3")
    w = plan.timeout_word()
    assert w is not None and w[0] == 0
    dA = dev(A.val, "float32")
    out = dev(np.zeros(len(A.val)), "float32")
    plan.mul(dA, dA, out)
    plan.status()                                   # nothing recorded: S_OK
    w[0] = 1                                        # plant a time-out record
    with pytest.raises(sf.SFormatError) as e:
        plan.mul(dA, dA, out)
    assert e.value.status == sf.S_ERR_TIMEOUT
    assert w[0] == 0                                # reported once, then cleared
    plan.mul(dA, dA, out)                           # the next call runs
    plan.status()
    assert rel_frob(host(out), want) <= 1e-5
    w[0] = 1
    with pytest.raises(sf.SFormatError) as e:
        plan.status()
    assert e.value.status == sf.S_ERR_TIMEOUT
    plan.status()
    # a graph of the plan's product checks the record before each replay
    g = plan.graph(dA, dA, out)
    g.launch()
    w[0] = 1
    with pytest.raises(sf.SFormatError) as e:
        g.launch()
    assert e.value.status == sf.S_ERR_TIMEOUT
    g.launch()
    plan.status()
    # the float plan's K-major kernel waits on its bulk copies with the same bound and the
    # same record
    p32 = sf.Plan(P, P, P, "fp32")
    w32 = p32.timeout_word()
    assert w32 is not None and w32[0] == 0
    o32 = dev(np.zeros(len(A.val)), "float32")
    p32.mul(dA, dA, o32)
    p32.status()
    w32[0] = 1
    with pytest.raises(sf.SFormatError) as e:
        p32.mul(dA, dA, o32)
    assert e.value.status == sf.S_ERR_TIMEOUT
    p32.mul(dA, dA, o32)
    p32.status()
    assert rel_frob(host(o32), want) <= 1e-6
