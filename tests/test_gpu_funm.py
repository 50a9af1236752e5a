"""GPU parity of the matrix-function drivers (Newton-Schulz square root, Taylor exponential
with scaling and squaring) against the FP64 oracle on the same compressed inputs.

Tolerance 1e-10 relative Frobenius for FP64: 25 Newton-Schulz steps (75 products) or
7 + s products each lose at most a few ulps relative to the oracle's summation order, and
the iterations are contractive near the fixed point."""
import numpy as np
import pytest

import workloads as W
from oracle import funm as ofunm
from oracle.pipeline import compress_kernel
from tests.gpu_util import dev, host, pattern_of, rel_frob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphere():
    w = W.WORKLOADS["matern52_sphere"]
    n = 2048
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, 1.0 / n, w.nugget)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    return c, levels


def test_sqrt_parity(sphere):
    from paper_2211_11681_gb300 import sformat as sf
    c, levels = sphere
    A = c.A
    P = pattern_of(A, levels)
    F = dev(np.zeros(len(A.val)))
    res = sf.funm(P, "sqrt", dev(A.val), F, steps=25, residual=True)
    X = ofunm.sqrtm_ns(A, steps=25, nthreads=8)
    assert rel_frob(host(F), X.val) <= 1e-10
    assert res == pytest.approx(ofunm.sqrt_residual(X, A, nthreads=8), rel=1e-6)
    Fdf = dev(np.zeros(len(A.val)))
    sf.funm(P, "sqrt", dev(A.val), Fdf, steps=25, prec="fp64_df")
    assert rel_frob(host(Fdf), X.val) <= 1e-10
    F32 = dev(np.zeros(len(A.val)))
    res32 = sf.funm(P, "sqrt", dev(A.val), F32, steps=25, prec="fp32", residual=True)
    assert rel_frob(host(F32), X.val) <= 1e-5
    assert res32 < 10 * res + 1e-5


@pytest.mark.parametrize("fn,sign", [("exp", 1.0), ("exp_neg", -1.0)])
def test_exp_parity(sphere, fn, sign):
    from paper_2211_11681_gb300 import sformat as sf
    c, levels = sphere
    A = c.A
    P = pattern_of(A, levels)
    for scale in (1.0, 12.0):                  # 12x forces squarings
        As = A.like(A.val * scale)
        F = dev(np.zeros(len(A.val)))
        sf.funm(P, fn, dev(As.val), F)
        E = ofunm.expm_taylor(As, sign=sign, nthreads=8)
        assert rel_frob(host(F), E.val) <= 1e-10


def test_mixed_sqrt_with_double_residual_correction(sphere):
    # float Newton-Schulz steps, then two residual-correction steps in double
    # (R = A/c - P_S(Y Y), Y += P_S(Z R)/2): the coupled iteration keeps Y Z^{-1} = A/c, so
    # its own steps never remove the float error in that direction; the correction does.
    # The oracle runs the same method in double throughout.  The correction contracts
    # linearly (Z is only an approximate inverse on the pattern; factors ~0.1 and ~0.25 per
    # step on this matrix in the oracle), so a float start 1.8e-7 away ends ~1e-8 from the
    # double-started result after two steps: bound 3e-8.
    from paper_2211_11681_gb300 import sformat as sf
    c, levels = sphere
    A = c.A
    P = pattern_of(A, levels)
    X = ofunm.sqrtm_ns(A, steps=25, nthreads=8, refine=2)
    F = dev(np.zeros(len(A.val)))
    res = sf.funm(P, "sqrt", dev(A.val), F, steps=25, prec="fp32", refine=2, residual=True)
    assert rel_frob(host(F), X.val) <= 3e-8
    F64 = dev(np.zeros(len(A.val)))
    res64 = sf.funm(P, "sqrt", dev(A.val), F64, steps=25, refine=2, residual=True)
    assert rel_frob(host(F64), X.val) <= 1e-10
    assert res64 == pytest.approx(ofunm.sqrt_residual(X, A, nthreads=8), rel=1e-4)
    # the corrected float result keeps the residual of double Newton-Schulz
    F0 = dev(np.zeros(len(A.val)))
    res0 = sf.funm(P, "sqrt", dev(A.val), F0, steps=25, residual=True)
    assert res64 <= res0 and res <= 3 * res0


def test_mixed_exp_double_squarings(sphere):
    from paper_2211_11681_gb300 import sformat as sf
    c, levels = sphere
    A = c.A.like(c.A.val * 12.0)
    P = pattern_of(A, levels)
    F = dev(np.zeros(len(A.val)))
    sf.funm(P, "exp_neg", dev(A.val), F, prec="fp32")
    E = ofunm.expm_taylor(A, sign=-1.0, nthreads=8)
    assert rel_frob(host(F), E.val) <= 1e-5


def test_divergence_is_reported(sphere):
    # a scaling c far below lambda_max puts eigenvalues of A/c beyond the Newton-Schulz
    # region of convergence: the driver returns S_ERR_NOT_CONVERGED (a host-side status)
    from paper_2211_11681_gb300 import sformat as sf
    c, levels = sphere
    A = c.A
    P = pattern_of(A, levels)
    lam = ofunm.norm_estimate(A)
    F = dev(np.zeros(len(A.val)))
    with pytest.raises(sf.SFormatError) as e:
        sf.funm(P, "sqrt", dev(A.val), F, steps=25, scale=0.2 * lam)
    assert e.value.status == sf.S_ERR_NOT_CONVERGED
    # the library stays usable afterwards
    sf.funm(P, "sqrt", dev(A.val), F, steps=25)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_tensor_core_forms_in_the_drivers(sphere, prec):
    # the split tensor-core products (float iterates) drive the same iterations: the square
    # root with two double residual corrections lands near the oracle's corrected double
    # result (the tensor-core products are about ten times less accurate than the compensated
    # float ones, so the start is ~2e-6 away; the two corrections contract by ~0.1 and ~0.25:
    # ~5e-8, bound 3e-7), and the exponential (tensor-core Horner products, double squarings)
    # within the float-class bound of the other mixed form
    from paper_2211_11681_gb300 import sformat as sf
    c, levels = sphere
    A = c.A
    P = pattern_of(A, levels)
    F = dev(np.zeros(len(A.val)))
    if prec == "bf16x3" and np.any(A.bsize % 2):
        # split-bfloat16 staging needs even block sizes: refused with S_ERR_ARG, no device work
        with pytest.raises(sf.SFormatError) as e:
            sf.funm(P, "sqrt", dev(A.val), F, steps=25, prec=prec, refine=2)
        assert e.value.status == sf.S_ERR_ARG
        return
    X = ofunm.sqrtm_ns(A, steps=25, nthreads=8, refine=2)
    sf.funm(P, "sqrt", dev(A.val), F, steps=25, prec=prec, refine=2)
    assert rel_frob(host(F), X.val) <= 3e-7
    A12 = A.like(A.val * 12.0)
    E = ofunm.expm_taylor(A12, sign=-1.0, nthreads=8)
    G = dev(np.zeros(len(A.val)))
    sf.funm(P, "exp_neg", dev(A12.val), G, prec=prec)
    assert rel_frob(host(G), E.val) <= 1e-5
