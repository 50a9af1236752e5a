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
