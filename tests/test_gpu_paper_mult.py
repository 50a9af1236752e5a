"""The multiplication benchmark of Sec. 5.1 on the GPU, against the FP64 oracle: the
formatted product K (.) K~ of the compressed exponential kernel matrix K (exp(-r)/N, q+1 = 4
vanishing moments, eta = 1.25, tau = 1e-5/N) and its perturbation K~ = K (1 + 0.1 u) on
K's a-posteriori pattern, and the error estimator e_F(K K~ - K (.) K~) with X in R^{N x 10}.

Inputs are shared (built by the oracle pipeline at N = 4096 and uploaded).  K is symmetric,
K~ is not, so the product reads B = K~ through a transposed copy.  Tolerances: FP64 product
1e-12 relative Frobenius; float products 1e-6 (every kernel shape); e_F through s_spmm
within 1e-10 of the oracle's e_F of the same product values (both FP64 on identical data)."""
import numpy as np
import pytest

import workloads as W
from oracle import estimators
from oracle import product as oprod
from oracle.pipeline import compress_kernel
from tests.gpu_util import dev, host, pattern_of, rel_frob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["paper_mult_2d", "paper_mult_3d"])
def case(request):
    w = W.WORKLOADS[request.param]
    n = 4096
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, W.tau_of(w, n), 1.0 / n, w.nugget)
    K = c.A
    Kt = K.like(K.val * W.perturbation_factors(len(K.val), w.seed + 100))
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    C = oprod.mul_masked(K, Kt, K, nthreads=8)
    X = W.estimator_probe(n)
    return w, K, Kt, levels, C, X


def gpu_ef(sf, P, K, Kt, C, X):
    """e_F(K K~ - C) through s_spmm: ||K (K~ X) - C X||_F / ||X||_F."""
    Xd = dev(np.ascontiguousarray(X.T))
    T1, T2, T3 = (dev(np.zeros(X.T.shape)) for _ in range(3))
    sf.spmm(P, Kt, Xd, T1)
    sf.spmm(P, K, T1, T2)
    sf.spmm(P, C, Xd, T3)
    return float(np.linalg.norm(host(T2) - host(T3)) / np.linalg.norm(X))


def test_fp64_product_and_estimator(case):
    from paper_2211_11681_gb300 import sformat as sf
    w, K, Kt, levels, C, X = case
    P = pattern_of(K, levels)
    dK, dKt = dev(K.val), dev(Kt.val)
    plan = sf.Plan(P, P, P, "fp64")
    assert plan.stats() == oprod.mul_count(K, Kt, K)
    out = dev(np.full(len(K.val), np.nan))
    plan.mul(dK, dKt, out)
    got = host(out)
    assert rel_frob(got, C.val) <= 1e-12
    e_gpu = gpu_ef(sf, P, dK, dKt, out, X)
    e_ref = estimators.ef(K, Kt, C, X)
    assert e_gpu == pytest.approx(e_ref, rel=1e-10)
    # the masked product drops terms: e_F is small against the product, but not zero
    scale = estimators.ef_of(C, X)
    assert 0.0 < e_ref < 1e-2 * scale


@pytest.mark.parametrize("sym", [False, True])
def test_float_products_every_shape(case, sym):
    from paper_2211_11681_gb300 import sformat as sf
    w, K, Kt, levels, C, X = case
    P = pattern_of(K, levels)
    dK, dKt = dev(K.val, "float32"), dev(Kt.val, "float32")
    plan = sf.Plan(P, P, P, "fp32")
    plan.set_symmetric_a(sym)          # K is symmetric; K~ is a different buffer
    for v in range(plan.num_variants()):
        plan.set_variant(v)
        out = dev(np.full(len(K.val), np.nan), "float32")
        plan.mul(dK, dKt, out)
        assert rel_frob(host(out), C.val) <= 1e-6, (v, sym)
    # the estimator of the float result against the oracle's on the same values
    cf = host(out)
    e_gpu = gpu_ef(sf, P, dev(K.val), dev(Kt.val), dev(cf), X)
    e_ref = estimators.ef(K, Kt, C.like(cf), X)
    assert e_gpu == pytest.approx(e_ref, rel=1e-10)
