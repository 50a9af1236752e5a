"""Reverse mode on the GPU: the Newton-Schulz backward (s_funm_sqrt_backward, behind
torch.autograd) against the FP64 oracle's backward, the loss gradient in the lengthscale
against central finite differences of the GPU forward (step 1e-5) and against the oracle
gradient stored by tests/golden/make_ns_grad_golden.py (N = 4096, 10 steps), and the
builder's d/dell values against the oracle's.

Tolerances: dL/dA within 1e-10 relative Frobenius (FP64, 70 products of rounding);
dL/dell within 1e-8 of the oracle's value; central differences within 1e-5 (truncation
h^2 ~ 1e-10, cancellation ~ 1e-16/h ~ 1e-11, both far below); builder d/dell values
within float rounding of the oracle's (2e-6 of the largest entry).

The mixed form (float iteration, float checkpoints, float reverse mode) differentiates the
same 10-step iteration in float.  Every masked product of it carries a relative error of
at most about 5e-7 (compensated float sums over the lambda blocks, inputs rounded to float:
measured 1e-7 to 3e-7), and the forward and reverse passes chain 30 and 60 of them; errors of
that size add up to at most about 60 x 5e-7 = 3e-5 relative in dL/dA, and to 1.5e-5 in the
loss.  The tests allow 1e-4 for the gradient quantities and 3e-5 for the loss."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import funm as ofunm
from oracle.pipeline import compress_kernel, dA_dell
from oracle.sformat import BlockCSR

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ns_grad_4096.json")


def _setup(n, ell, nugget=0.0):
    w = W.WORKLOADS["matern32_3d_grad"]
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, ell, w.q, w.leaf, w.eta, 0.0, 1.0 / n, nugget)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    return w, x, c, levels


def _gpu_loss_grad(P, Aval, zs, steps, cfix, prec="fp64"):
    import torch
    from paper_2211_11681_gb300.autograd import QuadForm, SqrtmNS
    from tests.gpu_util import dev
    A = dev(Aval).requires_grad_(True)
    X = SqrtmNS.apply(A, P, steps, cfix, prec)
    L = QuadForm.apply(X, P, dev(zs))
    L.backward()
    torch.cuda.synchronize()
    return float(L.detach()), A.grad


def test_ns_backward_matches_oracle():
    from tests.gpu_util import host, pattern_of, rel_frob
    w, x, c, levels = _setup(1024, 0.15)
    A = c.A
    zs = c.basis.T @ W.random_vector(1024, 17)
    cfix = 1.01 * ofunm.norm_estimate(A)
    X, hist, _ = ofunm.sqrtm_ns(A, steps=10, c=cfix, return_history=True, nthreads=os.cpu_count())
    dA = oadj.sqrtm_ns_backward(oadj.quad_form_grad(A, zs), hist, cfix, nthreads=os.cpu_count())
    P = pattern_of(A, levels)
    L, g = _gpu_loss_grad(P, A.val, zs, 10, cfix)
    assert L == pytest.approx(oadj.quad_form(X, zs), rel=1e-12)
    assert rel_frob(host(g), dA.val) <= 1e-10


def test_ns_lengthscale_gradient_golden_and_finite_differences():
    from tests.gpu_util import host, pattern_of
    gold = json.load(open(GOLDEN))
    n, ell, steps, h = gold["n"], gold["ell"], gold["steps"], 1e-5
    w, x, c, levels = _setup(n, ell, gold["nugget"])
    A = c.A
    assert len(A.val) == gold["nnz"]
    zs = c.basis.T @ W.random_vector(n, 17)
    cfix = gold["c"]
    assert 1.01 * ofunm.norm_estimate(A) == pytest.approx(cfix, rel=1e-10)
    P = pattern_of(A, levels)
    L, g = _gpu_loss_grad(P, A.val, zs, steps, cfix)
    g = host(g)
    dl = float(g @ dA_dell(x, c.basis, A, w.nu, ell, 1.0 / n).val)
    assert L == pytest.approx(gold["loss"], rel=1e-10)
    assert dl == pytest.approx(gold["dloss_dell"], rel=1e-8)
    assert float(g @ W.random_values(len(A.val), gold["proj_seed"])) == pytest.approx(gold["proj"], rel=1e-8)
    # central differences in ell on the fixed pattern (no re-thresholding)
    from paper_2211_11681_gb300 import sformat as sf
    from tests.gpu_util import dev

    def loss_at(l):
        cl = compress_kernel(x, w.nu, l, w.q, w.leaf, w.eta, 0.0, 1.0 / n, gold["nugget"])
        Al = BlockCSR.from_dense(cl.Khat, A.bsize, A.rowptr, A.colidx)
        F = dev(np.zeros(len(A.val)))
        sf.funm(P, "sqrt", dev(Al.val), F, steps=steps, scale=cfix)
        return sf.quad_form(P, F, dev(zs))

    fd = (loss_at(ell + h) - loss_at(ell - h)) / (2 * h)
    assert dl == pytest.approx(fd, rel=1e-5)


def test_builder_dell_values_match_oracle():
    from paper_2211_11681_gb300.builder import Builder
    from tests.gpu_util import host
    n = 2048
    w, x, c, levels = _setup(n, 0.15)
    b = Builder(x, w.leaf, w.q, w.eta)
    pat, vals = b.values(w.nu, 0.15, 1.0 / n, 0.0, 0.0)
    assert pat.nblocks == c.A.nblocks
    d = host(b.values_dell(pat, w.nu, 0.15, 1.0 / n))
    ref = dA_dell(x, c.basis, c.A, w.nu, 0.15, 1.0 / n).val
    assert np.abs(d - ref).max() <= 2e-6 * np.abs(ref).max()
    # samplet coordinates of a vector
    v = W.random_vector(n, 3)
    np.testing.assert_allclose(b.transform(v), c.basis.T @ v, atol=1e-12 * np.abs(v).max())


def test_mixed_ns_backward_matches_oracle():
    from tests.gpu_util import host, pattern_of, rel_frob
    w, x, c, levels = _setup(1024, 0.15)
    A = c.A
    zs = c.basis.T @ W.random_vector(1024, 17)
    cfix = 1.01 * ofunm.norm_estimate(A)
    X, hist, _ = ofunm.sqrtm_ns(A, steps=10, c=cfix, return_history=True, nthreads=os.cpu_count())
    dA = oadj.sqrtm_ns_backward(oadj.quad_form_grad(A, zs), hist, cfix, nthreads=os.cpu_count())
    P = pattern_of(A, levels)
    L, g = _gpu_loss_grad(P, A.val, zs, 10, cfix, "fp32")
    assert L == pytest.approx(oadj.quad_form(X, zs), rel=3e-5)
    assert rel_frob(host(g), dA.val) <= 1e-4


def test_mixed_ns_lengthscale_gradient_golden():
    from tests.gpu_util import host, pattern_of
    gold = json.load(open(GOLDEN))
    n, ell, steps = gold["n"], gold["ell"], gold["steps"]
    w, x, c, levels = _setup(n, ell, gold["nugget"])
    A = c.A
    zs = c.basis.T @ W.random_vector(n, 17)
    P = pattern_of(A, levels)
    L, g = _gpu_loss_grad(P, A.val, zs, steps, gold["c"], "fp32")
    g = host(g)
    dl = float(g @ dA_dell(x, c.basis, A, w.nu, ell, 1.0 / n).val)
    assert L == pytest.approx(gold["loss"], rel=3e-5)
    assert dl == pytest.approx(gold["dloss_dell"], rel=1e-4)
    assert float(g @ W.random_values(len(A.val), gold["proj_seed"])) == pytest.approx(gold["proj"], rel=1e-4)
