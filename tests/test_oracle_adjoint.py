"""Pins of the oracle's reverse mode: the dot-product identity of the masked product's
adjoint, and central finite differences of L(ell) = z^T P_S(A(ell)^{1/2}) z."""
import numpy as np

import workloads as W
from oracle import adjoint, funm, product
from oracle.pipeline import compress_kernel, dA_dell
from tests.test_oracle_product import random_bcsr


def test_adjoint_dot_product_identity():
    rng = np.random.Generator(np.random.PCG64(4))
    bsize = rng.integers(1, 7, size=15)
    A = random_bcsr(bsize, 0.4, 1)
    B = random_bcsr(bsize, 0.4, 2)
    Cp = random_bcsr(bsize, 0.5, 3)
    dC = Cp.like(W.random_values(len(Cp.val), 9))
    dA, dB = adjoint.mul_masked_adjoint(dC, A, B)
    # <dC, P_C(dA' B)> = <P_A(dC B^T), dA'> and <dC, P_C(A dB')> = <P_B(A^T dC), dB'>
    pA = A.like(W.random_values(len(A.val), 11))
    pB = B.like(W.random_values(len(B.val), 12))
    lhs1 = np.dot(dC.val, product.mul_masked(pA, B, Cp).val)
    lhs2 = np.dot(dC.val, product.mul_masked(A, pB, Cp).val)
    assert np.isclose(lhs1, np.dot(dA.val, pA.val), rtol=1e-12)
    assert np.isclose(lhs2, np.dot(dB.val, pB.val), rtol=1e-12)


def test_ns_gradient_matches_finite_differences():
    w = W.WORKLOADS["matern32_3d_grad"]
    n = 512
    x = W.points(w, n)
    ell, h, steps = w.ell, 1e-5, 10
    nug = 1e-2

    def build(l):
        return compress_kernel(x, w.nu, l, w.q, w.leaf, w.eta, 0.0, 1.0 / n, nug)

    c0 = build(ell)
    A = c0.A
    z = c0.basis.T @ W.random_vector(n, 17)              # samplet coordinates of z
    cfix = 1.01 * funm.norm_estimate(A)                  # frozen scaling

    def loss(Am):
        return adjoint.quad_form(funm.sqrtm_ns(Am, steps=steps, c=cfix), z)

    X, hist, c = funm.sqrtm_ns(A, steps=steps, c=cfix, return_history=True)
    dX = adjoint.quad_form_grad(A, z)
    dA = adjoint.sqrtm_ns_backward(dX, hist, c)
    # FD in ell on the fixed pattern (same S, no re-thresholding)
    from oracle.sformat import BlockCSR

    def A_at(l):
        cl = build(l)
        return BlockCSR.from_dense(cl.Khat, A.bsize, A.rowptr, A.colidx)

    fd = (loss(A_at(ell + h)) - loss(A_at(ell - h))) / (2 * h)
    g = np.dot(dA.val, dA_dell(x, c0.basis, A, w.nu, ell, 1.0 / n).val)
    assert np.isclose(g, fd, rtol=1e-5), (g, fd)
    # directional derivative along a random direction in the values
    E = A.like(W.random_values(len(A.val), 23))
    eps = 1e-6
    fd2 = (loss(A.like(A.val + eps * E.val)) - loss(A.like(A.val - eps * E.val))) / (2 * eps)
    assert np.isclose(np.dot(dA.val, E.val), fd2, rtol=1e-5)
