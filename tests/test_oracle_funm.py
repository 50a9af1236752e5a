"""Pins of the oracle's addition, norm estimate, Newton-Schulz square root and Taylor
exponential: full-pattern cases against eigendecompositions (textbook), diagonal cases
against scalar functions, exp(0) = I, and the residual of the masked square root."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import funm, product
from oracle.pipeline import compress_kernel
from oracle.sformat import BlockCSR


def full_case(n=200, nugget=1e-2):
    w = W.WORKLOADS["matern52_sphere"]
    x = W.points(w, n)
    return compress_kernel(x, w.nu, w.ell, w.q, w.leaf, np.inf, 0.0, 1.0 / n, nugget)


def test_add():
    c = full_case(100)
    A = c.A
    B = A.like(W.random_values(len(A.val), 3))
    C = funm.add(A, B, 2.0, -0.5, 0.25)
    np.testing.assert_allclose(C.to_dense(), 2 * A.to_dense() - 0.5 * B.to_dense() + 0.25 * np.eye(A.n), atol=1e-15)


def test_norm_estimate():
    c = full_case(300)
    lam = funm.norm_estimate(c.A)
    ev = np.linalg.eigvalsh(c.A.to_dense())
    assert lam <= ev[-1] * (1 + 1e-12)          # a Rayleigh quotient never exceeds lambda_max
    assert lam == pytest.approx(ev[-1], rel=1e-6)


def test_sqrt_full_pattern_matches_eigh():
    c = full_case(200, nugget=5e-2)
    A = c.A
    X = funm.sqrtm_ns(A, steps=25)
    ev, V = np.linalg.eigh(A.to_dense())
    want = (V * np.sqrt(ev)) @ V.T
    np.testing.assert_allclose(X.to_dense(), want, atol=1e-10 * np.abs(want).max())
    assert funm.sqrt_residual(X, A) < 1e-10


def test_sqrt_diagonal_is_elementwise():
    bsize = np.array([3, 2, 4])
    rowptr = np.array([0, 1, 2, 3])
    colidx = np.array([0, 1, 2])
    A = BlockCSR(bsize, rowptr, colidx)
    d = np.linspace(0.2, 1.0, 9)
    A.val[:] = np.concatenate([np.diag(d[0:3]).ravel(), np.diag(d[3:5]).ravel(), np.diag(d[5:9]).ravel()])
    X = funm.sqrtm_ns(A, steps=30)
    np.testing.assert_allclose(np.diag(X.to_dense()), np.sqrt(d), rtol=1e-12)


def test_masked_sqrt_residual_small_on_compressed_matrix():
    w = W.WORKLOADS["matern52_sphere"]
    x = W.points(w, 1024)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, 0.0, 1.0 / 1024, w.nugget)
    X = funm.sqrtm_ns(c.A, steps=25, nthreads=4)
    r = funm.sqrt_residual(X, c.A, nthreads=4)
    assert r < 1e-3


def test_exp_full_pattern_matches_expm():
    c = full_case(150, nugget=0.0)
    A = c.A
    for sign in (1.0, -1.0):
        E = funm.expm_taylor(A, sign=sign)
        want = expm(sign * A.to_dense())
        np.testing.assert_allclose(E.to_dense(), want, atol=1e-9 * np.abs(want).max())
    # a matrix with lambda_max > theta takes squarings
    B = A.like(A.val * 40.0)
    s = funm.exp_scaling(funm.norm_estimate(B))
    assert s >= 1
    np.testing.assert_allclose(funm.expm_taylor(B, -1.0).to_dense(), expm(-B.to_dense()), atol=1e-8)


def test_exp_of_zero_is_identity():
    c = full_case(60)
    Z = c.A.like()
    np.testing.assert_array_equal(funm.expm_taylor(Z).to_dense(), np.eye(c.A.n))


def test_taylor_degree8_scalar():
    # 1x1 block: Horner on the degree-8 series equals the truncated series exactly
    A = BlockCSR(np.array([1]), np.array([0, 1]), np.array([0]), np.array([0.3]))
    E = funm.expm_taylor(A, s=0)
    assert E.val[0] == pytest.approx(sum(0.3 ** k / math.factorial(k) for k in range(9)), rel=1e-15)


def _sqrt_and_inverse(B):
    ev, V = np.linalg.eigh(B.to_dense())
    return (V * np.sqrt(ev)) @ V.T, (V / np.sqrt(ev)) @ V.T


def test_refine_contraction_commuting_perturbation():
    # Y = (1 + e) S with S = B^{1/2} and Z = S^{-1} exactly: R = B - Y^2 = -(2e + e^2) S^2 and
    # Y + Z R / 2 = (1 - e^2/2) S, so one correction leaves the relative error e^2/2 and a
    # second one (e^2/2)^2 / 2 = e^4/8.  A sign slip gives (1 + 2e) S; a lost factor 1/2
    # gives (1 - e - e^2) S.
    c = full_case(120, nugget=5e-2)
    A = c.A
    B = A.like(A.val / (1.01 * funm.norm_estimate(A)))
    S, Si = _sqrt_and_inverse(B)
    eps = 1e-3
    Y = BlockCSR.from_dense((1 + eps) * S, A.bsize, A.rowptr, A.colidx)
    Z = BlockCSR.from_dense(Si, A.bsize, A.rowptr, A.colidx)
    ns = np.linalg.norm(S)
    Y1 = funm.ns_refine(B, Y, Z, 1)
    assert np.linalg.norm(Y1.to_dense() - S) / ns == pytest.approx(eps ** 2 / 2, rel=1e-6)
    Y2 = funm.ns_refine(B, Y, Z, 2)
    assert np.linalg.norm(Y2.to_dense() - S) / ns < 2e-13 + eps ** 4 / 8 * 1.01


def test_refine_one_step_closed_form_general_perturbation():
    # Y = S + E, Z = S^{-1}: Y + Z (B - Y^2)/2 = S + E/2 - S^{-1} E S / 2 - S^{-1} E^2 / 2
    # exactly, for any E (the non-commuting part of E survives to first order).
    c = full_case(100, nugget=5e-2)
    A = c.A
    B = A.like(A.val / (1.01 * funm.norm_estimate(A)))
    S, Si = _sqrt_and_inverse(B)
    rng = np.random.Generator(np.random.PCG64(11))
    E = rng.standard_normal(S.shape) * 1e-4 * np.abs(S).max()
    Y = BlockCSR.from_dense(S + E, A.bsize, A.rowptr, A.colidx)
    Z = BlockCSR.from_dense(Si, A.bsize, A.rowptr, A.colidx)
    got = funm.ns_refine(B, Y, Z, 1).to_dense()
    want = S + E / 2 - Si @ E @ S / 2 - Si @ E @ E / 2
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(S).max())


def test_sqrtm_ns_refine_improves_an_unconverged_iteration():
    # four Newton-Schulz steps leave the full-pattern square root far from converged; the
    # two double corrections of sqrtm_ns(refine=2) move it towards the eigh square root
    c = full_case(120, nugget=5e-2)
    A = c.A
    ev, V = np.linalg.eigh(A.to_dense())
    want = (V * np.sqrt(ev)) @ V.T
    e0 = np.linalg.norm(funm.sqrtm_ns(A, steps=4).to_dense() - want)
    e2 = np.linalg.norm(funm.sqrtm_ns(A, steps=4, refine=2).to_dense() - want)
    assert e2 < 0.1 * e0
