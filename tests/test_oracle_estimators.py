"""Pins of the oracle's e_F estimator of the multiplication benchmark (Sec. 5.1):
e_F(M) = ||M X||_F / ||X||_F with M = A B - A (.) B applied as A (B X) - C X.

  * closed form: e_F(alpha I) = |alpha| for any X;
  * exactness: on the full pattern the formatted product is the exact product, so e_F
    vanishes to rounding;
  * brute force: on random block patterns S_A != S_B != S_C, the dense library product
    (A B - C) X of the matrices written out densely.
"""
import numpy as np
import pytest

import workloads as W
from oracle import estimators, product
from oracle.pipeline import compress_kernel
from oracle.sformat import BlockCSR
from tests.test_oracle_product import random_bcsr


def test_ef_of_scaled_identity_is_alpha():
    bsize = np.array([3, 5, 2, 4])
    A = BlockCSR(bsize, np.arange(5), np.arange(4)).identity_like(-2.5)
    X = W.estimator_probe(A.n, 10, seed=3)
    assert estimators.ef_of(A, X) == pytest.approx(2.5, rel=1e-15)


def test_ef_vanishes_on_the_full_pattern():
    w = W.WORKLOADS["paper_mult_2d"]
    n = 300
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, np.inf, 0.0, 1.0 / n)
    A = c.A
    B = A.like(A.val * W.perturbation_factors(len(A.val), 5))
    C = product.mul_masked(A, B, A)
    X = W.estimator_probe(n)
    e = estimators.ef(A, B, C, X)
    scale = np.linalg.norm(A.to_dense() @ B.to_dense() @ X) / np.linalg.norm(X)
    assert e <= 1e-14 * scale


@pytest.mark.parametrize("seed", [1, 2])
def test_ef_against_dense_product(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = rng.integers(1, 7, size=14)
    A = random_bcsr(bsize, 0.4, seed * 10)
    B = random_bcsr(bsize, 0.4, seed * 20, diag=False)
    Cp = random_bcsr(bsize, 0.5, seed * 30)
    C = product.mul_masked(A, B, Cp)
    X = W.estimator_probe(A.n, 10, seed=seed)
    M = A.to_dense() @ B.to_dense() - C.to_dense()
    want = np.linalg.norm(M @ X) / np.linalg.norm(X)
    assert estimators.ef(A, B, C, X) == pytest.approx(want, rel=1e-13)
    assert want > 0.1                    # the mask does drop terms here


def test_perturbed_operand_is_not_symmetric():
    # the benchmark's second factor breaks the symmetry of the first (Sec. 5.1)
    w = W.WORKLOADS["paper_mult_2d"]
    n = 400
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, W.tau_of(w, n), 1.0 / n)
    A = c.A
    f = W.perturbation_factors(len(A.val), 6)
    assert f.min() >= 1.0 and f.max() < 1.1
    B = A.like(A.val * f).to_dense()
    assert np.abs(B - B.T).max() > 1e-3 * np.abs(B).max()
