"""Pins of the oracle's samplet basis (Sec. 3.2, Thm. (waveletProperties)): the Haar
closed form, orthonormality, vanishing moments, the l1 bound on coefficient vectors, the
QR against LAPACK, and the magnitude of the compression error printed in Sec. 5.1."""
import os

import numpy as np
import pytest

from oracle.pipeline import compress_kernel
from oracle.samplets import householder_qr, m_q, monomial_exponents, monomials, samplet_basis
from oracle.tree import build_tree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_m_q_counts():
    # m_q = sum_{l<=q} C(l+d-1, d-1): 6 moments in 2D for q=2, 20 in 3D for q=3
    assert m_q(2, 2) == 6 and m_q(3, 3) == 20 and m_q(3, 2) == 10 and m_q(1, 0) == 1
    e = monomial_exponents(2, 2).tolist()
    assert e == [[0, 0], [1, 0], [0, 1], [2, 0], [1, 1], [0, 2]]


@pytest.mark.parametrize("shape", [(7, 3), (12, 6), (5, 5), (3, 6), (20, 20), (40, 20)])
def test_householder_against_lapack(shape):
    rng = np.random.Generator(np.random.PCG64(sum(shape)))
    A = rng.standard_normal(shape)
    Q, R = householder_qr(A)
    Ql, Rl = np.linalg.qr(A, mode="complete")
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(shape[0]), atol=1e-14)
    assert np.allclose(np.tril(R, -1), 0.0, atol=1e-13)
    # same reflector convention as LAPACK's geqrf: same Q and R up to rounding
    np.testing.assert_allclose(Q, Ql, atol=1e-12)
    np.testing.assert_allclose(R, Rl, atol=1e-12)


def test_haar_closed_form():
    x = (np.arange(8) / 7.0)[:, None]
    cl = build_tree(x, 1)
    B = samplet_basis(x, cl, 0)
    gold = _load("haar_8.txt")
    np.testing.assert_allclose(np.abs(B.T) * np.sqrt(8.0), gold, atol=1e-13)
    np.testing.assert_allclose(B.T @ B.T.T, np.eye(8), atol=1e-15)
    # samplets (all rows but the root scaling function) annihilate constants
    np.testing.assert_allclose(B.T[1:] @ np.ones(8), 0.0, atol=1e-14)


@pytest.mark.parametrize("n,d,q,leaf,dom", [(512, 2, 2, 16, "cube"), (700, 3, 3, 32, "cube"),
                                            (600, 3, 2, 16, "sphere"), (300, 1, 3, 4, "cube")])
def test_basis_properties(n, d, q, leaf, dom):
    rng = np.random.Generator(np.random.PCG64(n + d))
    x = rng.random((n, d))
    if dom == "sphere":
        g = rng.standard_normal((n, d))
        x = g / np.linalg.norm(g, axis=1, keepdims=True)
    cl = build_tree(x, leaf)
    B = samplet_basis(x, cl, q)
    T = B.T
    # Thm. (waveletProperties): orthonormal basis of the span of the Dirac measures
    np.testing.assert_allclose(T @ T.T, np.eye(n), atol=1e-13)
    assert B.boff[-1] == n
    # vanishing moments of order q+1 (Eq. (vanishingMoments)) for every samplet row:
    # the root's scaling rows are the only ones with nonzero moments
    P = monomials(x, monomial_exponents(d, q))
    mom = T @ P
    ns0 = B.nscal[0]
    scale = np.abs(P).max() * np.sqrt(n)
    assert np.abs(mom[ns0:]).max() <= 1e-11 * scale
    assert np.linalg.norm(mom[:ns0]) > 1e-3
    # ||omega_{j,k}||_1 <= sqrt(|nu|) for a samplet supported on nu
    for c in cl:
        r0 = B.boff[c.id] + (ns0 if c.id == 0 else 0)
        rows = T[r0:B.boff[c.id + 1]]
        if rows.size:
            outside = np.setdiff1d(np.arange(n), c.idx)
            assert np.abs(rows[:, outside]).max(initial=0.0) == 0.0      # supported on nu
            assert np.abs(rows).sum(axis=1).max() <= np.sqrt(len(c.idx)) * (1 + 1e-12)


def test_samplets_per_level_grow_like_2j():
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.random((4096, 2))
    cl = build_tree(x, 16)
    B = samplet_basis(x, cl, 2)
    per_level = {}
    for c in cl:
        per_level[c.level] = per_level.get(c.level, 0) + int(B.bsize[c.id])
    # Thm. (waveletProperties) 1.: the number of samplets on level j behaves like 2^j
    for j in range(2, max(per_level)):
        assert per_level[j] == pytest.approx(6 * 2 ** j, rel=0.01) or per_level[j] == 10 * 2 ** j


@pytest.mark.parametrize("d", [2, 3])
def test_compression_error_magnitude_matches_paper(d):
    gold = {int(r[0]): r[1] for r in _load("paper_compression_error.txt")}
    n = 4096
    rng = np.random.Generator(np.random.PCG64(11 + d))
    x = rng.random((n, d))
    c = compress_kernel(x, 0.5, 1.0, 3, 16 if d == 2 else 32, 1.25, tau=1e-5 / n, scale=1.0 / n)
    err = np.linalg.norm(c.Khat - c.A.to_dense()) / np.linalg.norm(c.Khat)
    # same order of magnitude as the paper's figure (N = 4096 is below its smallest N)
    assert gold[d] / 10 < err < gold[d] * 3


def test_full_pattern_round_trip():
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.random((300, 2))
    c = compress_kernel(x, 1.5, 0.2, 2, 16, np.inf, scale=1.0 / 300, nugget=1e-3)
    assert c.A.nblocks == int(np.sum(c.basis.bsize > 0)) ** 2
    from oracle.kernels import kernel_matrix
    K = kernel_matrix(x, 1.5, 0.2, 1.0 / 300) + 1e-3 * np.eye(300)
    T = c.basis.T
    np.testing.assert_allclose(T.T @ c.A.to_dense() @ T, K, atol=1e-14)
