"""Pins of the oracle's masked product, Eq. (product): against a dense library matmul
followed by the mask (the product is exact on the pattern, Sec. 4.1), identity, symmetry,
general patterns S_A != S_B != S_C, empty rows, and the operation count."""
import numpy as np
import pytest

import workloads as W
from oracle import product
from oracle.pipeline import compress_kernel
from oracle.sformat import BlockCSR


def random_pattern(nc, density, seed, diag=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    M = rng.random((nc, nc)) < density
    if diag:
        np.fill_diagonal(M, True)
    rowptr = np.zeros(nc + 1, dtype=np.int64)
    cols = []
    for i in range(nc):
        js = np.nonzero(M[i])[0]
        cols.extend(js.tolist())
        rowptr[i + 1] = len(cols)
    return rowptr, np.array(cols, dtype=np.int64)


def random_bcsr(bsize, density, seed, diag=True):
    rowptr, colidx = random_pattern(len(bsize), density, seed, diag)
    A = BlockCSR(bsize, rowptr, colidx)
    A.val[:] = W.random_values(len(A.val), seed + 1)
    return A


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_against_dense_matmul_then_mask(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    bsize = rng.integers(0, 9, size=23)          # includes empty clusters
    A = random_bcsr(bsize, 0.3, seed * 10)
    B = random_bcsr(bsize, 0.4, seed * 20, diag=False)
    Cp = random_bcsr(bsize, 0.35, seed * 30, diag=False)
    C = product.mul_masked(A, B, Cp)
    want = (A.to_dense() @ B.to_dense()) * Cp.mask()
    np.testing.assert_allclose(C.to_dense(), want, rtol=1e-13, atol=1e-13)
    # the subset mode computes exactly the listed blocks
    sub = np.arange(0, Cp.nblocks, 3)
    Cs = product.mul_masked(A, B, Cp, subset=sub)
    for k in range(Cp.nblocks):
        if k % 3 == 0:
            np.testing.assert_array_equal(Cs.block(k), C.block(k))
        else:
            assert not np.any(Cs.block(k))


def test_compressed_kernel_matrix_product():
    w = W.WORKLOADS["matern32_2d_4096"]
    x = W.points(w, 1024)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, 1.0 / 1024, w.nugget)
    A = c.A
    C = product.mul_masked(A, A, A, nthreads=4)
    D = A.to_dense()
    np.testing.assert_allclose(C.to_dense(), (D @ D) * A.mask(), rtol=1e-12, atol=1e-15)
    # symmetric A on a symmetric pattern gives a symmetric P_S(A A)
    Cd = C.to_dense()
    np.testing.assert_allclose(Cd, Cd.T, atol=1e-15 * np.abs(Cd).max())
    # A = I gives C = P_S(B)
    I = A.identity_like()
    np.testing.assert_array_equal(product.mul_masked(I, A, A).val, A.val)
    # count: triples and flops by brute force over the block pattern
    t, f = product.mul_count(A, A, A)
    P = {(int(A.brow[k]), int(A.colidx[k])) for k in range(A.nblocks)}
    rows = {}
    for (i, j) in P:
        rows.setdefault(i, []).append(j)
    tt, ff = 0, 0.0
    for (i, j) in P:
        for l in rows[i]:
            if (l, j) in P:
                tt += 1
                ff += 2.0 * A.bsize[i] * A.bsize[l] * A.bsize[j]
    assert t == tt and f == ff


def test_spmv_and_transpose():
    bsize = np.array([3, 0, 5, 2, 4])
    A = random_bcsr(bsize, 0.6, 77)
    x = W.random_vector(A.n, 5)
    np.testing.assert_allclose(product.spmv(A, x), A.to_dense() @ x, rtol=1e-14)
    np.testing.assert_array_equal(A.transpose().to_dense(), A.to_dense().T)


def test_empty_output_and_empty_operands():
    bsize = np.array([4, 3])
    Z = BlockCSR(bsize, np.zeros(3, dtype=np.int64), np.zeros(0, dtype=np.int64))
    A = random_bcsr(bsize, 1.0, 3)
    assert product.mul_masked(A, A, Z).val.size == 0
    np.testing.assert_array_equal(product.mul_masked(Z, A, A).val, 0.0)


def test_product_of_two_kernels_on_three_eta_patterns():
    # K_A and K_B compressed on one tree with different kernels and different eta, C on a
    # third eta pattern: the oracle product equals the dense product masked to S_C
    from oracle.pattern import eta_pattern
    S = W.PAIR_2D
    w = W.Workload("pair", S["seed"], 500, S["d"], "cube", 0.0, 0.0, 0.0, S["q"], S["leaf"], 0.0, 0.0)
    x = W.points(w)
    (nua, la, ea), (nub, lb, eb) = S["a"], S["b"]
    ca = compress_kernel(x, nua, la, S["q"], S["leaf"], ea, 0.0, 1.0 / 500, S["nugget"])
    cb = compress_kernel(x, nub, lb, S["q"], S["leaf"], eb, 0.0, 1.0 / 500, S["nugget"])
    rp, ci = eta_pattern(ca.clusters, ca.basis.bsize, S["c_eta"])
    Cp = BlockCSR(ca.A.bsize, rp, ci)
    C = product.mul_masked(ca.A, cb.A, Cp)
    want = (ca.A.to_dense() @ cb.A.to_dense()) * Cp.mask()
    np.testing.assert_allclose(C.to_dense(), want, atol=1e-13 * np.abs(want).max())
    assert Cp.nblocks < cb.A.nblocks < ca.A.nblocks
