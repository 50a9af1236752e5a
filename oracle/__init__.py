"""Plain, slow, FP64 CPU oracle for the samplet S-format algebra (Harbrecht, Multerer,
Schenk, Schwab, "Multiresolution kernel matrix algebra", arXiv 2211.11681).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call, link or
execute anything here; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` do.  The oracle shares no code with the CUDA path: it has its own
cluster tree, samplet basis, pattern, values, block-CSR container, product (plain C,
``product.c``), addition, norm estimate, Newton-Schulz, exponential and adjoint.

Modules and the passage of the paper each one follows:

  kernels   Matern kernels, Eq. (matern) and the half-integer closed form (Sec. 2).
  tree      cluster tree and bounding boxes, Def. cluster-tree and the bounding-box
            lemma (Sec. 3.2).
  samplets  moment matrix, QR two-scale transform, samplet basis: refinement relation,
            Eq. (QR), Eq. (vanishingMomentsQR), Eq. (Wbasis) (Sec. 3.2).
  pattern   eta-admissibility, Eq. (cutoff), over T x T (Thm. S-compression, Sec. 3.3).
  sformat   block-CSR container; values P_S(T K T^T) with threshold tau (Sec. 3.3 and
            the a-posteriori pattern of Sec. 5).
  product   masked product, Eq. (product) of Thm. (product), Sec. 4.1, in plain C.
  funm      addition (Sec. 4.1), norm estimate by Rayleigh quotients (Sec. 5.3),
            coupled Newton-Schulz square root, Taylor scaling-and-squaring exponential
            (the power series of Sec. 4.4 with squaring added).
  adjoint   reverse mode of the masked product and of the Newton-Schulz iteration.
  estimators  the error estimator e_F of the multiplication benchmark (Sec. 5.1).
  selinv    selected inversion P_S((A + sigma I)^{-1}) and the block elimination game for
            the pattern of the factor (Sec. 4.2, Eq. (blockInv)).
  contour   A^{-1/2} by the contour-integral quadrature, Eq. (ContInt) (Sec. 4.4).

Every function with no independent pin says "parity unpinned" in its docstring.  At the
time of writing every function is pinned by a test under ``tests/test_oracle_*.py``.
"""
