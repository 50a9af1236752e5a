"""Seeded synthetic inputs shared by the product path, the tests and the benchmark.

This module holds no arithmetic of the method: only point clouds drawn from numpy's
PCG64 generator, the parameter sets of the workloads, and random vectors/values used as
inputs.  Workloads (uniform points in the unit cube as in the paper's multiplication
benchmark, Sec. 5.1; points on the unit sphere as a stand-in for the 3D scan of
Sec. 5.3):

  matern32_2d_4096    N=4096 uniform [0,1]^2, Matern-3/2, ell=0.2, nugget 1e-3, q=2,
                      leaf 16, eta=1.25, tau=1e-10; C = P_S(A A) in FP64.
  matern12_3d_1m      N=2^20 uniform [0,1]^3, Matern-1/2, ell=0.1, q=3, leaf 32,
                      eta=1.0, tau=1e-8; FP64 vs mixed precision.
  matern52_sphere     N=2^18 on the unit sphere, Matern-5/2, ell=0.3, nugget 1e-2, q=2,
                      leaf 16, eta=1.25; A^{1/2} (25 Newton-Schulz steps), exp(-A).
  matern32_2d_batch   256 matrices, N log-uniform in [2^10, 2^16], uniform [0,1]^2,
                      Matern-3/2, ell ~ U[0.05, 0.5], q=2, leaf 16, eta=1.25.
  matern32_3d_grad    N=2^20 uniform [0,1]^3, Matern-3/2, ell=0.15, q=2, 10 NS steps,
                      gradient checked at N=4096.
  paper_mult_2d/3d    the multiplication benchmark of Sec. 5.1: uniform [0,1]^d, the
                      exponential kernel exp(-r)/N (Matern-1/2, ell=1), q+1 = 4 vanishing
                      moments (q=3), eta=1.25, a-posteriori tau = 1e-5/N, leaf 2*m_q (20 in
                      2D, 40 in 3D); N from 5,000 to 1,000,000 (PAPER_MULT_NS).  The second
                      factor is the first with every stored entry a scaled by (1 + 0.1 u),
                      u uniform in [0,1] (perturbation_factors).
  selinv_2d           selected inversion (K + mu I)^{-1} on S (Sec. 4.2, 5.2): paper_mult_2d's
                      points and kernel, mu in {1e-2, 1e-4, 1e-6}; N = 16384 by default.
  contour_sphere      A^{1/2} by Eq. (ContInt) (Sec. 4.4, 5.3): N = 16384 on the unit sphere,
                      exp(-2r)/N (Matern-1/2, ell = 0.5), q = 3, leaf 40, eta = 1.25,
                      tau = 1e-5/N, A = K + 1e-4 I, c_lo = 1e-4, c_hi = 1, 7 nodes.
  pair_2d_4096        two kernels on one tree for a product of different matrices: N=4096
                      uniform [0,1]^2, q=2, leaf 16; A Matern-3/2 ell=0.2 on the eta=1.25
                      pattern, B Matern-5/2 ell=0.1 on the eta=1.0 pattern, C on the eta=0.8
                      pattern (PAIR_2D).
"""
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    n: int
    d: int
    domain: str          # "cube" or "sphere"
    nu: float
    ell: float
    nugget: float
    q: int
    leaf: int
    eta: float
    tau: float
    scale_by_n: bool = True   # kernel scaled by 1/N as in Sec. 5

    @property
    def scale(self):
        return 1.0 / self.n if self.scale_by_n else 1.0

    def with_n(self, n):
        return replace(self, n=n)


WORKLOADS = {
    "matern32_2d_4096": Workload("matern32_2d_4096", 1, 4096, 2, "cube", 1.5, 0.2, 1e-3, 2, 16, 1.25, 1e-10),
    "matern12_3d_1m": Workload("matern12_3d_1m", 2, 1 << 20, 3, "cube", 0.5, 0.1, 0.0, 3, 32, 1.0, 1e-8),
    "matern52_sphere": Workload("matern52_sphere", 3, 1 << 18, 3, "sphere", 2.5, 0.3, 1e-2, 2, 16, 1.25, 0.0),
    "matern32_2d_batch": Workload("matern32_2d_batch", 4, 0, 2, "cube", 1.5, 0.0, 0.0, 2, 16, 1.25, 0.0),
    "matern32_3d_grad": Workload("matern32_3d_grad", 5, 1 << 20, 3, "cube", 1.5, 0.15, 0.0, 2, 16, 1.25, 0.0),
}


PAPER_MULT_NS = (5000, 10000, 50000, 100000, 250000, 500000, 1000000)

PAPER_MULT = {
    "paper_mult_2d": Workload("paper_mult_2d", 6, 100000, 2, "cube", 0.5, 1.0, 0.0, 3, 20, 1.25, 1e-5),
    "paper_mult_3d": Workload("paper_mult_3d", 7, 100000, 3, "cube", 0.5, 1.0, 0.0, 3, 40, 1.25, 1e-5),
}
WORKLOADS.update(PAPER_MULT)

# Selected inversion and the contour integral (Sec. 4.2-4.4 and the experiments of Sec. 5.2
# and 5.3): the inversion experiment's uniform [0,1]^2 points and exp(-r)/N kernel, ridge mu
# given at run time; the matrix-function experiment's exp(-2r)/N kernel (ell = 0.5) with
# ridge mu = 1e-4 on a closed surface (the unit sphere standing in for the 3D scan).
SELINV = {
    "selinv_2d": Workload("selinv_2d", 8, 16384, 2, "cube", 0.5, 1.0, 0.0, 3, 20, 1.25, 1e-5),
    "contour_sphere": Workload("contour_sphere", 9, 16384, 3, "sphere", 0.5, 0.5, 1e-4, 3, 40, 1.25, 1e-5),
}
WORKLOADS.update(SELINV)

# Product of two different kernels on one tree (same points, leaf and q), three patterns:
# (nu, ell, eta) of A, of B, and the eta of C's pattern.
PAIR_2D = {"seed": 8, "n": 4096, "d": 2, "q": 2, "leaf": 16,
           "a": (1.5, 0.2, 1.25), "b": (2.5, 0.1, 1.0), "c_eta": 0.8, "nugget": 1e-3}


def tau_of(w, n):
    """Absolute threshold of a workload at size n: the paper-benchmark workloads state tau
    relative to 1/N (tau = 1e-5/N), the others absolutely."""
    return w.tau / n if w.name.startswith(("paper_mult", "selinv", "contour")) else w.tau


def perturbation_factors(count, seed):
    """1 + 0.1 u with u uniform in [0, 1): the factors of the perturbed second operand of the
    multiplication benchmark, one per stored entry (host, FP64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + 0.1 * rng.random(count)


def estimator_probe(n, k=10, seed=99):
    """The N x k matrix X of independent uniform [0,1) entries of the e_F estimator."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, k))


def points(w, n=None, seed=None):
    """n points of the workload's domain from PCG64(seed)."""
    n = w.n if n is None else n
    rng = np.random.Generator(np.random.PCG64(w.seed if seed is None else seed))
    if w.domain == "cube":
        return rng.random((n, w.d))
    if w.domain == "sphere":
        g = rng.standard_normal((n, w.d))
        return g / np.linalg.norm(g, axis=1, keepdims=True)
    raise ValueError(w.domain)


def batch_workloads(count=256, seed=4, nmin_log2=10, nmax_log2=16):
    """The batched workload: N = floor(2^U[10,16]), ell ~ U[0.05, 0.5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.floor(2.0 ** rng.uniform(nmin_log2, nmax_log2, size=count)).astype(np.int64)
    ells = rng.uniform(0.05, 0.5, size=count)
    base = WORKLOADS["matern32_2d_batch"]
    return [replace(base, name="%s_%d" % (base.name, i), seed=1000 + i, n=int(n), ell=float(l))
            for i, (n, l) in enumerate(zip(ns, ells))]


def random_vector(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


def random_values(count, seed, lo=-1.0, hi=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=count)
