"""Writes ns_grad_4096.json: the oracle's loss and lengthscale gradient through 10 masked
Newton-Schulz steps at N = 4096.  Calls only oracle/ (and the seeded input generators);
run from the repository root:  python tests/golden/make_ns_grad_golden.py

Workload: 4096 points uniform in [0,1]^3 (seed 5), Matern-3/2 kernel, lengthscale 0.15,
scaled by 1/N, no nugget, samplets of degree 2, leaf 16, eta = 1.25, no threshold.
Loss L(ell) = z^T P_S(A(ell)^{1/2}) z with z = T g, g ~ N(0, I) (seed 17), A^{1/2} by 10
coupled Newton-Schulz steps with the scaling c = 1.01 * lambda_max frozen.  Stored: L,
dL/dell = <dL/dA, P_S(T dK/dell T^T)>, and the projection <dL/dA, R> on a seeded uniform
[-1, 1] vector R (seed 31) of the values.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import adjoint, funm  # noqa: E402
from oracle.pipeline import compress_kernel, dA_dell  # noqa: E402

N, ELL, STEPS, NUGGET = 4096, 0.15, 10, 0.0


def main():
    w = W.WORKLOADS["matern32_3d_grad"]
    threads = os.cpu_count() or 1
    x = W.points(w, N)
    c = compress_kernel(x, w.nu, ELL, w.q, w.leaf, w.eta, 0.0, 1.0 / N, NUGGET)
    A = c.A
    zs = c.basis.T @ W.random_vector(N, 17)
    cfix = 1.01 * funm.norm_estimate(A)
    X, hist, _ = funm.sqrtm_ns(A, steps=STEPS, c=cfix, return_history=True, nthreads=threads)
    L = adjoint.quad_form(X, zs)
    dA = adjoint.sqrtm_ns_backward(adjoint.quad_form_grad(A, zs), hist, cfix, nthreads=threads)
    g = float(dA.val @ dA_dell(x, c.basis, A, w.nu, ELL, 1.0 / N).val)
    proj = float(dA.val @ W.random_values(len(A.val), 31))
    out = {"n": N, "ell": ELL, "steps": STEPS, "nugget": NUGGET, "c": cfix, "nnz": int(len(A.val)),
           "loss": L, "dloss_dell": g, "proj_seed": 31, "proj": proj}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "ns_grad_4096.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
