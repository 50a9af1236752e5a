"""Selected inversion at the size `bench.py --workload selinv_2d` times (N = 16384, uniform
[0,1]^2, exp(-r)/N, q+1 = 4, eta = 1.25, tau = 1e-5/N; inputs from the device builder, shared
by both sides), in the bench's launch configuration: sampled columns of (K + mu I)^{-1}
computed by the oracle with conjugate gradients on the CPU, compared on the entries of S in
those columns.  mu = 1e-2 (condition number about 1e2): CG to 1e-13 relative residual leaves
an error near 1e-11; tolerance 1e-9 of the column's largest entry."""
import numpy as np
import pytest

import workloads as W
from oracle import selinv as osel
from oracle.sformat import BlockCSR

pytestmark = pytest.mark.gpu


def test_sampled_columns_at_bench_size():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_11681_gb300 import selinv as si
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    w = W.WORKLOADS["selinv_2d"]
    n, mu = w.n, 1e-2
    b = Builder(W.points(w, n), w.leaf, w.q, w.eta)
    pat, K = b.values(w.nu, w.ell, 1.0 / n, 0.0, W.tau_of(w, n))
    del b
    inv = si.SelInv(pat)
    Z = torch.empty_like(K)
    inv.factor(K, mu)
    inv.invert(Z)
    inv.status()
    bo, rowptr, colidx = sf.pattern_arrays(pat.h)
    bsize = np.diff(bo)
    A = BlockCSR(bsize, rowptr, colidx, K.cpu().numpy())
    Zs = osel.to_scipy(A.like(Z.cpu().numpy())).tocsc()
    cols = np.random.Generator(np.random.PCG64(17)).choice(n, size=4, replace=False)
    X = osel.inverse_columns(osel.to_scipy(A), mu, cols)
    for t, c in enumerate(cols):
        col = Zs[:, c]
        rows = col.indices
        assert len(rows) > 0
        got = col.data
        want = X[rows, t]
        assert np.abs(got - want).max() <= 1e-9 * np.abs(X[:, t]).max(), c
