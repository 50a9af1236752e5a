"""Batched products: several independent S-format matrices (each with its own tree, points
uniform in [0,1]^2, Matern-3/2 with its own lengthscale, q = 2, eta = 1.25) concatenated
into one pattern and multiplied in one launch, directly and through a captured CUDA graph,
with every float kernel variant of the autotuner; each part checked against the FP64
oracle (FP64 1e-12, compensated float 1e-6 relative Frobenius)."""
import numpy as np
import pytest

import workloads as W
from oracle import product as oprod
from oracle.pipeline import compress_kernel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def parts():
    ws = W.batch_workloads(count=6, seed=4, nmin_log2=8, nmax_log2=11)
    out = []
    for w in ws:
        x = W.points(w)
        c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, 0.0, 1.0 / w.n, w.nugget)
        levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
        out.append((c.A, levels, oprod.mul_masked(c.A, c.A, c.A).val))
    return out


def test_batched_product_graph_and_variants(parts):
    import torch
    from paper_2211_11681_gb300 import sformat as sf
    from tests.gpu_util import dev, host, pattern_of, rel_frob
    pats = [pattern_of(A, lv) for A, lv, _ in parts]
    P = sf.concat(pats)
    assert P.nnz == sum(len(A.val) for A, _, _ in parts)
    vals = np.concatenate([A.val for A, _, _ in parts])
    want = np.concatenate([c for _, _, c in parts])
    offs = np.cumsum([0] + [len(A.val) for A, _, _ in parts])
    # double
    p64 = sf.Plan(P, P, P, "fp64")
    d64 = dev(vals)
    c64 = dev(np.zeros(len(vals)))
    p64.mul(d64, d64, c64)
    got = host(c64)
    for q in range(len(parts)):
        assert rel_frob(got[offs[q]:offs[q + 1]], want[offs[q]:offs[q + 1]]) <= 1e-12
    # float, every variant, direct and replayed from a graph
    p32 = sf.Plan(P, P, P, "fp32")
    d32 = dev(vals, "float32")
    for v in range(sf.lib.s_plan_num_variants()):
        p32.set_variant(v)
        c32 = dev(np.zeros(len(vals)), "float32")
        p32.mul(d32, d32, c32)
        g32 = host(c32)
        for q in range(len(parts)):
            assert rel_frob(g32[offs[q]:offs[q + 1]], want[offs[q]:offs[q + 1]]) <= 1e-6, (v, q)
        cg = dev(np.zeros(len(vals)), "float32")
        g = p32.graph(d32, d32, cg)
        g.launch()
        g.launch()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(cg), g32)          # deterministic replay
    shape = p32.autotune(d32, d32, dev(np.zeros(len(vals)), "float32"))
    assert shape["tile"] in (8, 10, 12, 16, 20)
