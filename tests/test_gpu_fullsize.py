"""Parity at the benchmark's full size (N = 2^20 points in [0,1]^3, Matern-1/2, ell = 0.1,
q = 3, leaf 32, eta = 1.0, tau = 1e-8), in the launch configuration bench.py times (symmetric A, float
kernel shape picked by the autotuner on this pattern): the FP64, mixed (compensated float),
split-bfloat16 and split-TF32 tensor-core products of the whole pattern on the GPU, compared on a seeded sample of
output blocks that the FP64 oracle computes one by one (plus every block of the root's row,
whose lambda lists are the longest, and the last block).

Tolerances: FP64 within 1e-12 relative Frobenius over the sampled blocks, mixed
(compensated float) within 1e-6, split-bfloat16 tensor-core products within 5e-6: the
tensor cores' float accumulation over the 18 k8 steps of a lambda slice loses about 2^-23
per step (measured 2.2e-6 over the whole product), above the 1e-6 the compensated float
kernel reaches.  Split-TF32 (tcgen05) within 1e-6: each stage's accumulator is at most nine
MMAs deep and the sums over the lambda stages are compensated (measured 3.8e-7 over the whole
product)."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    import torch
    from paper_2211_11681_gb300 import sformat as sf
    from paper_2211_11681_gb300.builder import Builder
    w = W.WORKLOADS["matern12_3d_1m"]
    b = Builder(W.points(w), w.leaf, w.q, w.eta)
    pat, vals = b.values(w.nu, w.ell, w.scale, w.nugget, w.tau)
    C64 = torch.empty_like(vals)
    sf.Plan(pat, pat, pat, "fp64").mul(vals, vals, C64)
    A32 = vals.float()
    C32 = torch.empty_like(A32)
    # the timed configuration of bench.py: symmetric A, kernel shape chosen by the autotuner
    p32 = sf.Plan(pat, pat, pat, "fp32")
    p32.set_symmetric_a(True)
    shape = p32.autotune(A32, A32, C32)
    C32.fill_(float("nan"))
    p32.mul(A32, A32, C32)
    assert p32.variant() == shape
    print("fullsize: autotuned float variant %d %s" % (p32.variant_index, shape))
    Cb = torch.empty_like(A32)
    pb = sf.Plan(pat, pat, pat, "bf16x3")
    pb.set_symmetric_a(True)
    pb.mul(A32, A32, Cb)
    cb = Cb.double().cpu().numpy()
    del pb
    pt = sf.Plan(pat, pat, pat, "tf32x3")
    pt.set_symmetric_a(True)
    pt.mul(A32, A32, Cb)
    torch.cuda.synchronize()
    return (pat, vals.cpu().numpy(), C64.cpu().numpy(), C32.double().cpu().numpy(), cb,
            Cb.double().cpu().numpy())


def test_fullsize_sampled_parity(c2):
    from oracle import product as oprod
    from oracle.sformat import BlockCSR
    pat, aval, c64, c32, cb, ct = c2
    bo, rp, ci = pat.arrays()
    A = BlockCSR(np.diff(bo), rp, ci.astype(np.int64), aval)
    rng = np.random.Generator(np.random.PCG64(2024))
    sub = np.unique(np.concatenate([rng.choice(A.nblocks, 3000, replace=False),
                                    np.arange(rp[0], rp[1]), [A.nblocks - 1]]))
    ref = oprod.mul_masked(A, A, A, subset=sub, nthreads=os.cpu_count())
    idx = np.concatenate([np.arange(A.voff[k], A.voff[k + 1]) for k in sub])
    want = ref.val[idx]
    n = np.linalg.norm(want)
    assert np.linalg.norm(c64[idx] - want) <= 1e-12 * n
    assert np.linalg.norm(c32[idx] - want) <= 1e-6 * n
    assert np.linalg.norm(cb[idx] - want) <= 5e-6 * n
    assert np.linalg.norm(ct[idx] - want) <= 1e-6 * n
