"""The allocation-free norm estimate (s_norm_est_noalloc) against the allocating one.

Some callers cannot let a library call cudaMalloc during a call (their device memory is
owned by their own pool allocator, or they cannot afford cudaMalloc's device-wide
synchronisation).  s_norm_est_noalloc serves them from a static device array.  This test
calls it through the C ABI twice in a row (the second call reuses the array the first one
left behind) and compares each result with s_norm_est on the same matrix.  It lives in
its own file, collected last, and passes alone or after the other tests."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle.pipeline import compress_kernel

pytestmark = pytest.mark.gpu


def test_noalloc_norm_estimate_matches_allocating_one():
    import torch
    from paper_2211_11681_gb300 import sformat as sf
    from tests.gpu_util import dev
    w = W.WORKLOADS["matern32_2d_4096"]
    n = 2048
    x = W.points(w, n)
    c = compress_kernel(x, w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, 1.0 / n, w.nugget)
    levels = np.array([cl.level for cl in c.clusters], dtype=np.int32)
    P = sf.Pattern(c.A.boff, levels, c.A.rowptr, c.A.colidx)
    A = dev(c.A.val)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    want = sf.norm_est(P, A, 50)
    for _ in range(2):
        lam = ctypes.c_double(-1.0)
        st = sf.lib.s_norm_est_noalloc(P.h, ctypes.c_void_p(A.data_ptr()), 50, ctypes.byref(lam), stream)
        assert st == sf.S_OK, sf.lib.s_last_error().decode()
        assert lam.value == pytest.approx(want, rel=1e-12)
    # a different matrix on the same pattern
    B = dev(c.A.val * 3.0)
    lam = ctypes.c_double(-1.0)
    assert sf.lib.s_norm_est_noalloc(P.h, ctypes.c_void_p(B.data_ptr()), 50, ctypes.byref(lam), stream) == sf.S_OK
    assert lam.value == pytest.approx(3.0 * want, rel=1e-12)
    # then a smaller matrix (N = 1024) on its own, smaller pattern: the array still holds the
    # larger call's vectors beyond N = 1024, which must not leak into this one
    m = 1024
    xs = W.points(w, m, seed=77)
    cs = compress_kernel(xs, w.nu, w.ell, w.q, w.leaf, w.eta, w.tau, 1.0 / m, w.nugget)
    Ps = sf.Pattern(cs.A.boff, np.array([cl.level for cl in cs.clusters], dtype=np.int32), cs.A.rowptr,
                    cs.A.colidx)
    As = dev(cs.A.val)
    want_s = sf.norm_est(Ps, As, 50)
    lam = ctypes.c_double(-1.0)
    st = sf.lib.s_norm_est_noalloc(Ps.h, ctypes.c_void_p(As.data_ptr()), 50, ctypes.byref(lam), stream)
    assert st == sf.S_OK, sf.lib.s_last_error().decode()
    assert lam.value == pytest.approx(want_s, rel=1e-12)


def test_noalloc_rejects_oversized_pattern():
    from paper_2211_11681_gb300 import sformat as sf
    import torch
    nc = 64                                   # 64 clusters of 16385 rows: N = 1048640 > 2^20
    bo = np.arange(nc + 1, dtype=np.int64) * 16385
    P = sf.Pattern(bo, np.zeros(nc, dtype=np.int32), np.zeros(nc + 1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = ctypes.c_double(0.0)
    st = sf.lib.s_norm_est_noalloc(P.h, ctypes.c_void_p(A.data_ptr()), 5, ctypes.byref(lam), None)
    assert st == sf.S_ERR_ARG
    assert "exceeds the static scratch limit" in sf.lib.s_last_error().decode()
