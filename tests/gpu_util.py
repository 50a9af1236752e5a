"""Helpers of the GPU tests: oracle BlockCSR <-> library patterns and device buffers."""
import numpy as np


def pattern_of(A, levels=None):
    from paper_2211_11681_gb300 import sformat as sf
    lv = np.zeros(A.nclusters, dtype=np.int32) if levels is None else np.asarray(levels, dtype=np.int32)
    return sf.Pattern(A.boff, lv, A.rowptr, A.colidx)


def dev(val, dtype="float64"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(val, dtype=dtype)).cuda()


def host(t):
    return t.detach().double().cpu().numpy()


def rel_frob(got, want):
    want = np.asarray(want, dtype=np.float64)
    d = np.linalg.norm(np.asarray(got, dtype=np.float64) - want)
    n = np.linalg.norm(want)
    return d / n if n > 0 else d
