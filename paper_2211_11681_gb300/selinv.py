"""Python binding of the selected inversion and the contour-integral inverse square root
(C ABI in include/sselinv.h): argument marshalling only.

    inv = SelInv(pattern)                  # symbolic analysis, factor storage on the device
    inv.factor(A, sigma)                   # A + sigma I = L D L^T (A: float64 CUDA tensor on S)
    inv.invert(Z)                          # Z = P_S((A + sigma I)^{-1})
    inv.status()                           # raises SFormatError(S_ERR_NOT_SPD) after a bad pivot
    inv.invsqrt(A, c_lo, c_hi, n, Z)       # Z = P_S(A^{-1/2}) by Eq. (ContInt), n nodes
"""
import ctypes

import numpy as np

from . import sformat as _sf

lib = _sf.lib
_i32, _i64, _vp, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
_P = ctypes.POINTER
for _name, (_res, _args) in {
    "s_selinv_order": (_i32, [_i32, _P(_i64), _P(_i32), _P(_i32), _P(_i32), _P(_i64), _P(_i32)]),
    "s_selinv_create": (_i32, [_vp, _P(_vp)]),
    "s_selinv_destroy": (_i32, [_vp]),
    "s_selinv_stats": (_i32, [_vp, _P(_i64), _P(_i64), _P(_i32), _P(_dbl), _P(_dbl)]),
    "s_selinv_factor": (_i32, [_vp, _vp, _dbl, _vp]),
    "s_selinv_invert": (_i32, [_vp, _dbl, _dbl, _vp, _vp]),
    "s_selinv_status": (_i32, [_vp, _vp]),
    "s_selinv_invsqrt": (_i32, [_vp, _vp, _dbl, _dbl, _i32, _vp, _vp]),
    "s_contour_nodes": (_i32, [_dbl, _dbl, _i32, _P(_dbl), _P(_dbl)]),
}.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def order(bsize, rowptr, colidx):
    """Host elimination order of a symmetric block pattern: (perm, factor blocks, levels)."""
    bs = np.ascontiguousarray(bsize, dtype=np.int32)
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    nc = len(bs)
    perm = np.zeros(nc, dtype=np.int32)
    nl, lv = _i64(), _i32()
    _sf.check(lib.s_selinv_order(nc, rp.ctypes.data_as(_P(_i64)), ci.ctypes.data_as(_P(_i32)),
                                 bs.ctypes.data_as(_P(_i32)), perm.ctypes.data_as(_P(_i32)), ctypes.byref(nl),
                                 ctypes.byref(lv)))
    return perm, nl.value, lv.value


def contour_nodes(c_lo, c_hi, n):
    """Shifts w_k^2 and weights of the n-node rule of Eq. (ContInt)."""
    w2, wt = np.zeros(n), np.zeros(n)
    _sf.check(lib.s_contour_nodes(float(c_lo), float(c_hi), int(n), w2.ctypes.data_as(_P(_dbl)),
                                  wt.ctypes.data_as(_P(_dbl))))
    return w2, wt


class SelInv:
    """Selected inversion plan on a symmetric pattern (s_selinv_create)."""

    def __init__(self, pattern):
        h = _vp()
        _sf.check(lib.s_selinv_create(pattern.h, ctypes.byref(h)))
        self.h = h
        self.pattern = pattern

    def stats(self):
        nb, ne, lv, ff, fi = _i64(), _i64(), _i32(), _dbl(), _dbl()
        _sf.check(lib.s_selinv_stats(self.h, ctypes.byref(nb), ctypes.byref(ne), ctypes.byref(lv), ctypes.byref(ff),
                                     ctypes.byref(fi)))
        return {"l_blocks": nb.value, "l_entries": ne.value, "levels": lv.value, "flops_factor": ff.value,
                "flops_invert": fi.value}

    def factor(self, A, sigma=0.0, stream=None):
        _sf.check(lib.s_selinv_factor(self.h, _sf._ptr(A), float(sigma), _sf._stream(stream)))

    def invert(self, out, alpha=1.0, beta=0.0, stream=None):
        _sf.check(lib.s_selinv_invert(self.h, float(alpha), float(beta), _sf._ptr(out), _sf._stream(stream)))

    def status(self, stream=None):
        _sf.check(lib.s_selinv_status(self.h, _sf._stream(stream)))

    def invsqrt(self, A, c_lo, c_hi, n, out, stream=None):
        _sf.check(lib.s_selinv_invsqrt(self.h, _sf._ptr(A), float(c_lo), float(c_hi), int(n), _sf._ptr(out),
                                       _sf._stream(stream)))

    def __del__(self):
        try:
            if self.h.value:
                lib.s_selinv_destroy(self.h)
        except Exception:
            pass
