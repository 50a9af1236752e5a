"""Python binding of the input builder (include/sbuild.h): argument marshalling only.

    b = Builder(points, leaf=32, q=3, eta=1.0)      # tree, two-scale transforms, eta pattern
    pattern, values = b.values(nu, ell, kscale, nugget, tau)   # kept pattern + device values
"""
import ctypes

import numpy as np

from . import sformat as _sf

lib = _sf.lib
_i32, _i64, _vp, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
_P = ctypes.POINTER
for _name, (_res, _args) in {
    "s_build_create": (_i32, [_i64, _i32, _P(_dbl), _i32, _i32, _dbl, _P(_vp)]),
    "s_build_destroy": (_i32, [_vp]),
    "s_build_sizes": (_i32, [_vp, _P(_i32), _P(_i64), _P(_i64)]),
    "s_build_arrays": (_i32, [_vp, _P(_P(_i64)), _P(_P(_i32)), _P(_P(_i64)), _P(_P(_i32)), _P(_P(_i64))]),
    "s_build_dense_transform": (_i32, [_vp, _P(_dbl)]),
    "s_build_values": (_i32, [_vp, _dbl, _dbl, _dbl, _dbl, _dbl, _P(_vp)]),
    "s_build_take_values": (_i32, [_vp, _vp, _vp]),
    "s_build_values_dell": (_i32, [_vp, _dbl, _dbl, _dbl, _vp, _vp]),
    "s_build_transform": (_i32, [_vp, _P(_dbl), _P(_dbl)]),
    "s_build_kernel_matvec": (_i32, [_vp, _dbl, _dbl, _dbl, _dbl, _P(_dbl), _P(_dbl)]),
}.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class _Borrowed:
    """Pattern handle created by the builder (owned by Python)."""

    def __init__(self, h):
        self.h = h

    @property
    def nnz(self):
        return int(lib.s_pattern_nnz(self.h))

    @property
    def nblocks(self):
        return int(lib.s_pattern_nblocks(self.h))

    @property
    def n(self):
        return _sf.pattern_dim(self.h)

    def block_offsets(self):
        out = np.zeros(self.nblocks + 1, dtype=np.int64)
        _sf.check(lib.s_pattern_block_offsets(self.h, out.ctypes.data_as(_P(_i64))))
        return out

    def arrays(self):
        return _sf.pattern_arrays(self.h)

    def __del__(self):
        try:
            if self.h.value:
                lib.s_pattern_destroy(self.h)
        except Exception:
            pass


class Builder:
    def __init__(self, points, leaf, q, eta):
        x = np.ascontiguousarray(points, dtype=np.float64)
        n, d = x.shape
        h = _vp()
        _sf.check(lib.s_build_create(n, d, x.ctypes.data_as(_P(_dbl)), int(leaf), int(q), float(eta), ctypes.byref(h)))
        self.h = h
        self.n = n
        nc, nb, nnz = _i32(), _i64(), _i64()
        _sf.check(lib.s_build_sizes(h, ctypes.byref(nc), ctypes.byref(nb), ctypes.byref(nnz)))
        self.nclusters, self.nblocks_apriori, self.nnz_apriori = nc.value, nb.value, nnz.value
        bo, lv, rp, ci, pm = _P(_i64)(), _P(_i32)(), _P(_i64)(), _P(_i32)(), _P(_i64)()
        _sf.check(lib.s_build_arrays(h, ctypes.byref(bo), ctypes.byref(lv), ctypes.byref(rp), ctypes.byref(ci),
                                     ctypes.byref(pm)))
        cnc, cnb = self.nclusters, self.nblocks_apriori
        self.block_offset = np.ctypeslib.as_array(bo, shape=(cnc + 1,)).copy()
        self.level = np.ctypeslib.as_array(lv, shape=(cnc,)).copy()
        self.rowptr = np.ctypeslib.as_array(rp, shape=(cnc + 1,)).copy()
        self.colidx = np.ctypeslib.as_array(ci, shape=(max(cnb, 1),))[:cnb].copy()
        self.perm = np.ctypeslib.as_array(pm, shape=(n,)).copy()

    @property
    def bsize(self):
        return np.diff(self.block_offset)

    def dense_transform(self):
        T = np.zeros((self.n, self.n))
        _sf.check(lib.s_build_dense_transform(self.h, T.ctypes.data_as(_P(_dbl))))
        return T

    def values(self, nu, ell, kscale=1.0, nugget=0.0, tau=0.0):
        """(pattern handle, torch float64 CUDA tensor of its values)."""
        import torch
        ph = _vp()
        _sf.check(lib.s_build_values(self.h, float(nu), float(ell), float(kscale), float(nugget), float(tau),
                                     ctypes.byref(ph)))
        pat = _Borrowed(ph)
        out = torch.empty(max(pat.nnz, 1), dtype=torch.float64, device="cuda")
        _sf.check(lib.s_build_take_values(self.h, _vp(out.data_ptr()), _sf._stream(None)))
        return pat, out[:pat.nnz]

    def values_dell(self, pattern, nu, ell, kscale=1.0):
        """d/dell of the compressed values on `pattern` (torch float64 CUDA tensor)."""
        import torch
        out = torch.empty(max(pattern.nnz, 1), dtype=torch.float64, device="cuda")
        _sf.check(lib.s_build_values_dell(self.h, float(nu), float(ell), float(kscale), pattern.h,
                                          _vp(out.data_ptr())))
        return out[:pattern.nnz]

    def kernel_matvec(self, nu, ell, kscale, nugget, v):
        """(kscale K + nugget I) v with the uncompressed kernel matrix (host vectors, original
        point order)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n)
        _sf.check(lib.s_build_kernel_matvec(self.h, float(nu), float(ell), float(kscale), float(nugget),
                                            v.ctypes.data_as(_P(_dbl)), out.ctypes.data_as(_P(_dbl))))
        return out

    def transform(self, v):
        """T v (samplet coordinates) of a host vector in original point order."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n)
        _sf.check(lib.s_build_transform(self.h, v.ctypes.data_as(_P(_dbl)), out.ctypes.data_as(_P(_dbl))))
        return out

    def __del__(self):
        try:
            if self.h.value:
                lib.s_build_destroy(self.h)
        except Exception:
            pass
