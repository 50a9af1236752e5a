"""ctypes front end of the plain-C oracle product (``product.c``).

Test infrastructure only (see ``oracle/__init__``).  ``build()`` compiles the C file into
``oracle/_build/liboracle.so`` with the host C compiler.
"""
import ctypes
import os
import subprocess

import numpy as np

from .sformat import BlockCSR

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force=False):
    """Compile product.c (gcc -O2 -fopenmp).  Returns the path of the shared object."""
    src = os.path.join(_HERE, "product.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _p64(a):
    return a.ctypes.data_as(_i64p)


def _pf(a):
    return a.ctypes.data_as(_f64p)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def mul_masked(A, B, Cpat, subset=None, nthreads=1):
    """C = P_{S_C}(A B), Eq. (product).  ``Cpat`` is a BlockCSR giving S_C (its values are
    ignored).  With ``subset`` (C block indices) only those blocks are computed and the
    rest of the result is zero.  Returns a new BlockCSR on S_C."""
    lib = _load()
    assert np.array_equal(A.bsize, B.bsize) and np.array_equal(A.bsize, Cpat.bsize)
    C = Cpat.like()
    bsize = _i64(A.bsize)
    ar, ac, av = _i64(A.rowptr), _i64(A.colidx), _i64(A.voff)
    br, bc, bv = _i64(B.rowptr), _i64(B.colidx), _i64(B.voff)
    cb, cc, cv = _i64(C.brow), _i64(C.colidx), _i64(C.voff)
    aval = np.ascontiguousarray(A.val, dtype=np.float64)
    bval = np.ascontiguousarray(B.val, dtype=np.float64)
    if subset is not None:
        sub = _i64(subset)
        sp, ns = _p64(sub), len(sub)
    else:
        sp, ns = None, 0
    lib.oracle_mul_masked(_p64(bsize), _p64(ar), _p64(ac), _p64(av), _pf(aval),
                          _p64(br), _p64(bc), _p64(bv), _pf(bval),
                          ctypes.c_int64(C.nblocks), _p64(cb), _p64(cc), _p64(cv), _pf(C.val),
                          sp, ctypes.c_int64(ns), ctypes.c_int(nthreads))
    return C


def mul_count(A, B, Cpat, subset=None):
    """(triples, useful flops) of P_{S_C}(A B), or of the listed C blocks only."""
    lib = _load()
    t = ctypes.c_int64(0)
    f = ctypes.c_double(0.0)
    if subset is not None:
        sub = _i64(subset)
        sp, ns = _p64(sub), len(sub)
    else:
        sp, ns = None, 0
    lib.oracle_mul_count(_p64(_i64(A.bsize)), _p64(_i64(A.rowptr)), _p64(_i64(A.colidx)),
                         _p64(_i64(B.rowptr)), _p64(_i64(B.colidx)), ctypes.c_int64(Cpat.nblocks),
                         _p64(_i64(Cpat.brow)), _p64(_i64(Cpat.colidx)), sp, ctypes.c_int64(ns),
                         ctypes.byref(t), ctypes.byref(f))
    return int(t.value), float(f.value)


def spmv(A, x):
    """y = A x."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.n)
    lib.oracle_spmv(ctypes.c_int64(A.nclusters), _p64(_i64(A.bsize)), _p64(_i64(A.boff)),
                    _p64(_i64(A.rowptr)), _p64(_i64(A.colidx)), _p64(_i64(A.voff)),
                    _pf(np.ascontiguousarray(A.val)), _pf(x), _pf(y))
    return y
