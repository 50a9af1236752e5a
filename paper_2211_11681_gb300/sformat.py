"""Python binding of libsformat.so (C ABI in include/sformat.h): argument marshalling only.

Value buffers are torch CUDA tensors (float64 or float32, contiguous); patterns are built
from numpy arrays.  Every call checks the returned status and raises ``SFormatError``
carrying the library's message.  There is no fallback: if the shared library is missing
the import of this module fails.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsformat.so")

S_OK, S_ERR_ARG, S_ERR_PATTERN, S_ERR_MISMATCH, S_ERR_NOMEM, S_ERR_CUDA, S_ERR_NOT_CONVERGED, S_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
S_ERR_NOT_SPD = -8
S_FP64, S_FP32, S_BF16X3, S_FP64_DF, S_TF32X3 = 0, 1, 2, 3, 4
S_SQRT, S_EXP, S_EXP_NEG = 0, 1, 2

PREC = {"fp64": S_FP64, "fp32": S_FP32, "bf16x3": S_BF16X3, "fp64_df": S_FP64_DF, "tf32x3": S_TF32X3}


class SFormatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("sformat status %d: %s" % (status, msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsformat.so is not built (%s); run paper_2211_11681_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, vp, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "s_pattern_create": (i32, [i32, P(i64), P(i32), P(i64), P(i32), P(vp)]),
        "s_pattern_destroy": (i32, [vp]),
        "s_pattern_nnz": (i64, [vp]),
        "s_pattern_nblocks": (i64, [vp]),
        "s_pattern_block_offsets": (i32, [vp, P(i64)]),
        "s_pattern_host_arrays": (i32, [vp, P(i32), P(P(i64)), P(P(i64)), P(P(i32))]),
        "s_plan_create": (i32, [vp, vp, vp, i32, P(vp)]),
        "s_plan_destroy": (i32, [vp]),
        "s_plan_stats": (i32, [vp, P(i64), P(dbl)]),
        "s_plan_status": (i32, [vp, vp]),
        "s_plan_timeout_word": (i32, [vp, P(P(ctypes.c_uint))]),
        "s_plan_autotune": (i32, [vp, vp, vp, vp, vp, P(i32)]),
        "s_plan_variant": (i32, [vp, i32, P(i32), P(i32), P(i32), P(i32)]),
        "s_plan_set_variant": (i32, [vp, i32]),
        "s_plan_set_symmetric_a": (i32, [vp, i32]),
        "s_plan_num_variants": (i32, []),
        "s_plan_num_variants_of": (i32, [vp]),
        "s_pattern_concat": (i32, [i32, P(vp), P(vp)]),
        "s_graph_capture_mul": (i32, [vp, vp, vp, vp, P(vp)]),
        "s_graph_launch": (i32, [vp, vp]),
        "s_graph_destroy": (i32, [vp]),
        "s_mul_masked": (i32, [vp, vp, vp, vp, vp]),
        "s_mul_masked_adjoint": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "s_add": (i32, [vp, i32, dbl, vp, dbl, vp, dbl, vp, vp]),
        "s_norm_est": (i32, [vp, vp, i32, P(dbl), vp]),
        "s_spmm": (i32, [vp, vp, vp, i32, vp, vp]),
        "s_norm_est_noalloc": (i32, [vp, vp, i32, P(dbl), vp]),
        "s_funm": (i32, [vp, i32, vp, vp, vp, vp]),
        "s_funm_sqrt_backward": (i32, [vp, i32, dbl, vp, vp, vp, vp]),
        "s_funm_sqrt_backward_prec": (i32, [vp, i32, i32, dbl, vp, vp, vp, vp]),
        "s_quad_form": (i32, [vp, vp, vp, P(dbl), vp]),
        "s_quad_form_grad": (i32, [vp, vp, vp, vp]),
        "s_peak_fma": (i32, [i32, P(dbl), vp]),
        "s_last_error": (ctypes.c_char_p, []),
        "s_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class FunmOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("taylor_degree", ctypes.c_int), ("prec", ctypes.c_int),
                ("scale", ctypes.c_double), ("squarings", ctypes.c_int),
                ("residual", ctypes.POINTER(ctypes.c_double)), ("checkpoints", ctypes.c_void_p),
                ("refine", ctypes.c_int)]


def check(st):
    if st != S_OK:
        raise SFormatError(st, lib.s_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("value buffers must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _a(x, dt):
    return np.ascontiguousarray(x, dtype=dt)


def pattern_arrays(h):
    """(block_offset, rowptr, colidx) numpy copies of a pattern handle's host arrays."""
    nc = ctypes.c_int32()
    bo, rp, ci = ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int32)()
    check(lib.s_pattern_host_arrays(h, ctypes.byref(nc), ctypes.byref(bo), ctypes.byref(rp), ctypes.byref(ci)))
    n = nc.value
    rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    nb = int(rowptr[-1])
    colidx = np.ctypeslib.as_array(ci, shape=(max(nb, 1),))[:nb].copy() if nb else np.zeros(0, np.int32)
    return np.ctypeslib.as_array(bo, shape=(n + 1,)).copy(), rowptr, colidx


def pattern_dim(h):
    """Matrix dimension of a pattern handle (its last block offset)."""
    nc = ctypes.c_int32()
    bo, rp, ci = ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int64)(), ctypes.POINTER(ctypes.c_int32)()
    check(lib.s_pattern_host_arrays(h, ctypes.byref(nc), ctypes.byref(bo), ctypes.byref(rp), ctypes.byref(ci)))
    return int(bo[nc.value])


class Pattern:
    """A block pattern S on the device (s_pattern_create)."""

    def __init__(self, block_offset, level, rowptr, colidx):
        self._bo = _a(block_offset, np.int64)
        self._lv = _a(level, np.int32)
        self._rp = _a(rowptr, np.int64)
        self._ci = _a(colidx, np.int32)
        h = ctypes.c_void_p()
        P = ctypes.POINTER
        check(lib.s_pattern_create(len(self._bo) - 1, self._bo.ctypes.data_as(P(ctypes.c_int64)),
                                   self._lv.ctypes.data_as(P(ctypes.c_int32)),
                                   self._rp.ctypes.data_as(P(ctypes.c_int64)),
                                   self._ci.ctypes.data_as(P(ctypes.c_int32)), ctypes.byref(h)))
        self.h = h

    @property
    def nnz(self):
        return int(lib.s_pattern_nnz(self.h))

    @property
    def nblocks(self):
        return int(lib.s_pattern_nblocks(self.h))

    @property
    def n(self):
        """Matrix dimension (the last block offset)."""
        return pattern_dim(self.h)

    def block_offsets(self):
        out = np.zeros(self.nblocks + 1, dtype=np.int64)
        check(lib.s_pattern_block_offsets(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return out

    def arrays(self):
        return pattern_arrays(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.s_pattern_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Symbolic phase of C = P_{S_C}(A B) (s_plan_create)."""

    def __init__(self, A, B, C, prec="fp64"):
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        self.pats = (A, B, C)           # the patterns must outlive the plan
        h = ctypes.c_void_p()
        check(lib.s_plan_create(A.h, B.h, C.h, self.prec, ctypes.byref(h)))
        self.h = h

    def stats(self):
        t = ctypes.c_int64()
        f = ctypes.c_double()
        check(lib.s_plan_stats(self.h, ctypes.byref(t), ctypes.byref(f)))
        return int(t.value), float(f.value)

    def autotune(self, A, B, C, stream=None):
        """Pick the fastest float kernel variant on these operands; returns its shape."""
        v = ctypes.c_int32(-1)
        check(lib.s_plan_autotune(self.h, _ptr(A), _ptr(B), _ptr(C), _stream(stream), ctypes.byref(v)))
        self.variant_index = v.value
        return self.variant()

    def set_symmetric_a(self, flag=True):
        """Caller asserts A is symmetric; the product reads A through its transposed index."""
        check(lib.s_plan_set_symmetric_a(self.h, 1 if flag else 0))

    def num_variants(self):
        return int(lib.s_plan_num_variants_of(self.h))

    def set_variant(self, v):
        check(lib.s_plan_set_variant(self.h, int(v)))
        self.variant_index = int(v)

    def variant(self):
        t, r, c, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib.s_plan_variant(self.h, -1, ctypes.byref(t), ctypes.byref(r), ctypes.byref(c), ctypes.byref(k)))
        return {"tile": t.value, "micro": (r.value, c.value), "stage_k": k.value}

    def graph(self, A, B, C):
        """CUDA graph of mul(A, B, C) on these buffers."""
        return Graph(self, A, B, C)

    def mul(self, A, B, C, stream=None):
        check(lib.s_mul_masked(self.h, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
        return C

    def status(self, stream=None):
        """Synchronise the stream and raise SFormatError(S_ERR_TIMEOUT) if a bounded device
        wait of an earlier product of this plan ran out (s_plan_status)."""
        check(lib.s_plan_status(self.h, _stream(stream)))

    def timeout_word(self):
        """ctypes pointer to the plan's host-mapped time-out word (None when it has none)."""
        w = ctypes.POINTER(ctypes.c_uint)()
        check(lib.s_plan_timeout_word(self.h, ctypes.byref(w)))
        return w if w else None

    def adjoint(self, dC, A, B, dA=None, dB=None, stream=None):
        check(lib.s_mul_masked_adjoint(self.h, _ptr(dC), _ptr(A), _ptr(B), _ptr(dA), _ptr(dB), _stream(stream)))
        return dA, dB

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.s_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    def __init__(self, plan, A, B, C):
        self.keep = (plan, A, B, C)
        h = ctypes.c_void_p()
        check(lib.s_graph_capture_mul(plan.h, _ptr(A), _ptr(B), _ptr(C), ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None):
        check(lib.s_graph_launch(self.h, _stream(stream)))

    def __del__(self):
        try:
            if self.h.value:
                lib.s_graph_destroy(self.h)
        except Exception:
            pass


class _Owned:
    """A pattern handle created by the library (s_pattern_concat)."""

    def __init__(self, h):
        self.h = h

    nnz = property(lambda self: int(lib.s_pattern_nnz(self.h)))
    nblocks = property(lambda self: int(lib.s_pattern_nblocks(self.h)))

    def arrays(self):
        return pattern_arrays(self.h)

    def __del__(self):
        try:
            if self.h.value:
                lib.s_pattern_destroy(self.h)
        except Exception:
            pass


def concat(patterns):
    """One pattern holding the given patterns' matrices side by side (s_pattern_concat)."""
    arr = (ctypes.c_void_p * len(patterns))(*[p.h.value for p in patterns])
    h = ctypes.c_void_p()
    check(lib.s_pattern_concat(len(patterns), arr, ctypes.byref(h)))
    return _Owned(h)


def add(pattern, A, B, C, alpha=1.0, beta=1.0, gamma=0.0, prec="fp64", stream=None):
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    check(lib.s_add(pattern.h, p, float(alpha), _ptr(A), float(beta), _ptr(B), float(gamma), _ptr(C),
                    _stream(stream)))
    return C


def spmm(pattern, A, X, Y, stream=None):
    """Y = A X for a double value buffer A and N x k matrices X, Y stored column-major (torch
    tensors of shape (k, N), contiguous, float64) (s_spmm)."""
    if X.dim() != 2 or Y.shape != X.shape or X.shape[1] != pattern.n:
        raise ValueError("spmm: X and Y must have shape (k, N)")
    check(lib.s_spmm(pattern.h, _ptr(A), _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)))
    return Y


def norm_est(pattern, A, iters=50, stream=None):
    lam = ctypes.c_double()
    check(lib.s_norm_est(pattern.h, _ptr(A), int(iters), ctypes.byref(lam), _stream(stream)))
    return float(lam.value)


def norm_est_noalloc(pattern, A, iters=50, stream=None):
    """s_norm_est_noalloc: the same estimate with no device allocation during the call."""
    lam = ctypes.c_double()
    check(lib.s_norm_est_noalloc(pattern.h, _ptr(A), int(iters), ctypes.byref(lam), _stream(stream)))
    return float(lam.value)


def funm(pattern, fn, A, F, steps=0, taylor_degree=0, prec="fp64", scale=0.0, squarings=-1, residual=False,
         checkpoints=None, refine=0, stream=None):
    """F = f(A) with f in {"sqrt", "exp", "exp_neg"}; returns the residual for sqrt if asked."""
    code = {"sqrt": S_SQRT, "exp": S_EXP, "exp_neg": S_EXP_NEG}[fn]
    res = ctypes.c_double(-1.0)
    o = FunmOpts(int(steps), int(taylor_degree), PREC[prec] if isinstance(prec, str) else int(prec),
                 float(scale), int(squarings), ctypes.pointer(res) if residual else None,
                 _ptr(checkpoints), int(refine))
    check(lib.s_funm(pattern.h, code, _ptr(A), _ptr(F), ctypes.byref(o), _stream(stream)))
    return float(res.value) if residual else None


def peak_fma(prec="fp32", stream=None):
    """Measured multiply-add rate of the device in flop/s (s_peak_fma)."""
    v = ctypes.c_double()
    check(lib.s_peak_fma(PREC[prec], ctypes.byref(v), _stream(stream)))
    return float(v.value)


def version():
    return lib.s_version().decode()


def sqrt_backward(pattern, steps, c, checkpoints, dF, dA, prec="fp64", stream=None):
    """dA of the Newton-Schulz square root from its checkpoints (double for "fp64", float for
    "fp32")."""
    check(lib.s_funm_sqrt_backward_prec(pattern.h, PREC[prec], int(steps), float(c), _ptr(checkpoints), _ptr(dF),
                                        _ptr(dA), _stream(stream)))
    return dA


def quad_form(pattern, X, z, stream=None):
    out = ctypes.c_double()
    check(lib.s_quad_form(pattern.h, _ptr(X), _ptr(z), ctypes.byref(out), _stream(stream)))
    return float(out.value)


def quad_form_grad(pattern, z, dX, stream=None):
    check(lib.s_quad_form_grad(pattern.h, _ptr(z), _ptr(dX), _stream(stream)))
    return dX
