"""Inverse square root by the contour-integral quadrature of Eq. (ContInt) (Sec. 4.4
"Matrix functions", after Hale, Higham and Trefethen), in FP64.

Test infrastructure only (see ``oracle/__init__``).

For a symmetric positive definite A with spectrum in [c_lo, c_hi]:

    A^{-1/2} ~ (2 K(m) sqrt(c_lo) / (pi n)) sum_k dn(t_k|m) / cn(t_k|m)^2 (A + w_k^2 I)^{-1},
    w_k = sqrt(c_lo) sn(t_k|m) / cn(t_k|m),   t_k = K(m) (k - 1/2) / n,   m = 1 - c_lo/c_hi,

n quadrature nodes, sn/cn/dn the Jacobian elliptic functions of parameter m.

Reading of the printed formula: its prefactor and node spacing name "E, the complete
elliptic integral of the second kind associated with the parameter c_lo/c_hi".  The rule is
the midpoint rule for (2/pi) int_0^inf (A + w^2 I)^{-1} dw = A^{-1/2} after the substitution
w = sqrt(c_lo) sn(t|m)/cn(t|m), dw = sqrt(c_lo) dn/cn^2 dt, which maps t in [0, K(m)] onto
w in [0, inf) because cn(K(m)|m) = 0.  So the constant is K(m), the complete integral of
the FIRST kind at parameter m = 1 - c_lo/c_hi; with any other constant the sum does not
converge to A^{-1/2}.  The tests pin this reading on scalars.

Each shifted inverse is taken on the pattern S (``selinv.selected_inverse``), so the result
is P_S of the quadrature applied to A; A^{1/2} = A . A^{-1/2} is then the formatted product
P_S(A A^{-1/2}) (Eq. (product)).  The elliptic functions come from scipy.special.
"""
import math

import numpy as np
from scipy.special import ellipj, ellipk

from . import product as _prod
from .selinv import selected_inverse


def nodes(c_lo, c_hi, n):
    """Shifts w_k^2 and weights of the n-node rule for the spectral interval [c_lo, c_hi]."""
    if not (0.0 < c_lo <= c_hi):
        raise ValueError("need 0 < c_lo <= c_hi")
    m = 1.0 - c_lo / c_hi
    Km = float(ellipk(m))
    t = Km * (np.arange(1, n + 1) - 0.5) / n
    sn, cn, dn, _ = ellipj(t, m)
    w2 = c_lo * (sn / cn) ** 2
    wt = 2.0 * Km * math.sqrt(c_lo) / (math.pi * n) * dn / cn ** 2
    return w2, wt


def invsqrt(A, c_lo, c_hi, n):
    """P_S of the quadrature for A^{-1/2}: sum_k wt_k P_S((A + w_k^2 I)^{-1})."""
    w2, wt = nodes(c_lo, c_hi, n)
    Z = A.like()
    for s, c in zip(w2, wt):
        Z.val += c * selected_inverse(A, float(s)).val
    return Z


def sqrt(A, Zinv, nthreads=1):
    """A^{1/2} = P_S(A A^{-1/2}), the formatted product (Eq. (product))."""
    return _prod.mul_masked(A, Zinv, A, nthreads=nthreads)
