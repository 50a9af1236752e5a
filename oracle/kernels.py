"""Matern kernels (Sec. 2, Eq. (matern) and the closed form for half-integer smoothness).

Test infrastructure only (see ``oracle/__init__``).
"""
from math import factorial, sqrt

import numpy as np


def matern_half_integer(r, nu, ell):
    """kappa_{p+1/2}(r) for nu = p + 1/2, written out from the half-integer closed form
    of Sec. 2:  exp(-sqrt(2 nu) r / ell) * p!/(2p)! * sum_{q=0}^{p} (p+q)!/(q!(p-q)!)
    * (sqrt(8 nu) r / ell)^{p-q}.

    Pinned against the Bessel-function definition Eq. (matern) (scipy's K_nu) and the
    familiar forms for p = 0, 1, 2 in tests/test_oracle_kernels.py.
    """
    p = int(round(nu - 0.5))
    if abs(p + 0.5 - nu) > 1e-12 or p < 0:
        raise ValueError("nu must be a half integer p + 1/2, p >= 0")
    r = np.asarray(r, dtype=np.float64)
    s = sqrt(8.0 * nu) * r / ell
    acc = np.zeros_like(r)
    for q in range(p + 1):
        acc = acc + factorial(p + q) / (factorial(q) * factorial(p - q)) * s ** (p - q)
    return np.exp(-sqrt(2.0 * nu) * r / ell) * (factorial(p) / factorial(2 * p)) * acc


def matern_half_integer_dell(r, nu, ell):
    """d kappa / d ell of the closed form above, by the chain rule with t = r/ell:
    kappa = f(t), dkappa/dell = f'(t) * (-r / ell^2), f'(t) differentiated term by term.

    Pinned by central finite differences in ell (tests/test_oracle_kernels.py).
    """
    p = int(round(nu - 0.5))
    r = np.asarray(r, dtype=np.float64)
    a = sqrt(2.0 * nu)
    b = sqrt(8.0 * nu)
    t = r / ell
    poly = np.zeros_like(r)
    dpoly = np.zeros_like(r)
    for q in range(p + 1):
        c = factorial(p + q) / (factorial(q) * factorial(p - q)) * b ** (p - q)
        poly = poly + c * t ** (p - q)
        if p - q >= 1:
            dpoly = dpoly + c * (p - q) * t ** (p - q - 1)
    pref = factorial(p) / factorial(2 * p)
    e = np.exp(-a * t)
    dfdt = pref * e * (dpoly - a * poly)
    return dfdt * (-r / ell ** 2)


def kernel_matrix(points, nu, ell, scale=1.0):
    """K = scale * [kappa(|x_i - x_j|)]_{i,j}, Eq. (KernelMatrix); the benchmarks of
    Sec. 5 use scale = 1/N."""
    x = np.asarray(points, dtype=np.float64)
    diff = x[:, None, :] - x[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=-1))
    return scale * matern_half_integer(r, nu, ell)


def kernel_matrix_dell(points, nu, ell, scale=1.0):
    """d K / d ell, entrywise."""
    x = np.asarray(points, dtype=np.float64)
    diff = x[:, None, :] - x[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=-1))
    return scale * matern_half_integer_dell(r, nu, ell)
