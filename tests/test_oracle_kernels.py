"""Pins of the oracle's kernels (Sec. 2): the half-integer closed form against the Bessel
definition Eq. (matern) and the familiar p = 0, 1, 2 forms; d/dell by finite differences."""
import numpy as np
import pytest
from scipy.special import gamma, kv

from oracle.kernels import matern_half_integer, matern_half_integer_dell


def matern_bessel(r, nu, ell):
    # Eq. (matern): 2^{1-nu}/Gamma(nu) (sqrt(2nu) r/ell)^nu K_nu(sqrt(2nu) r/ell)
    z = np.sqrt(2 * nu) * r / ell
    return 2 ** (1 - nu) / gamma(nu) * z ** nu * kv(nu, z)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5, 3.5])
@pytest.mark.parametrize("ell", [0.1, 0.3, 1.0])
def test_closed_form_matches_bessel(nu, ell):
    r = np.linspace(1e-3, 3.0, 200)
    np.testing.assert_allclose(matern_half_integer(r, nu, ell), matern_bessel(r, nu, ell), rtol=1e-10, atol=1e-300)


def test_familiar_forms():
    r = np.linspace(0.0, 2.0, 50)
    ell = 0.37
    t = r / ell
    np.testing.assert_allclose(matern_half_integer(r, 0.5, ell), np.exp(-t), rtol=1e-14)
    np.testing.assert_allclose(matern_half_integer(r, 1.5, ell), (1 + np.sqrt(3) * t) * np.exp(-np.sqrt(3) * t),
                               rtol=1e-14)
    np.testing.assert_allclose(matern_half_integer(r, 2.5, ell),
                               (1 + np.sqrt(5) * t + 5 * t * t / 3) * np.exp(-np.sqrt(5) * t), rtol=1e-13)
    assert matern_half_integer(np.array([0.0]), 2.5, ell)[0] == pytest.approx(1.0)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_dell_finite_difference(nu):
    r = np.linspace(0.01, 1.5, 40)
    ell, h = 0.15, 1e-6
    fd = (matern_half_integer(r, nu, ell + h) - matern_half_integer(r, nu, ell - h)) / (2 * h)
    np.testing.assert_allclose(matern_half_integer_dell(r, nu, ell), fd, rtol=1e-6, atol=1e-9)


def test_dell_matern32_closed_form():
    # d/dell of (1 + sqrt3 r/ell) exp(-sqrt3 r/ell) = 3 r^2 / ell^3 exp(-sqrt3 r/ell)
    r = np.linspace(0.0, 1.0, 30)
    ell = 0.15
    np.testing.assert_allclose(matern_half_integer_dell(r, 1.5, ell),
                               3 * r * r / ell ** 3 * np.exp(-np.sqrt(3) * r / ell), rtol=1e-12, atol=1e-300)
