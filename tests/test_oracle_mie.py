"""Pins for the oracle's Mie series (CPU only): coefficients against scipy's
spherical Bessel functions (the textbook formula, evaluated independently of
the recurrences), the Rayleigh limit, no absorption for real m, and the
extinction paradox (Q_ext -> 2) for large spheres."""
import numpy as np
import pytest
from scipy import special

from oracle import mie


def _coeffs_scipy(m, x, nmax):
    n = np.arange(1, nmax + 1)
    mx = m * x

    def psi(z):
        return z * special.spherical_jn(n, z)

    def dpsi(z):
        return special.spherical_jn(n, z) + z * special.spherical_jn(n, z, derivative=True)

    def xi(z):
        return z * (special.spherical_jn(n, z) + 1j * special.spherical_yn(n, z))

    def dxi(z):
        h = special.spherical_jn(n, z) + 1j * special.spherical_yn(n, z)
        dh = (special.spherical_jn(n, z, derivative=True)
              + 1j * special.spherical_yn(n, z, derivative=True))
        return h + z * dh

    a = (m * psi(mx) * dpsi(x) - psi(x) * dpsi(mx)) / (m * psi(mx) * dxi(x) - xi(x) * dpsi(mx))
    b = (psi(mx) * dpsi(x) - m * psi(x) * dpsi(mx)) / (psi(mx) * dxi(x) - m * xi(x) * dpsi(mx))
    return a, b


@pytest.mark.parametrize("m,x", [(1.33 + 0.01j, 1.0), (1.5 + 0.02j, 5.0),
                                 (1.7 + 0.1j, 8.0), (1.33 + 0.01j, 25.0),
                                 (0.9656 + 1.8628j, 3.09)])
def test_coefficients_match_spherical_bessel_formula(m, x):
    a, b = mie.mie_coefficients(m, x)
    ar, br = _coeffs_scipy(m, x, len(a))
    assert np.allclose(a, ar, rtol=1e-9, atol=1e-13)
    assert np.allclose(b, br, rtol=1e-9, atol=1e-13)


def test_rayleigh_limit():
    m, x = 1.33 + 0.05j, 0.01
    qe, qa, qs = mie.mie_q(m, x)
    K = (m * m - 1) / (m * m + 2)
    assert abs(qa / (4 * x * K.imag) - 1) < 1e-3
    assert abs(qs / (8 / 3 * x ** 4 * abs(K) ** 2) - 1) < 1e-3


@pytest.mark.parametrize("x", [0.5, 3.0, 12.0])
def test_real_index_does_not_absorb(x):
    qe, qa, qs = mie.mie_q(1.5, x)
    assert abs(qa) < 1e-12 * qe


def test_extinction_paradox():
    """Q_ext -> 2 for large spheres, the excess falling roughly as x^(-2/3)."""
    dev = [abs(mie.mie_q(1.33 + 0.1j, x)[0] - 2.0) for x in (100.0, 400.0, 1600.0)]
    assert dev[0] > dev[1] > dev[2]
    assert dev[2] < 0.02
