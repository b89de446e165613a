"""Mie series for a homogeneous sphere -- TEST INFRASTRUCTURE ONLY (CPU oracle).

The DDSCAT 7.3 guide measures the DDA against exact Mie results for spheres
(Sec. "Applicability of the DDA", Figs. 1-2) and uses the Bohren & Huffman
(1983) conventions for the amplitude matrix.  This module evaluates the
standard series

    Q_ext = (2/x^2) sum_n (2n+1) Re(a_n + b_n)
    Q_sca = (2/x^2) sum_n (2n+1) (|a_n|^2 + |b_n|^2),   Q_abs = Q_ext - Q_sca

with the Riccati-Bessel functions psi_n(x) = x j_n(x), xi_n(x) = x h_n^(1)(x)
from upward recurrence and the logarithmic derivative D_n(mx) = psi_n'/psi_n
(mx) from downward recurrence, which stays stable for absorbing spheres.  The
series stops at n = x + 4 x^(1/3) + 2 (Wiscombe's rule).
"""
from __future__ import annotations

import math

import numpy as np


def mie_coefficients(m: complex, x: float):
    """(a_n, b_n) for n = 1..nstop."""
    m = complex(m)
    x = float(x)
    nstop = int(x + 4.0 * x ** (1.0 / 3.0) + 2.0)
    mx = m * x
    nmx = int(max(nstop, abs(mx))) + 16
    D = np.zeros(nmx + 1, dtype=np.complex128)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi_prev, psi = math.cos(x), math.sin(x)         # psi_{-1}, psi_0
    chi_prev, chi = -math.sin(x), math.cos(x)        # chi_{-1}, chi_0 (xi = psi - i chi)
    a = np.zeros(nstop, dtype=np.complex128)
    b = np.zeros(nstop, dtype=np.complex128)
    for n in range(1, nstop + 1):
        psi_n = (2 * n - 1) / x * psi - psi_prev
        chi_n = (2 * n - 1) / x * chi - chi_prev
        xi_n = psi_n - 1j * chi_n
        xi_nm1 = psi - 1j * chi
        ta = D[n] / m + n / x
        tb = m * D[n] + n / x
        a[n - 1] = (ta * psi_n - psi) / (ta * xi_n - xi_nm1)
        b[n - 1] = (tb * psi_n - psi) / (tb * xi_n - xi_nm1)
        psi_prev, psi = psi, psi_n
        chi_prev, chi = chi, chi_n
    return a, b


def mie_q(m: complex, x: float):
    """(Q_ext, Q_abs, Q_sca) of a sphere with size parameter x = k a."""
    a, b = mie_coefficients(m, x)
    n = np.arange(1, len(a) + 1)
    qext = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * np.real(a + b)))
    qsca = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2)))
    return qext, qext - qsca, qsca
