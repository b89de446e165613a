"""The lattice dispersion relation pins LATTDR's coefficients and GKDLDR's form.

The guide's point-dipole prescriptions (Sec. "Point Dipoles: Options LATTDR and
GKDLDR") choose alpha so that an infinite cubic lattice of polarizable points
carries a plane wave exactly as a continuum of refractive index m would: the
dipoles P_j = P exp(i q . r_j), q = m k khat, must reproduce themselves,

    (1/alpha) P = T(k, q) P,    T = sum_{j != 0} G(r_j) exp(i q . r_j),

with G the point-dipole tensor (k^2 + grad grad) e^{ikr}/r.  The sum converges
only conditionally; here it is evaluated by Ewald summation (the lattice sum
split into a real-space part with erfc screening and a reciprocal-lattice part
with Gaussian factors), written in this file from that textbook method and
independent of the oracle's polarizability formulas.  The test checks the
summation itself (the result does not depend on the splitting parameter; the
imaginary part is exactly -(2/3) k^3, the radiation reaction, because no Bragg
order radiates for q > k), then takes the small-k expansion of
T - 4 pi (k^2 I - q q)/(q^2 - k^2) (the long-wavelength pole removed):
    constant term      = (4 pi / 3) I            (the Lorentz field)
    (kd)^2 term, projected on the plane normal to khat
                       = (b1 + m^2 b2) I + m^2 b3 diag(khat_a^2)
and compares b1, b2, b3 with the oracle's LATTDR constants.  The same
expansion shows why a scalar alpha can match only one polarization for a
general direction (LATTDR's S = e . diag(khat_a^2) . e), and that the tensor
diagonal on the lattice axes with khat_a^2 in place of S (the oracle's
GKDLDR) matches the lattice for every transverse polarization.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import dda

SQPI = math.sqrt(math.pi)


def lattice_sum(k, q, E=SQPI, nmax=6):
    """T(k, q) = sum over the unit cubic lattice minus the origin of
    G(r_j) exp(i q . r_j), by Ewald summation with splitting parameter E.

    Real space: the screened Green function
        g_R(r) = [e^{ikr} erfc(E r + i a) + e^{-ikr} erfc(E r - i a)] / (2 r),
    a = k / (2E), written with Faddeeva's w(z) = e^{-z^2} erfc(-iz), so that
    e^{ikr} erfc(E r + i a) = e^{a^2 - E^2 r^2} w(-a + i E r).  Reciprocal
    space: the smooth remainder g - g_R has the Fourier transform
    4 pi exp((k^2 - p^2) / (4 E^2)) / (p^2 - k^2), summed at p = q + G.  The
    origin's screened remainder g - g_R = c0 + c2 r^2 + ... is removed
    analytically: (k^2 + grad grad)(c0 + c2 r^2) = (k^2 c0 + 2 c2) I."""
    q = np.asarray(q, dtype=np.float64)
    a = k / (2.0 * E)
    r1 = np.arange(-nmax, nmax + 1)
    X, Y, Z = np.meshgrid(r1, r1, r1, indexing="ij")
    R = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    R = R[np.any(R != 0, axis=1)]
    r = np.linalg.norm(R, axis=1)
    n = R / r[:, None]
    screen = np.exp(a * a - E * E * r * r)
    wp = special.wofz(-a + 1j * E * r)
    wm = special.wofz(a + 1j * E * r)
    # w(r) = 2 r g_R(r) and its r-derivatives (w'' from the Helmholtz equation)
    w0 = screen * (wp + wm)
    w1 = 1j * k * screen * (wp - wm) - (4.0 * E / SQPI) * screen
    w2 = -k * k * w0 + (8.0 * E ** 3 * r / SQPI) * screen
    g = w0 / (2 * r)
    g1 = w1 / (2 * r) - w0 / (2 * r * r)
    g2 = w2 / (2 * r) - w1 / r ** 2 + w0 / r ** 3
    eye = np.eye(3)
    nn = n[:, :, None] * n[:, None, :]
    # grad grad of a radial function: n n g'' + (I - n n) g'/r
    H = (k * k * g + g1 / r)[:, None, None] * eye + (g2 - g1 / r)[:, None, None] * nn
    T = np.einsum("j,jab->ab", np.exp(1j * (R @ q)), H)
    # the origin: (g - g_R)(r) = u(r) / (2r), u = 2 e^{ikr} - w, u(0) = 0
    ea = math.exp(a * a)
    erfi = special.erfi(a)
    w1_0 = 2.0 * k * erfi - (4.0 * E / SQPI) * ea
    c0 = 0.5 * (2j * k - w1_0)
    c2 = (-2j * k ** 3 + k * k * w1_0 - (8.0 * E ** 3 / SQPI) * ea) / 12.0
    T -= (k * k * c0 + 2.0 * c2) * eye
    # reciprocal lattice (2 pi Z^3, unit cell volume 1)
    p = q[None, :] + 2.0 * math.pi * np.vstack([np.zeros(3), R])
    p2 = np.sum(p * p, axis=1)
    f = 4.0 * math.pi * np.exp((k * k - p2) / (4.0 * E * E)) / (p2 - k * k)
    T += np.einsum("j,jab->ab", f, k * k * eye[None] - p[:, :, None] * p[:, None, :])
    return T


def pole(k, q):
    """The long-wavelength term of the reciprocal sum (G = 0, no Gaussian)."""
    return 4.0 * math.pi * (k * k * np.eye(3) - np.outer(q, q)) / (q @ q - k * k)


def expansion(m, khat, ks=(0.01, 0.02, 0.03, 0.04, 0.05)):
    """Constant and (kd)^2 coefficients of Re[T - pole] along q = m k khat
    (even in k: least squares in 1, k^2, k^4, k^6)."""
    khat = np.asarray(khat, np.float64) / np.linalg.norm(khat)
    A, V = [], []
    for k in ks:
        q = m * k * khat
        V.append((lattice_sum(k, q) - pole(k, q)).real.ravel())
        A.append([1.0, k ** 2, k ** 4, k ** 6])
    coef = np.linalg.lstsq(np.array(A), np.array(V), rcond=None)[0]
    return coef[0].reshape(3, 3), coef[1].reshape(3, 3)


def transverse(khat):
    khat = np.asarray(khat, np.float64) / np.linalg.norm(khat)
    return np.eye(3) - np.outer(khat, khat)


CASES = [(1.5, (1, 0, 0)), (1.33, (1, 2, 3)), (2.0, (0.3, -0.5, 0.8)), (1.7, (1, 1, 1)),
         (1.2, (0, 0.6, 0.8))]


def test_ewald_sum_does_not_depend_on_the_splitting():
    for m, kh in CASES[:3]:
        kh = np.asarray(kh, float) / np.linalg.norm(kh)
        k = 0.07
        ref = lattice_sum(k, m * k * kh)
        for E in (0.8 * SQPI, 1.3 * SQPI):
            assert np.abs(lattice_sum(k, m * k * kh, E) - ref).max() < 1e-12 * np.abs(ref).max()


def test_radiation_reaction_is_the_imaginary_part():
    for m, kh in CASES:
        kh = np.asarray(kh, float) / np.linalg.norm(kh)
        for k in (0.02, 0.1, 0.3):
            T = lattice_sum(k, m * k * kh)
            assert np.abs(T.imag + (2.0 / 3.0) * k ** 3 * np.eye(3)).max() < 1e-13


def test_static_term_is_the_lorentz_field():
    for m, kh in CASES:
        T0, _ = expansion(m, kh)
        assert np.abs(T0 - (4.0 * math.pi / 3.0) * np.eye(3)).max() < 1e-10


def test_ldr_coefficients_from_the_dispersion_relation():
    """Least squares for (b1, b2, b3) over several m and directions from the
    transverse (kd)^2 term; they equal the oracle's LATTDR constants to the
    digits those carry, and the fitted form leaves no residual."""
    rows, rhs = [], []
    for m, kh in CASES:
        kh = np.asarray(kh, float) / np.linalg.norm(kh)
        P = transverse(kh)
        _, C2 = expansion(m, kh)
        got = P @ C2 @ P
        basis = [P @ np.eye(3) @ P, m * m * P @ np.eye(3) @ P, m * m * P @ np.diag(kh ** 2) @ P]
        rows.append(np.stack([b.ravel() for b in basis], axis=1))
        rhs.append(got.ravel())
    A, y = np.vstack(rows), np.concatenate(rhs)
    b, *_ = np.linalg.lstsq(A, y, rcond=None)
    assert np.abs(A @ b - y).max() < 1e-7
    assert abs(b[0] - dda.LDR_B1) < 2e-7
    assert abs(b[1] - dda.LDR_B2) < 2e-7
    assert abs(b[2] - dda.LDR_B3) < 2e-7


@pytest.mark.parametrize("m,kh", CASES)
def test_gkdldr_matches_the_lattice_for_every_polarization(m, kh):
    """Transverse block of d^3/alpha - T: GKDLDR's tensor leaves only O(k^4)
    (the relation holds for both polarizations), while LATTDR's scalar alpha,
    built for one polarization e1, leaves an O(k^2) coupling to the other one
    whenever the direction is not along a lattice axis or diagonal plane."""
    kh = np.asarray(kh, float) / np.linalg.norm(kh)
    P = transverse(kh)
    e1 = np.cross(kh, [0.31, 0.17, 0.93])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(kh, e1)
    worst_gkd, worst_ldr = [], []
    for k in (0.02, 0.04):
        T = lattice_sum(k, m * k * kh)
        ginv = np.diag(1.0 / dda.polarizability_tensor("GKDLDR", m, k, kh))
        lin = 1.0 / dda.polarizability("LDR", m, k, kh, e1) * np.eye(3)
        worst_gkd.append(np.abs(P @ (ginv - T) @ P).max() / k ** 2)
        worst_ldr.append(abs(e2 @ (lin - T) @ e1) / k ** 2)
        # LATTDR does satisfy the relation for its own polarization
        assert abs(e1 @ (lin - T) @ e1) / k ** 2 < 0.01
    assert worst_gkd[1] < 0.01 and worst_gkd[1] > 3.0 * worst_gkd[0] * 0.9  # O(k^4)
    aniso = np.abs(P @ np.diag(kh ** 2) @ P - (e1 @ np.diag(kh ** 2) @ e1) * P).max()
    if aniso > 1e-3:
        assert worst_ldr[0] > 0.05 * m * m * abs(dda.LDR_B3) * aniso
