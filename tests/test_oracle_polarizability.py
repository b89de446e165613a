"""Pins for the oracle's polarizabilities (CPU only).

The guide prints alpha_CM and the FLTRCD correction (Sec. "Filtered Coupled
Dipole"); LATTDR's and GKDLDR's coefficients come from cited papers (they are
derived from the lattice's dipole sum in test_oracle_lattice_dispersion.py).
What the physics fixes independently of those formulas: every prescription
tends to Clausius-Mossotti as kd -> 0; a lossless material (real m) absorbs
nothing, so -Im(1/alpha) - (2/3) k^3 = 0 on every axis (the per-dipole
absorption weight of C_abs); a lossy one absorbs (weight > 0); and a physical
response obeys alpha(-k) = conj(alpha(k)) for real m.  Every check runs on the
diagonal of the polarizability tensor (the scalar methods repeat alpha on it).
"""
import math

import numpy as np
import pytest

from oracle import dda

KH = np.array([1.0, 0.0, 0.0])
EY = np.array([0.0, 1.0, 0.0])


def absorption_weight(alpha, kd):
    return -np.imag(1.0 / alpha) - (2.0 / 3.0) * kd ** 3


def test_alpha_cm_limits():
    assert dda.alpha_cm(1.0) == 0.0
    assert abs(dda.alpha_cm(1e8) - 3.0 / (4.0 * math.pi)) < 1e-12
    # eps = m^2 -> the (eps-1)/(eps+2) form
    m = 1.7 + 0.1j
    eps = m * m
    assert abs(dda.alpha_cm(m) - 3 / (4 * math.pi) * (eps - 1) / (eps + 2)) < 1e-15


@pytest.mark.parametrize("method", dda.METHODS)
@pytest.mark.parametrize("m", [1.33 + 0.01j, 1.7 + 0.1j, 0.9656 + 1.8628j])
def test_static_limit_is_clausius_mossotti(method, m):
    a = dda.polarizability_tensor(method, m, 1e-6, np.array([0.36, 0.48, 0.8]), EY)
    assert np.all(np.abs(a / dda.alpha_cm(m) - 1.0) < 1e-9)


@pytest.mark.parametrize("method", dda.METHODS)
@pytest.mark.parametrize("m", [1.2, 1.5, 2.0, 3.0])
@pytest.mark.parametrize("kd", [0.05, 0.2, 0.6])
def test_lossless_material_does_not_absorb(method, m, kd):
    for e in (EY, np.array([0.0, 0.6, 0.8]), np.array([0, 1, 1j]) / math.sqrt(2)):
        a = dda.polarizability_tensor(method, m, kd, np.array([0.6, 0.8, 0.0]), e)
        assert np.all(np.abs(absorption_weight(a, kd)) < 1e-13 * np.abs(1.0 / a))


@pytest.mark.parametrize("method", dda.METHODS)
@pytest.mark.parametrize("m", [1.33 + 0.01j, 1.7 + 0.1j, 0.9656 + 1.8628j])
def test_lossy_material_absorbs(method, m):
    a = dda.polarizability_tensor(method, m, 0.3, np.array([0.6, 0.0, 0.8]), EY)
    assert np.all(absorption_weight(a, 0.3) > 0.0)


@pytest.mark.parametrize("method", dda.METHODS)
def test_reality_condition(method):
    for kd in (0.1, 0.4, 0.9):
        kh = np.array([0.6, 0.0, 0.8])
        ap = dda.polarizability_tensor(method, 1.6, kd, kh, EY)
        am = dda.polarizability_tensor(method, 1.6, -kd, kh, EY)
        assert np.all(np.abs(am - np.conj(ap)) < 1e-14 * np.abs(ap))


def test_literal_fltrcd_formula_fails_the_physical_pins():
    """The FLTRCD expression as printed ("1 + D", no (kd)^3 on the log) gives
    negative absorption for real m and breaks alpha(-k) = conj(alpha(k)); this is
    why the oracle adopts the sign-corrected, (kd)^3-weighted reading."""
    def literal(m, kd):
        a0 = dda.alpha_cm(m)
        D = a0 * ((4 / 3) * kd ** 2 + (2 / (3 * math.pi)) * math.log((math.pi - kd) / (math.pi + kd))
                  + (2 / 3) * 1j * kd ** 3)
        return a0 / (1 + D)
    assert absorption_weight(literal(1.5, 0.3), 0.3) < 0.0
    assert abs(literal(1.5, -0.3) - np.conj(literal(1.5, 0.3))) > 1e-3 * abs(literal(1.5, 0.3))


def test_ldr_s_factor():
    assert dda.ldr_s(KH, EY) == 0.0
    kh = np.ones(3) / math.sqrt(3)
    e = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
    assert abs(dda.ldr_s(kh, e) - 1.0 / 3.0) < 1e-15


def test_gkdldr_equals_ldr_on_the_axes_of_a_linear_polarization():
    """For a wave along a lattice axis with e along another, GKDLDR's alpha on
    the two transverse axes equals LATTDR's (S = 0 = khat_a^2 there); along the
    propagation axis it differs (khat_x^2 = 1)."""
    m, kd = 1.5 + 0.2j, 0.25
    a = dda.polarizability_tensor("GKDLDR", m, kd, KH, EY)
    ldr = dda.polarizability("LDR", m, kd, KH, EY)
    assert abs(a[1] / ldr - 1) < 1e-15 and abs(a[2] / ldr - 1) < 1e-15
    assert abs(a[0] / ldr - 1) > 1e-3
    with pytest.raises(ValueError):
        dda.polarizability("GKDLDR", m, kd, KH, EY)
