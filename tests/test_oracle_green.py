"""Pins for the oracle's interaction tensors (CPU only).

Each test checks the oracle against something other than its own formula: a
finite-difference Hessian of the scalar Green function, the static dipole
field, direct quadrature of the band-limited integral, and symmetries.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import dda

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _fd_hessian(f, r, h):
    H = np.zeros((3, 3), dtype=np.complex128)
    e = np.eye(3)
    for a in range(3):
        for b in range(3):
            def fd(ha, hb):
                return f(r + ha * e[a] + hb * e[b])
            if a == b:
                H[a, a] = (fd(h, 0) - 2 * f(r) + fd(-h, 0)) / (h * h)
            else:
                H[a, b] = (fd(h, h) - fd(h, -h) - fd(-h, h) + fd(-h, -h)) / (4 * h * h)
    return H


def _num_hessian(f, r, h=2e-3):
    """Central-difference Hessian with one Richardson step (error O(h^4))."""
    return (4.0 * _fd_hessian(f, r, h / 2) - _fd_hessian(f, r, h)) / 3.0


@pytest.mark.parametrize("kd", [0.05, 0.3, 1.1])
def test_point_green_is_k2_plus_grad_grad_of_scalar_green(kd):
    rng = np.random.default_rng(1)
    for _ in range(5):
        r = rng.uniform(-4, 4, size=3)
        if np.linalg.norm(r) < 1.0:
            r += 2.0

        def g(x):
            rr = np.linalg.norm(x)
            return np.exp(1j * kd * rr) / rr
        ref = kd * kd * g(r) * np.eye(3) + _num_hessian(g, r)
        G = dda.green_point(r, kd)
        assert np.abs(G - ref).max() < 1e-8 * np.abs(ref).max()


def test_point_green_static_limit_is_dipole_field():
    r = np.array([1.0, -2.0, 0.5])
    rr = np.linalg.norm(r)
    n = r / rr
    static = (3 * np.outer(n, n) - np.eye(3)) / rr ** 3
    assert np.allclose(dda.green_point(r, 1e-9), static, atol=1e-12)


def test_point_green_far_field_is_transverse():
    r = 4000.0 * np.array([0.3, 0.4, np.sqrt(1 - 0.25)])
    kd = 0.7
    rr = np.linalg.norm(r)
    n = r / rr
    far = kd ** 2 * np.exp(1j * kd * rr) / rr * (np.eye(3) - np.outer(n, n))
    G = dda.green_point(r, kd)
    assert np.abs(G - far).max() < 2e-3 * np.abs(far).max()


def test_green_symmetries():
    rng = np.random.default_rng(2)
    r = rng.normal(size=(20, 3)) * 3
    for f in (dda.green_point, dda.green_fcd):
        G = f(r, 0.4)
        assert np.allclose(G, np.swapaxes(G, -1, -2), atol=1e-14)
        assert np.allclose(G, f(-r, 0.4), atol=1e-14)


@pytest.mark.parametrize("kd", [0.1, 0.5, 1.2])
@pytest.mark.parametrize("r", [1.0, 1.7320508, 3.0, 11.3])
def test_filtered_scalar_green_matches_quadrature(kd, r):
    kf = math.pi
    # principal value part: int_0^kF [q sin(qr)/(q+k)] / (q-k) dq
    pv, _ = integrate.quad(lambda q: q * math.sin(q * r) / (q + kd), 0.0, kf,
                           weight="cauchy", wvar=kd, limit=400)
    # outgoing prescription adds i*pi times the residue q sin(qr)/(2q) at q = k
    ref = 2.0 / (math.pi * r) * (pv + 1j * math.pi * math.sin(kd * r) / 2.0)
    g, _, _ = dda.filtered_scalar_green(np.array([r]), kd)
    assert abs(g[0] - ref) < 1e-10 * max(1.0, abs(ref))


def test_filtered_scalar_green_derivatives():
    kd = 0.6
    r = np.array([1.0, 2.3, 7.0])
    h = 1e-4
    g, g1, g2 = dda.filtered_scalar_green(r, kd)
    gp, _, _ = dda.filtered_scalar_green(r + h, kd)
    gm, _, _ = dda.filtered_scalar_green(r - h, kd)
    assert np.allclose(g1, (gp - gm) / (2 * h), rtol=1e-6)
    assert np.allclose(g2, (gp - 2 * g + gm) / h ** 2, rtol=1e-5)


def test_filtered_green_tends_to_point_green_without_filter():
    r = np.array([2.0, 5.0, 9.0])
    kd = 0.4
    g, _, _ = dda.filtered_scalar_green(r, kd, kf=2e5)
    assert np.allclose(g, np.exp(1j * kd * r) / r, atol=3e-5)


def test_fcd_tensor_is_k2_plus_grad_grad_of_filtered_green():
    kd = 0.35
    rng = np.random.default_rng(5)
    for _ in range(4):
        r = rng.uniform(-5, 5, size=3)
        if np.linalg.norm(r) < 1.0:
            r += 2.0

        def g(x):
            return dda.filtered_scalar_green(np.array([np.linalg.norm(x)]), kd)[0][0]
        ref = kd * kd * g(r) * np.eye(3) + _num_hessian(g, r)
        G = dda.green_fcd(r, kd)
        assert np.abs(G - ref).max() < 1e-7 * np.abs(ref).max()
