"""The library's host-side scattering helpers against the oracle (CPU: these
functions do no device work).  Direction sets, orientation samples and
weights must agree to rounding; S_1..S_4 and S_ij to 1e-13 relative."""
import math

import numpy as np
import pytest

from oracle import scattering as S


@pytest.fixture(scope="module")
def B():
    from paper_1305_6497_gb300 import build
    build.build()
    from paper_1305_6497_gb300 import binding
    return binding


@pytest.mark.parametrize("x,eta", [(0.05, 1.0), (3.093665, 0.5), (7.5, 0.25), (25.0, 1.0)])
def test_scattering_directions(B, x, eta):
    th, ph, om = B.dda_scattering_directions(x, eta)
    rt, rp, ro = S.scattering_directions(x, eta)
    assert len(th) == len(rt)
    assert np.allclose(th, rt, rtol=0, atol=1e-14)
    assert np.allclose(ph, rp, rtol=0, atol=1e-14)
    assert np.allclose(om, ro, rtol=1e-13, atol=1e-16)
    with pytest.raises(B.DDAError):
        B.dda_scattering_directions(-1.0, 0.5)


def test_mueller_and_amplitude_matrices(B):
    rng = np.random.default_rng(11)
    n = 25
    f = rng.standard_normal((n, 2, 2)) + 1j * rng.standard_normal((n, 2, 2))
    phi = rng.uniform(0, 2 * math.pi, n)
    for e in (np.array([0, 1, 0], complex), np.array([0, 1, 1j]) / math.sqrt(2),
              np.array([0, 0.6, 0.8 * np.exp(0.3j)])):
        Sv, M = B.dda_mueller(f, e, phi)
        e2 = np.cross(np.array([1.0, 0, 0]), np.conj(e))
        for i in range(n):
            ref = S.amplitude_matrix(f[i], e, e2, phi[i])
            assert np.allclose(Sv[i], ref, rtol=1e-13, atol=1e-13)
            Mr = S.mueller_matrix(ref)
            assert np.allclose(M[i], Mr, rtol=1e-12, atol=1e-12 * np.abs(Mr).max())
    with pytest.raises(B.DDAError):
        B.dda_mueller(f, np.array([1.0, 0, 0]), phi)      # e01 along x_LF


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 2, 2), (3, 5, 4), (4, 8, 1)])
def test_orientation_grid(B, n):
    rng = ((0.1, 2.0), (0.2, 2.9), (0.0, math.pi))
    got = B.dda_orientation_grid(rng[0], n[0], rng[1], n[1], rng[2], n[2])
    ref = S.orientation_grid(rng[0], n[0], rng[1], n[1], rng[2], n[2])
    for a, b in zip(got, ref):
        assert np.allclose(a, b, rtol=1e-14, atol=1e-15)
