"""Input generators against the numbers the DDSCAT guide prints (CPU only).

Pseudosphere dipole counts (Sec. "ELLIPSOID" examples and the Mie comparison
figures): N = 304, 17904, 59728 for spheres filling 8^3, 32^3, 48^3 boxes;
derived scalars |m| k d; orientation formulas and sampling rules (Sec. "Target
Orientation" and "Sampling in Theta, Phi, and beta")."""
import math

import numpy as np
import pytest

from dda_inputs import orientation as ori
from dda_inputs import targets as tg
from dda_inputs import workloads as W


@pytest.mark.parametrize("n,N", [(8, 304), (32, 17904), (48, 59728)])
def test_guide_pseudosphere_counts(n, N):
    occ, _ = tg.sphere(n, n + 0.49)
    assert int(occ.sum()) == N


def test_workload_sizes():
    assert W.c1_sphere16().n_dipoles == 2176
    assert W.c2_sphere64().n_dipoles == 137376
    c3 = W.c3_ellipsoid()
    assert c3.n_dipoles == 347432 and c3.n_rhs == 64
    assert abs(W.c1_sphere16().kd - 0.12440) < 5e-5
    assert abs(W.c2_sphere64().kd - 0.15621) < 5e-5
    assert abs(c3.kd - 0.18344) < 5e-5


def test_guide_mkd_values():
    # ELLIPSOID example: 59728 dipoles, m = 1.5+0.01i, x = 5 -> |m|kd = 0.309
    kd = W.kd_for_size_parameter(5.0, 59728)
    assert abs(abs(1.5 + 0.01j) * kd - 0.309) < 5e-4
    # Appendix: N = 16384 -> d/aeff = 0.06346821
    assert abs(1.0 / tg.effective_radius(16384) - 0.06346821) < 1e-8


def test_orientation_examples_from_guide():
    d = math.radians
    a1, a2, a3 = ori.target_axes_in_lab_frame(d(90), 0.0, 0.0)
    assert np.allclose(a1, [0, 1, 0]) and np.allclose(a2, [-1, 0, 0])
    a1, a2, a3 = ori.target_axes_in_lab_frame(d(90), 0.0, d(90))
    assert np.allclose(a1, [0, 1, 0]) and np.allclose(a2, [0, 0, 1])
    x, y, z = ori.lab_axes_in_target_frame(d(54.7356), d(30), d(135))
    assert np.allclose(x, np.array([1, 1, 1]) / math.sqrt(3), atol=1e-6)
    assert np.allclose(y, np.array([1, -1, 0]) / math.sqrt(2), atol=1e-6)
    assert np.allclose(z, np.array([1, 1, -2]) / math.sqrt(6), atol=1e-6)


def test_forward_and_inverse_orientation_agree():
    rng = np.random.default_rng(0)
    for (t, p, b) in ori.random_orientations(rng, 10):
        A = np.array(ori.target_axes_in_lab_frame(t, p, b))   # rows a_i in LF
        L = np.array(ori.lab_axes_in_target_frame(t, p, b))   # rows LF axes in TF
        assert np.allclose(A @ A.T, np.eye(3), atol=1e-14)
        assert np.allclose(L, A.T, atol=1e-14)
        assert np.allclose(np.cross(L[0], L[1]), L[2], atol=1e-14)


def test_sampling_rules():
    assert np.allclose(np.degrees(ori.sample_beta(0, math.pi / 2, 2)), [22.5, 67.5])
    assert np.allclose(np.degrees(ori.sample_theta(0, math.pi / 2, 3)), [0, 60, 90])
    assert np.allclose(np.degrees(ori.sample_theta(0, math.pi / 2, 2)), [41.41, 75.52],
                       atol=5e-3)


def test_serving_stream_is_seeded_and_valid():
    a = W.serving_stream(n_requests=12)
    b = W.serving_stream(n_requests=12)
    for ra, rb in zip(a, b):
        assert ra["t_arrival"] == rb["t_arrival"] and np.array_equal(ra["occ"], rb["occ"])
        N = int(ra["occ"].sum())
        assert 900 <= N <= 1.1e6
        assert abs(ra["m"][0]) * ra["kd"] <= 1.0 + 1e-9
