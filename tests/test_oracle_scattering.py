"""Pins of the oracle's scattering-matrix, angular-average and orientation
machinery (oracle/scattering.py) against the guide's printed values, closed
forms and independent constructions."""
import math

import numpy as np
import pytest

from dda_inputs import targets as tg
from oracle import dda as O
from oracle import scattering as S

DEG = math.pi / 180


# ---- scattering directions (Sec. "Selection of Scattering Angles") ----------------
def test_direction_count_of_the_guide_example():
    """The guide's RCTGLPRSM example (K*AEFF = 3.093665, ETASCA = 0.5) prints
    NAVG = 962 (theta, phi) values."""
    th, ph, om = S.scattering_directions(3.093665, 0.5)
    assert len(th) == 962


@pytest.mark.parametrize("x,eta", [(0.1, 1.0), (3.093665, 0.5), (12.0, 0.3), (40.0, 1.0)])
def test_direction_set_structure_and_weights(x, eta):
    th, ph, om = S.scattering_directions(x, eta)
    assert th[0] == 0.0 and th[-1] == math.pi
    assert np.all(np.diff(th) >= 0)
    assert abs(om.sum() - 4 * math.pi) < 1e-12            # telescoping sum
    # the quadrature of smooth functions: <1> = 1, <cos> = 0 (exact by the
    # symmetric weights), <cos^2> = 1/3 to second order in the theta spacing
    avg = lambda f: np.sum(om * f) / (4 * math.pi)
    assert abs(avg(np.cos(th))) < 1e-12
    h = np.diff(np.unique(th)).max()
    assert abs(avg(np.cos(th) ** 2) - 1 / 3) < 0.15 * h * h
    assert abs(avg(np.sin(th) * np.cos(ph))) < 1e-12
    # forward directions are sampled more densely than backward ones
    dth = np.diff(np.unique(th))
    assert dth[0] < dth[-1]


def test_rayleigh_angular_averages():
    """Rayleigh scattering of unpolarized light: dC/dOmega ~ (1 + cos^2) / 2, so
    <cos> = 0 and <cos^2> = 2/5; a tiny sphere reproduces it, and the integral of
    dC/dOmega equals C_ext - C_abs."""
    occ, comp = tg.sphere(4)
    kd = 0.01
    th, ph, om = S.scattering_directions(kd * O.effective_radius(occ.sum()), 0.2)
    # real m: no absorption, so C_ext - C_abs = C_ext is not a small difference
    r = O.solve_target(occ, comp, [1.5], kd, [1, 0, 0], [0, 1, 0], [0, 1, 0], "LDR",
                       operator="dense", dirs=np.stack([th, ph], 1))
    aeff = O.effective_radius(occ.sum())
    av = [S.angular_averages(r["famp"][1:, :, l], th, ph, om, kd, aeff) for l in range(2)]
    q = 0.5 * (av[0]["Qsca"] + av[1]["Qsca"])
    assert abs(q / np.mean(r["Qsca"]) - 1) < 2e-3
    cos2 = (av[0]["Qsca"] * av[0]["cos2"] + av[1]["Qsca"] * av[1]["cos2"]) / (2 * q)
    g = (av[0]["Qsca"] * av[0]["g"][0] + av[1]["Qsca"] * av[1]["g"][0]) / (2 * q)
    assert abs(cos2 - 0.4) < 2e-3
    assert abs(g) < 1e-3


# ---- amplitude and Mueller matrices ------------------------------------------------
def _stokes(Epar, Eperp):
    """Bohren & Huffman's Stokes parameters of a Jones pair (E_par, E_perp)."""
    return np.array([abs(Epar) ** 2 + abs(Eperp) ** 2, abs(Epar) ** 2 - abs(Eperp) ** 2,
                     2 * (Epar * np.conj(Eperp)).real, -2 * (Epar * np.conj(Eperp)).imag])


def test_mueller_matrix_maps_stokes_vectors():
    """For an amplitude matrix A = [[S2, S3], [S4, S1]] the scattered Jones pair
    is A (E_par, E_perp); its Stokes vector must equal S_ij times the incident
    one, for every incident state (this fixes all 16 formulas)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        Sv = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        M = S.mueller_matrix(Sv)
        A = np.array([[Sv[1], Sv[2]], [Sv[3], Sv[0]]])
        for _ in range(4):
            Ein = rng.standard_normal(2) + 1j * rng.standard_normal(2)
            Eout = A @ Ein
            assert np.allclose(M @ _stokes(*Ein), _stokes(*Eout), rtol=1e-12, atol=1e-12)


def test_amplitude_matrix_against_direct_far_fields():
    """Solve for incident light polarized parallel and perpendicular to the
    scattering plane, take the far field of the dipoles, and project it on
    (theta_hat, -phi_hat): that is the definition of S_1..S_4 (eq. S_ampl_def).
    The four equations applied to f_ml of the (y, z)-polarized solves must give
    the same matrix."""
    occ, comp = tg.ellipsoid(5, 4, 6)
    kd, m = 0.6, 1.4 + 0.1j
    x_lf = np.array([1.0, 0, 0]); y_lf = np.array([0, 1.0, 0])
    flat, pos = O.site_positions(occ)
    for th_s, ph_s in ((30 * DEG, 20 * DEG), (120 * DEG, 250 * DEG)):
        r = O.solve_target(occ, comp, [m], kd, x_lf, y_lf, y_lf, "LDR", operator="dense",
                           dirs=[(th_s, ph_s)])
        Sv = S.amplitude_matrix(r["famp"][1], np.array([0, 1.0, 0]), np.array([0, 0, 1.0]), ph_s)
        e_par = np.array([0, math.cos(ph_s), math.sin(ph_s)])
        e_perp = np.array([0, math.sin(ph_s), -math.cos(ph_s)])
        n, th_hat, ph_hat = O.scattering_frame(x_lf, y_lf, th_s, ph_s)
        cols = []
        for e in (e_par, e_perp):
            ainv = O.site_alpha_inverse(comp.reshape(-1)[flat], [m], "LDR", kd, x_lf, e)
            A = O.dense_matrix(pos, ainv, kd, "LDR")
            P = np.linalg.solve(A, O.incident_field(pos, kd, x_lf, e).reshape(-1)).reshape(-1, 3)
            F = np.sum(P * np.exp(-1j * kd * (pos @ n))[:, None], axis=0)
            Es = kd ** 2 * (F - n * np.dot(n, F))     # E_s r e^{-ikr} in the far zone
            # (E_s.theta, -E_s.phi) = e^{ikr}/(-ikr) A (E_par, E_perp)
            cols.append(-1j * kd * np.array([np.dot(Es, th_hat), -np.dot(Es, ph_hat)]))
        A = np.array(cols).T
        ref = np.array([A[1, 1], A[0, 0], A[0, 1], A[1, 0]])      # S1, S2, S3, S4
        assert np.allclose(Sv, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


# ---- orientation sampling (Sec. "Sampling in Theta, Phi, and beta") ------------------
def test_orientation_samples_quoted_in_the_guide():
    b, t, p, wb, wa = S.orientation_grid((0, 90 * DEG), 2, (0, 90 * DEG), 2, (0, 180 * DEG), 2)
    assert np.allclose(b / DEG, [22.5, 67.5])
    assert np.allclose(p / DEG, [45, 135])
    assert np.allclose(t / DEG, [41.41, 75.52], atol=5e-3)       # cos = 0.75, 0.25
    _, t3, _, _, wa3 = S.orientation_grid((0, 0), 1, (0, 90 * DEG), 3, (0, 0), 1)
    assert np.allclose(t3 / DEG, [0, 60, 90])
    # Simpson over cos(Theta): weights 1/3, 4/3, 1/3 normalised to unit sum
    assert np.allclose(wa3[:, 0], np.array([1, 4, 1]) / 6)
    assert abs(wb.sum() - 1) < 1e-15 and abs(wa.sum() - 1) < 1e-15
    # Simpson integrates cos^3 over cos(Theta) in [-1, 1] exactly (odd -> 0), cos^2 -> 1/3
    _, t5, _, _, wa5 = S.orientation_grid((0, 0), 1, (0, math.pi), 5, (0, 0), 1)
    assert abs(np.sum(wa5[:, 0] * np.cos(t5) ** 2) - 1 / 3) < 1e-12


def test_lab_axes_are_a_right_handed_orthonormal_frame():
    rng = np.random.default_rng(0)
    for _ in range(10):
        th, ph, be = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
        x, y, z = S.lab_axes(th, ph, be)
        R = np.array([x, y, z])
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.allclose(np.cross(x, y), z, atol=1e-14)
        # a1 = x_TF makes the angle Theta with x_LF
        assert abs(x[0] - math.cos(th)) < 1e-14
    # Phi turns the Lab frame about x_LF: y(Phi) = y(0) cos - z(0) sin
    x0, y0, z0 = S.lab_axes(0.7, 0.0, 0.3)
    x1, y1, z1 = S.lab_axes(0.7, 0.4, 0.3)
    assert np.allclose(x1, x0) and np.allclose(y1, y0 * math.cos(0.4) - z0 * math.sin(0.4))


def test_orientation_average_of_single_orientation_is_the_solve():
    occ, comp = tg.ellipsoid(5, 6, 4)
    grid = ((0, 0), 1, (0, 0), 1, (0, 0), 1)
    av = S.orientation_average(occ, comp, [1.5 + 0.1j], 0.5, grid, eta=1.0,
                               sel=[(0.0, 0.0), (math.pi, 0.0)])
    r = O.solve_target(occ, comp, [1.5 + 0.1j], 0.5, [1, 0, 0], [0, 1, 0], [0, 1, 0], "LDR")
    assert np.allclose(av["Qext"], r["Qext"], rtol=1e-9)
    assert np.allclose(av["Qsca"], r["Qsca"], rtol=1e-9)
    # S_11(0) for unpolarized light = (|f11|^2 + |f21|^2 + |f12|^2 + |f22|^2) / 2
    f0 = r["famp"][0]
    assert abs(av["mueller"][0][0, 0] / (0.5 * np.sum(np.abs(f0) ** 2)) - 1) < 1e-9
    # Q_bk is dC/dOmega(pi) / (pi a^2) = S_11(180) / (pi x^2) (unpolarized)
    x = 0.5 * O.effective_radius(occ.sum())
    assert abs(np.mean(av["Qbk"]) / (av["mueller"][1][0, 0] / (math.pi * x * x)) - 1) < 1e-9


def test_q_bk_reading_reproduces_the_guide_table():
    """The guide prints Q_bk = 0.61831 and S_11(180) = 18.591 at x = 3.093665:
    Q_bk = S_11(180)/(pi x^2)."""
    assert abs(18.591 / (math.pi * 3.093665 ** 2) / 0.61831 - 1) < 1e-4


def test_guide_worked_example_angular_quantities():
    """RCTGLPRSM (Appendix w000r000ori.avg): g(1) = 0.41463, <cos^2> = 0.75169,
    Q_bk = 0.61831, Q_pha = -0.12614, S_12(20 deg) = -5.1645, S_11(90) = 1.1878.
    The guide used GKDLDR; the oracle has LATTDR, so agreement is at the
    percent level (the two prescriptions agree for |m| k d < 0.5)."""
    occ, comp = tg.rect_prism(16, 32, 32)
    kd = 3.093665 * 0.06346821
    m = 0.9656 + 1.8628j
    grid = ((0, 0), 1, (0, 0), 1, (0, 0), 1)
    av = S.orientation_average(occ, comp, [m], kd, grid, eta=0.5, tol=1e-7,
                               sel=[(20 * DEG, 0.0), (90 * DEG, 0.0), (90 * DEG, 90 * DEG)])
    assert av["n_sca"] == 962
    g = np.mean(av["g"][:, 0])
    assert abs(g / 0.41463 - 1) < 0.02
    assert abs(np.mean(av["cos2"]) / 0.75169 - 1) < 0.02
    assert abs(np.mean(av["Qbk"]) / 0.61831 - 1) < 0.03
    # Q_pha is Re f(0) on the scale of Q_ext (Im f(0)): compare on that scale
    assert abs(np.mean(av["Qpha"]) - (-0.12614)) < 0.005 * 3.6134
    # the direction quadrature is second order in the theta spacing: at eta = 0.5
    # its C_sca is within 2% of C_ext - C_abs (the normalised averages above,
    # ratios of two such sums, are far more accurate)
    assert abs(np.mean(av["Qsca_int"]) / np.mean(av["Qsca"]) - 1) < 0.02
    # S_12 is a difference of the two polarized intensities: compare it on the
    # scale of S_11(20 deg) = 39.245
    assert abs(av["mueller"][0][0, 0] / 39.245 - 1) < 0.03
    assert abs(av["mueller"][0][0, 1] - (-5.1645)) < 0.01 * 39.245
    assert abs(av["mueller"][1][0, 0] / 1.1878 - 1) < 0.03
    assert abs(av["mueller"][2][0, 0] / 1.1878 - 1) < 0.03
