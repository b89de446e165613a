"""Pins of the oracle's near field (Sec. "Near-Field Calculations").

* At target sites an exact solution satisfies P_j = alpha_j (E_inc + E_sca)_j
  (the identity the guide gives for its .E files), checked against the dense
  LU solve of A P = E.
* A single dipole radiates the textbook dipole field (Jackson's form, written
  out here independently of the oracle's tensor).
* In the quasi-static limit the macroscopic field inside a dielectric sphere is
  uniform, 3/(eps + 2) E_0, and far outside a small target the field is that of
  its total dipole moment.
* The extended box follows the r1..r6 definition with rounding to nearest.
"""
import math
import os
import sys

import numpy as np
import pytest

from dda_inputs import targets as tg
from dda_inputs import workloads as W
from oracle import dda as O

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def test_extended_box_definition():
    assert O.nearfield_box((7, 6, 5), [0] * 6) == ((5, 6, 7), (0, 0, 0))
    # n_x = 5: 0.5*5 = 2.5 -> 3 (halves away from zero), 0.2*5 = 1
    assert O.nearfield_box((7, 6, 5), [0.5, 0.2, 0, 1, 0.25, 0]) == ((9, 12, 9), (3, 0, 2))


@pytest.mark.parametrize("method", ["LDR", "CM", "FCD"])
def test_identity_at_target_sites(method):
    w = W.small_ellipsoid(5, 6, 4, m=1.6 + 0.2j, kd=0.5, method=method)
    ref = O.solve_target(w.occ, w.comp, w.m, w.kd, w.khat[0], w.yhat[0], w.e01[0], method,
                         npol=1, operator="dense")
    e1, _ = O.polarization_pair(w.khat[0], w.e01[0])
    P = ref["P"][0]
    nf = O.nearfield(w.occ, w.comp, w.m, w.kd, w.khat[0], e1, method, P, [0.4, 0.6, 0.3, 0.2, 0.5, 0.5])
    (nx, ny, nz), (lx, ly, lz) = nf["dims"], nf["lo"]
    flat, pos = O.site_positions(w.occ)
    tz, ty, tx = w.occ.shape
    ix, iy, iz = flat % tx, (flat // tx) % ty, flat // (tx * ty)
    etot = (nf["E_inc"] + nf["E_sca"])[:, iz + lz, iy + ly, ix + lx].T
    ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, method, w.kd, w.khat[0], e1)
    assert np.abs(P - etot / ainv[:, None]).max() < 1e-10 * np.abs(P).max()
    # the incident field at the target sites is the solve's right-hand side
    assert np.allclose(nf["E_inc"][:, iz + lz, iy + ly, ix + lx].T,
                       O.incident_field(pos, w.kd, w.khat[0], e1), rtol=0, atol=1e-14)
    # vacuum sites carry the microscopic field unchanged
    vac = nf["comp"] == 0
    em = nf["E_macro"].reshape(3, -1)[:, vac]
    assert np.array_equal(em, (nf["E_inc"] + nf["E_sca"]).reshape(3, -1)[:, vac])


def test_single_dipole_field_is_the_textbook_dipole_field():
    occ = np.ones((1, 1, 1), np.uint8)
    comp = occ.copy()
    kd = 0.7
    p = np.array([[0.3 + 0.1j, -0.2j, 0.5]])
    nf = O.nearfield(occ, comp, [1.5], kd, [1, 0, 0], [0, 1, 0], "CM", p, [3, 2, 2, 3, 1, 2])
    (nx, ny, nz), (lx, ly, lz) = nf["dims"], nf["lo"]
    pv = p[0]
    worst = 0.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                r = np.array([x - lx, y - ly, z - lz], float)
                rr = np.linalg.norm(r)
                E = nf["E_sca"][:, z, y, x]
                if rr == 0:
                    assert np.all(E == 0)
                    continue
                n = r / rr
                ref = np.exp(1j * kd * rr) * (
                    kd ** 2 * np.cross(np.cross(n, pv), n) / rr
                    + (3 * n * np.dot(n, pv) - pv) * (1 / rr ** 3 - 1j * kd / rr ** 2))
                worst = max(worst, np.abs(E - ref).max() / np.abs(ref).max())
    assert worst < 1e-12


def test_quasistatic_sphere_internal_field_is_uniform_3_over_eps_plus_2():
    n = 16
    occ, comp = tg.sphere(n)
    m = 1.5 + 0.0j
    kd = 1e-3
    khat, e = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    ref = O.solve_target(occ, comp, [m], kd, khat, [0, 1, 0], e, "CM", npol=1, tol=1e-12)
    c = n // 2
    nf = O.nearfield(occ, comp, [m], kd, khat, e, "CM", ref["P"][0], [0] * 6,
                     points=[(c * n + c) * n + c, ((c - 2) * n + c) * n + c + 2])
    want = 3.0 / (m * m + 2.0)
    for j in range(2):
        Em = nf["E_macro"][j]
        assert abs(Em[1] / want - 1) < 0.02, Em
        assert abs(Em[0]) < 0.02 and abs(Em[2]) < 0.02


def test_far_outside_a_small_target_the_field_is_its_total_dipole():
    occ, comp = tg.sphere(4)
    kd = 1e-3
    e = np.array([0, 0, 1.0])
    ref = O.solve_target(occ, comp, [2.0 + 0.5j], kd, [1, 0, 0], [0, 1, 0], e, "LDR", npol=1,
                         operator="dense")
    P = ref["P"][0]
    ptot = P.sum(axis=0)
    nf = O.nearfield(occ, comp, [2.0 + 0.5j], kd, [1, 0, 0], e, "LDR", P, [0, 12, 0, 0, 0, 0])
    (nx, ny, nz), (lx, ly, lz) = nf["dims"], nf["lo"]
    r = np.array([nx - 1 - lx - 1.5, 0.5, 0.5])       # farthest +x site, from the centre
    E = nf["E_sca"][:, 2, 2, nx - 1]
    rr = np.linalg.norm(r)
    nrm = r / rr
    dip = (3 * nrm * np.dot(nrm, ptot) - ptot) / rr ** 3
    assert np.abs(E - dip).max() < 0.02 * np.abs(dip).max()


def test_single_dipole_magnetic_field_is_the_textbook_one():
    """B = k^2 (n x p) (e^{ikr}/r)(1 - 1/(ikr)) for a point dipole (Jackson's
    dipole fields in Gaussian units), and B -> n x E in the far zone."""
    occ = np.ones((1, 1, 1), np.uint8)
    kd = 0.9
    p = np.array([[0.3 + 0.1j, -0.2j, 0.5]])
    nf = O.nearfield(occ, occ.copy(), [1.5], kd, [0, 0, 1], [1, 0, 0], "CM", p, [2, 3, 1, 2, 2, 1])
    (nx, ny, nz), (lx, ly, lz) = nf["dims"], nf["lo"]
    pv = p[0]
    worst = 0.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                r = np.array([x - lx, y - ly, z - lz], float)
                rr = np.linalg.norm(r)
                if rr == 0:
                    assert np.all(nf["B_sca"][:, z, y, x] == 0)
                    continue
                n = r / rr
                ref = kd ** 2 * np.cross(n, pv) * np.exp(1j * kd * rr) / rr * (1 - 1 / (1j * kd * rr))
                worst = max(worst, np.abs(nf["B_sca"][:, z, y, x] - ref).max() / np.abs(ref).max())
    assert worst < 1e-12
    # plane wave: B_inc = khat x E_inc
    assert np.allclose(nf["B_inc"][1], nf["E_inc"][0], atol=1e-15)   # z x x = y
    # far zone: B = n x E up to O(1/(kr))
    rr = 400.0
    n = np.array([0.6, 0.0, 0.8])
    E = O.green_point(rr * n, kd) @ pv
    B = np.cross(O.magnetic_vector(rr * n, kd), pv)
    assert np.abs(B - np.cross(n, E)).max() < 3.0 / (kd * rr) * np.abs(B).max()


def test_filtered_magnetic_vector_tends_to_the_point_one_far_away():
    for r in (15.0, 30.0):
        dr = np.array([r * 0.6, r * 0.0, r * 0.8])
        hp = O.magnetic_vector(dr, 0.4, "LDR")
        hf = O.magnetic_vector(dr, 0.4, "FCD")
        assert np.abs(hf - hp).max() < 0.05 * np.abs(hp).max()
        # a genuine filter: the two differ near the source
    hp = O.magnetic_vector(np.array([1.0, 0, 0]), 0.4, "LDR")
    hf = O.magnetic_vector(np.array([1.0, 0, 0]), 0.4, "FCD")
    assert np.abs(hf - hp).max() > 0.05 * np.abs(hp).max()


@pytest.mark.slow
def test_guide_nearfield_track_through_the_au_sphere():
    """The guide's ddpostprocess example (Sec. "The Program ddpostprocess"):
    the 59728-dipole Au pseudosphere (m = 0.96 + 1.01i, x = 5, k d = 0.20619,
    GKDLDR), E_y along the x axis through its centre on the 96^3 near-field
    box.  The oracle's microscopic field, interpolated trilinearly between
    sites, follows the printed values to 4.5% of the track's largest |E| on the
    illuminated side and inside the sphere, and to 7% on the shadow side
    (points within one spacing of the surface, where interpolation straddles
    the discontinuity, are skipped).  The printed shadow-side values match the
    oracle's one printed row (1.455 d) further from the sphere; the cause is
    not known, hence the looser bound there."""
    import nearfield_track as T
    occ, comp = tg.sphere(48, T.DIAMETER)
    N = int(occ.sum())
    assert N == 59728
    kd = T.X_SIZE / O.effective_radius(N)
    assert abs(kd - 0.20619) < 5e-6            # the printed k_inc d
    r = O.solve_target(occ, comp, [T.M_AU], kd, [1, 0, 0], [0, 1, 0], [0, 1, 0], "GKDLDR",
                       npol=1, tol=1e-8)
    dims, lo = O.nearfield_box(occ.shape, T.EXT)
    assert dims == (96, 96, 96)
    d_um = T.LAMBDA_UM * kd / (2 * math.pi)
    x_um, e_pr = T.printed()
    pts = sorted({i for x in x_um for i, _ in T.corners(x / d_um, lo, 48, dims)})
    nf = O.nearfield(occ, comp, [T.M_AU], kd, [1, 0, 0], [0, 1, 0], "GKDLDR", r["P"][0],
                     T.EXT, points=np.array(pts))
    etot = (nf["E_inc"] + nf["E_sca"])[:, 1]
    at = dict(zip(pts, etot))
    inner, shadow = T.compare(x_um, e_pr, lambda xd: sum(w * at[i] for i, w in
                                                         T.corners(xd, lo, 48, dims)),
                              d_um, 0.5 * T.DIAMETER)
    assert inner < 0.045, inner
    assert shadow < 0.07, shadow
