"""Scattering amplitude matrix, Mueller matrix, averages over scattering
directions and over target orientations -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy restatements of the DDSCAT 7.3 guide's definitions, used by
the tests to check the library's host-side post-processing and its
orientation-averaged solve.  Only the tests may import this module.

  scattering_directions -- the (theta_s, phi_s) set and solid-angle weights
                           Omega_jk of Sec. "Averaging over Scattering
                           Directions" ("Angular Averaging", "Selection of
                           Scattering Angles", eq. average)
  amplitude_matrix      -- S_1..S_4 from f_ml (eq. fml_rel_S_v4 and the four
                           equations that follow it)
  mueller_matrix        -- S_ij from S_1..S_4 (Sec. "Relation Between Stokes
                           Parameters of Incident and Scattered Radiation")
  angular_averages      -- C_sca by integration, <cos>, <cos^2>, g, Q_bk
  orientation_grid      -- beta, Theta, Phi samples and weights WGTB, WGTA
                           (Sec. "Sampling in Theta, Phi, and beta",
                           "Orientational Averaging")
  orientation_average   -- the whole average, one oracle solve per orientation

Readings (where the guide is silent or its text does not fix a detail):
  * N_theta is the nearest integer to the printed expression (this reproduces
    the guide's NAVG = 962 for x = 3.093665, eta = 0.5); phi_{j,1} = 0.
  * For odd NTHETA the Simpson weights (1, 4, 2, ..., 4, 1)/3 are normalised to
    unit sum, i.e. divided by (NTHETA - 1) NPHI: the printed divisor
    NTHETA x NPHI would not average a constant to itself.
  * Q_pha = (2 pi / k^2) Re f_ll(0) / (pi a_eff^2) (phase-shift cross section
    of Draine 1988, from the forward amplitude, as C_ext is (4 pi/k^2) Im f_ll(0)).
  * Q_bk = (dC_sca/dOmega at theta = pi) / (pi a_eff^2), area per steradian;
    for the guide's example this is S_11(180)/(pi x^2), as its table shows.
  * Orientation averages of g and <cos^2> are C_sca-weighted:
    g = <Q_sca g>_orient / <Q_sca>_orient.
  * The reported Q_sca is Q_ext - Q_abs; the direction quadrature's own
    integral (Qsca_int) converges to it as O(dtheta^2) (1.5% at eta = 0.5 for
    the guide's example, whose printed Q_sca equals Q_ext - Q_abs to 5e-5), so
    the quadrature serves the normalised averages g and <cos^2>.
"""
from __future__ import annotations

import math

import numpy as np

from . import dda as O


def _nint(v: float) -> int:
    return int(math.floor(v + 0.5))


def scattering_directions(x: float, eta: float):
    """Returns (theta [n], phi [n], omega [n]) in radians, j-major order."""
    th0 = 2.0 * math.pi / (1.0 + x)
    nt = _nint(1.0 + 2.0 * (3.0 + x) / eta * (1.0 + 1.0 / (math.pi + th0))
               / (1.0 + th0 / (math.pi + th0) ** 2))
    nt = max(nt, 3)
    ds = (math.pi + math.pi / (math.pi + th0)) / (nt - 1)
    th = []
    for j in range(nt):
        s = j * ds
        # s = theta + theta/(theta + theta0), solved for theta >= 0
        th.append(0.5 * ((s - 1.0 - th0) + math.sqrt((1.0 + th0 - s) ** 2 + 4.0 * th0 * s)))
    th[0], th[-1] = 0.0, math.pi
    T, F, W = [], [], []
    for j in range(nt):
        if j == 0 or j == nt - 1:
            nphi = 1
        else:
            nphi = max(3, _nint(4.0 * math.pi * math.sin(th[j]) / (th[j + 1] - th[j - 1])))
        if j == 0:
            om = 2.0 * math.pi / nphi * (1.0 - 0.5 * (math.cos(th[0]) + math.cos(th[1])))
        elif j == nt - 1:
            om = 2.0 * math.pi / nphi * (0.5 * (math.cos(th[-2]) + math.cos(th[-1])) + 1.0)
        else:
            om = math.pi / nphi * (math.cos(th[j - 1]) - math.cos(th[j + 1]))
        for k in range(nphi):
            T.append(th[j])
            F.append(2.0 * math.pi * k / nphi)
            W.append(om)
    return np.array(T), np.array(F), np.array(W)


def amplitude_matrix(f, e01_lab, e02_lab, phi_s):
    """S_1..S_4 (Bohren & Huffman) from f_ml at a direction of azimuth phi_s.

    f [2 (m), 2 (l)]; e01_lab, e02_lab: incident polarization vectors in the
    Lab Frame; a, b, c, d = e01^* . y, e01^* . z, e02^* . y, e02^* . z."""
    a, b = np.conj(e01_lab[1]), np.conj(e01_lab[2])
    c, d = np.conj(e02_lab[1]), np.conj(e02_lab[2])
    cp, sp = math.cos(phi_s), math.sin(phi_s)
    f11, f12, f21, f22 = f[0, 0], f[0, 1], f[1, 0], f[1, 1]
    S1 = -1j * (f21 * (b * cp - a * sp) + f22 * (d * cp - c * sp))
    S2 = -1j * (f11 * (a * cp + b * sp) + f12 * (c * cp + d * sp))
    S3 = 1j * (f11 * (b * cp - a * sp) + f12 * (d * cp - c * sp))
    S4 = 1j * (f21 * (a * cp + b * sp) + f22 * (c * cp + d * sp))
    return np.array([S1, S2, S3, S4])


def mueller_matrix(S):
    """4x4 S_ij from (S_1, S_2, S_3, S_4)."""
    S1, S2, S3, S4 = S
    a1, a2, a3, a4 = (abs(v) ** 2 for v in S)
    M = np.empty((4, 4))
    M[0, 0] = (a1 + a2 + a3 + a4) / 2
    M[0, 1] = (a2 - a1 + a4 - a3) / 2
    M[0, 2] = (S2 * np.conj(S3) + S1 * np.conj(S4)).real
    M[0, 3] = (S2 * np.conj(S3) - S1 * np.conj(S4)).imag
    M[1, 0] = (a2 - a1 + a3 - a4) / 2
    M[1, 1] = (a1 + a2 - a3 - a4) / 2
    M[1, 2] = (S2 * np.conj(S3) - S1 * np.conj(S4)).real
    M[1, 3] = (S2 * np.conj(S3) + S1 * np.conj(S4)).imag
    M[2, 0] = (S2 * np.conj(S4) + S1 * np.conj(S3)).real
    M[2, 1] = (S2 * np.conj(S4) - S1 * np.conj(S3)).real
    M[2, 2] = (S1 * np.conj(S2) + S3 * np.conj(S4)).real
    M[2, 3] = (S2 * np.conj(S1) + S4 * np.conj(S3)).imag
    M[3, 0] = (S4 * np.conj(S2) + S1 * np.conj(S3)).imag
    M[3, 1] = (S4 * np.conj(S2) - S1 * np.conj(S3)).imag
    M[3, 2] = (S1 * np.conj(S2) - S3 * np.conj(S4)).imag
    M[3, 3] = (S1 * np.conj(S2) - S3 * np.conj(S4)).real
    return M


def angular_averages(f_l, theta, phi, omega, kd, aeff):
    """For one incident polarization l: f_l [n, 2 (m)] at the directions.

    dC_sca/dOmega = (|f_1l|^2 + |f_2l|^2) / k^2 (eq. f_ml_def with |E_0| = 1)."""
    k = float(kd)
    dc = (np.abs(f_l[:, 0]) ** 2 + np.abs(f_l[:, 1]) ** 2) / k ** 2
    csca = float(np.sum(omega * dc))
    nvec = np.stack([np.cos(theta), np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi)], 1)
    g = (omega * dc) @ nvec / csca
    cos2 = float(np.sum(omega * dc * np.cos(theta) ** 2) / csca)
    back = np.argmin(np.abs(theta - math.pi))
    geo = math.pi * aeff ** 2
    return dict(Qsca=csca / geo, g=g, cos2=cos2, Qbk=float(dc[back] / geo))


def orientation_grid(beta, nbeta, theta, ntheta, phi, nphi):
    """beta, theta, phi: (min, max) radians.  Returns the sample values and
    the weights WGTB [nbeta], WGTA [ntheta, nphi] (each set sums to 1)."""
    def mids(lo, hi, n):
        return [lo + (hi - lo) * (i + 0.5) / n for i in range(n)]
    b = mids(beta[0], beta[1], nbeta)
    p = mids(phi[0], phi[1], nphi)
    c0, c1 = math.cos(theta[0]), math.cos(theta[1])
    if ntheta == 1:
        t, wt = [theta[0]], [1.0]
    elif ntheta % 2 == 1:
        cs = [c0 + (c1 - c0) * i / (ntheta - 1) for i in range(ntheta)]
        t = [math.acos(max(-1.0, min(1.0, v))) for v in cs]
        wt = [(1.0 if i in (0, ntheta - 1) else (4.0 if i % 2 else 2.0)) / 3.0 / (ntheta - 1)
              for i in range(ntheta)]
    else:
        cs = [c0 + (c1 - c0) * (i + 0.5) / ntheta for i in range(ntheta)]
        t = [math.acos(max(-1.0, min(1.0, v))) for v in cs]
        wt = [1.0 / ntheta] * ntheta
    wb = np.full(nbeta, 1.0 / nbeta)
    wa = np.array(wt)[:, None] * np.full((1, nphi), 1.0 / nphi)
    return np.array(b), np.array(t), np.array(p), wb, wa


def lab_axes(theta: float, phi: float, beta: float):
    """x_LF, y_LF, z_LF in Target-Frame coordinates for the orientation
    (Theta, Phi, beta) of target axes a1 = x_TF, a2 = y_TF (Sec. "Orientation
    of the Target in the Lab Frame"): a1 makes the angle Theta with x_LF, Phi
    turns a1 about x_LF (from the x_LF-y_LF plane toward z_LF), beta turns the
    target about a1.  Inverting the guide's a1, a2, a3 in Lab-Frame coordinates
    gives the rows returned here."""
    ct, st = math.cos(theta), math.sin(theta)
    cp, sp = math.cos(phi), math.sin(phi)
    cb, sb = math.cos(beta), math.sin(beta)
    x = np.array([ct, -st * cb, st * sb])
    y = np.array([st * cp, ct * cb * cp - sb * sp, -ct * sb * cp - cb * sp])
    z = np.array([st * sp, ct * cb * sp + sb * cp, -ct * sb * sp + cb * cp])
    return x, y, z


def orientation_average(occ, comp, m_list, kd, grid, method="LDR", e01_lab=(0, 1, 0),
                        eta=0.0, sel=(), tol=1e-11):
    """Average over target orientations, one oracle solve per (beta, Theta, Phi).

    grid = (beta (min, max), nbeta, theta (min, max), ntheta, phi (min, max), nphi).
    The Lab Frame incident wave travels along x_LF with polarization e01_lab
    (e02 = x_LF x e01^*); the target's orientation gives x_LF, y_LF, z_LF in the
    Target Frame (Sec. "Orientation of the Target in the Lab Frame").
    Returns per-polarization averages and the averaged Mueller matrix at `sel`.
    """
    b, t, p, wb, wa = orientation_grid(*grid)
    N = int(np.count_nonzero(occ))
    aeff = O.effective_radius(N)
    geo = math.pi * aeff ** 2
    k = float(kd)
    e1l = np.asarray(e01_lab, np.complex128)
    e1l = e1l / np.linalg.norm(e1l)
    e2l = np.cross(np.array([1.0, 0, 0]), np.conj(e1l))
    if eta > 0:
        th_s, ph_s, om = scattering_directions(aeff * k, eta)
    else:
        th_s = ph_s = om = np.zeros(0)
    sel = np.asarray(sel, np.float64).reshape(-1, 2)
    dirs = np.concatenate([np.stack([th_s, ph_s], 1), sel]) if len(sel) or len(th_s) \
        else np.zeros((0, 2))
    acc = {key: np.zeros(2) for key in ("Qext", "Qabs", "Qsca", "Qpha", "Qsca_int", "cos2",
                                        "Qbk")}
    acc["g"] = np.zeros((2, 3))
    mu = np.zeros((len(sel), 4, 4))
    for ib, beta in enumerate(b):
        for it, theta in enumerate(t):
            for ip, phi in enumerate(p):
                w = wb[ib] * wa[it, ip]
                x_lf, y_lf, z_lf = lab_axes(theta, phi, beta)
                e01 = e1l[1] * y_lf + e1l[2] * z_lf
                ref = O.solve_target(occ, comp, m_list, kd, x_lf, y_lf, e01, method,
                                     npol=2, tol=tol, dirs=dirs)
                f = ref["famp"]            # [1 + D, 2 (m), 2 (l)], forward first
                for l in range(2):
                    acc["Qext"][l] += w * ref["Qext"][l]
                    acc["Qabs"][l] += w * ref["Qabs"][l]
                    acc["Qsca"][l] += w * ref["Qsca"][l]
                    acc["Qpha"][l] += w * (2.0 * math.pi / k ** 2) * f[0, l, l].real / geo
                    if eta > 0:
                        av = angular_averages(f[1:1 + len(th_s), :, l], th_s, ph_s, om, kd, aeff)
                        acc["Qsca_int"][l] += w * av["Qsca"]
                        acc["g"][l] += w * av["Qsca"] * av["g"]
                        acc["cos2"][l] += w * av["Qsca"] * av["cos2"]
                        acc["Qbk"][l] += w * av["Qbk"]
                for s in range(len(sel)):
                    S = amplitude_matrix(f[1 + len(th_s) + s], e1l, e2l, sel[s, 1])
                    mu[s] += w * mueller_matrix(S)
    if eta > 0:
        for l in range(2):
            acc["g"][l] /= acc["Qsca_int"][l]
            acc["cos2"][l] /= acc["Qsca_int"][l]
    acc["mueller"] = mu
    acc["n_sca"] = len(th_s)
    return acc
