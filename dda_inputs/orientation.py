"""Target orientation and incident-beam vectors (input preparation only).

The DDSCAT 7.3 guide fixes a Lab Frame (LF) in which the incident wave travels
along +x_LF, and places the target by three angles: Theta (between target axis
a1 and x_LF), Phi (rotation of a1 about x_LF) and beta (rotation of the target
about a1) -- Sec. "Target Orientation", subsection "Orientation of the Target in
the Lab Frame".  The solver works in the Target Frame (TF), so a caller needs
x_LF, y_LF, z_LF written in TF coordinates; those are the inverse relations of
the same subsection.  For the shapes used here the target axes a1, a2, a3 are
the TF axes x, y, z.

Angles are sampled as in subsection "Sampling in Theta, Phi, and beta":
midpoints of NBETA (resp. NPHI) equal intervals for beta (resp. Phi), and
uniform in cos(Theta) -- midpoints of NTHETA intervals when NTHETA is even, the
end points included (Simpson nodes) when it is odd.
"""
from __future__ import annotations

import math

import numpy as np


def lab_axes_in_target_frame(theta: float, phi: float, beta: float):
    """Return (x_LF, y_LF, z_LF) as TF vectors for orientation (Theta, Phi, beta).

    Radians.  With a1, a2, a3 the TF basis, the guide writes x_LF, y_LF, z_LF as
    combinations of a1, a2, a3; the coefficients are returned as rows.
    """
    ct, st = math.cos(theta), math.sin(theta)
    cp, sp = math.cos(phi), math.sin(phi)
    cb, sb = math.cos(beta), math.sin(beta)
    x_lf = np.array([ct, -st * cb, st * sb])
    y_lf = np.array([st * cp, ct * cb * cp - sb * sp, -(ct * sb * cp + cb * sp)])
    z_lf = np.array([st * sp, ct * cb * sp + sb * cp, -(ct * sb * sp - cb * cp)])
    return x_lf, y_lf, z_lf


def target_axes_in_lab_frame(theta: float, phi: float, beta: float):
    """Return (a1, a2, a3) in LF coordinates (the forward relations)."""
    ct, st = math.cos(theta), math.sin(theta)
    cp, sp = math.cos(phi), math.sin(phi)
    cb, sb = math.cos(beta), math.sin(beta)
    a1 = np.array([ct, st * cp, st * sp])
    a2 = np.array([-st * cb, ct * cb * cp - sb * sp, ct * cb * sp + sb * cp])
    a3 = np.array([st * sb, -(ct * sb * cp + cb * sp), -(ct * sb * sp - cb * cp)])
    return a1, a2, a3


def sample_beta(bmin: float, bmax: float, n: int):
    """Midpoints of n equal intervals of [bmin, bmax] (also used for Phi)."""
    w = (bmax - bmin) / n
    return [bmin + (i + 0.5) * w for i in range(n)]


def sample_theta(tmin: float, tmax: float, n: int):
    """Theta values uniform in cos(Theta): midpoints if n even, ends if n odd."""
    c0, c1 = math.cos(tmin), math.cos(tmax)
    if n == 1:
        return [tmin]
    if n % 2 == 1:
        cs = [c0 + (c1 - c0) * i / (n - 1) for i in range(n)]
    else:
        cs = [c0 + (c1 - c0) * (i + 0.5) / n for i in range(n)]
    return [math.acos(max(-1.0, min(1.0, c))) for c in cs]


def incident_set(orientations):
    """Stack (khat, yhat, e01) TF arrays for a list of (Theta, Phi, beta).

    khat = x_LF, yhat = y_LF and e01 = y_LF (linear polarization along y_LF,
    the guide's common choice); e02 = khat x conj(e01) = z_LF is formed by the
    solver.  Returns khat [n,3], yhat [n,3], e01 [n,3] complex.
    """
    kh, yh, e1 = [], [], []
    for (t, p, b) in orientations:
        x_lf, y_lf, _ = lab_axes_in_target_frame(t, p, b)
        kh.append(x_lf)
        yh.append(y_lf)
        e1.append(y_lf.astype(np.complex128))
    return np.array(kh), np.array(yh), np.array(e1)


def random_orientations(rng: np.random.Generator, n: int):
    """n orientations with a1 uniform on the sphere and beta uniform."""
    out = []
    for _ in range(n):
        ct = rng.uniform(-1.0, 1.0)
        out.append((math.acos(ct), rng.uniform(0.0, 2.0 * math.pi),
                    rng.uniform(0.0, 2.0 * math.pi)))
    return out
