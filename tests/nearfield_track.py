"""The guide's near-field track (Sec. "The Program ddpostprocess"): E along the
x_TF axis through the centre of the Au pseudosphere of its ELLIPSOID_NEARFIELD
example, and how a track point's field is read off the extended box.

ddpostprocess's interpolation is not described; the reading here is trilinear
interpolation of the microscopic field E_inc + E_sca on the sites of the
extended box (the track at y = z = 0 runs midway between four site columns,
at +-d/2).  Helpers only: the tests call the oracle or the library."""
import math
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "nearfield_track_au_sphere.txt")
M_AU = 0.96 + 1.01j
X_SIZE = 5.0            # 2 pi a_eff / lambda
LAMBDA_UM = 0.5
DIAMETER = 48.49        # the guide's 48^3 pseudosphere (N = 59728)
EXT = [0.5] * 6         # the near-field box extends 50% on every side (96^3)


def printed():
    """x_TF (um) and complex E_y of the printed track points."""
    a = np.loadtxt(GOLD)
    return a[:, 0], a[:, 1] + 1j * a[:, 2]


def corners(x_d, lo, n_tgt, dims):
    """Extended-box sites around the point (x_d, 0, 0) (lattice units from the
    target's centre) and their trilinear weights: [(flat index, weight)]."""
    nxe, nye, _ = dims
    f = x_d + lo[0] + 0.5 * (n_tgt - 1)
    i0 = int(math.floor(f))
    wx = f - i0
    cy = lo[1] + (n_tgt - 1) // 2        # the two site rows at y = -d/2, +d/2
    cz = lo[2] + (n_tgt - 1) // 2
    out = []
    for ix, w in ((i0, 1.0 - wx), (i0 + 1, wx)):
        for iy in (cy, cy + 1):
            for iz in (cz, cz + 1):
                out.append((ix + nxe * (iy + nye * iz), 0.25 * w))
    return out


def compare(x_um, e_printed, ey_at, d_um, radius_d):
    """Largest |E_y - printed| / max|printed| over the track points more than
    one lattice spacing from the sphere's surface, (a) on the illuminated half
    and inside the sphere, (b) on the shadow side outside it."""
    scale = np.abs(e_printed).max()
    inner, shadow = 0.0, 0.0
    for x, ep in zip(x_um, e_printed):
        xd = x / d_um
        if abs(abs(xd) - radius_d) < 1.0:
            continue
        err = abs(ey_at(xd) - ep) / scale
        if xd > radius_d:
            shadow = max(shadow, err)
        else:
            inner = max(inner, err)
    return inner, shadow
