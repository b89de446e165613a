"""Seeded, synthetic target geometries on a cubic lattice (input generators only).

A target is an occupancy grid ``occ`` of shape (nz, ny, nx), dtype uint8, with
flat index ``ix + nx*(iy + ny*iz)``, plus a composition grid ``comp`` of the
same shape (1..ncomp on occupied sites, 0 on vacant ones).  Lattice sites sit
at integer positions; the generators below test the site centres measured from
the centroid of the bounding box, so a site (ix, iy, iz) is at
``(ix - (nx-1)/2, iy - (ny-1)/2, iz - (nz-1)/2)`` in units of d.

The shapes follow the target descriptions of the DDSCAT 7.3 guide:
ELLIPSOID (Sec. "ELLIPSOID = Homogeneous, isotropic ellipsoid"), CYLINDER1,
HEX_PRISM and RCTGLPRSM.  The guide fixes the continuous shapes; the choice of
which lattice sites fall inside is this module's: a site belongs to the target
when its centre satisfies the shape's inequality (boundary included).

This module holds no DDA arithmetic: it only decides which sites exist.
"""
from __future__ import annotations

import math

import numpy as np


def _centred_axes(nx: int, ny: int, nz: int):
    x = np.arange(nx, dtype=np.float64) - 0.5 * (nx - 1)
    y = np.arange(ny, dtype=np.float64) - 0.5 * (ny - 1)
    z = np.arange(nz, dtype=np.float64) - 0.5 * (nz - 1)
    return np.meshgrid(z, y, x, indexing="ij")  # arrays of shape (nz, ny, nx)


def _as_target(mask: np.ndarray):
    occ = mask.astype(np.uint8)
    comp = occ.copy()  # one composition
    return occ, comp


def ellipsoid(nx: int, ny: int, nz: int, sx: float | None = None,
              sy: float | None = None, sz: float | None = None):
    """ELLIPSOID: sites with (x/sx)^2 + (y/sy)^2 + (z/sz)^2 <= 1/4.

    sx, sy, sz are the full lengths (diameters) along x, y, z in units of d;
    they default to the box extents nx, ny, nz.  The guide's pseudospheres
    (N = 304, 17904, 59728 in its examples) come out of diameter = n + 0.49 on
    an n^3 box; diameter = n gives N = 2176, 137376, 8783848 for n = 16, 64, 256.
    """
    sx = float(nx if sx is None else sx)
    sy = float(ny if sy is None else sy)
    sz = float(nz if sz is None else sz)
    Z, Y, X = _centred_axes(nx, ny, nz)
    q = (X / sx) ** 2 + (Y / sy) ** 2 + (Z / sz) ** 2
    return _as_target(q <= 0.25)


def sphere(n: int, diameter: float | None = None):
    """A pseudosphere of the given diameter (default n) on an n^3 box."""
    d = float(n if diameter is None else diameter)
    return ellipsoid(n, n, n, d, d, d)


def rect_prism(nx: int, ny: int, nz: int):
    """RCTGLPRSM: every site of an nx x ny x nz brick."""
    return _as_target(np.ones((nz, ny, nx), dtype=bool))


def cylinder(length: float, diameter: float, axis: int = 1):
    """CYLINDER1: a cylinder of the given length and diameter (units of d).

    axis = 1, 2, 3 puts the cylinder axis along x, y, z of the target frame.
    The box is the smallest one that holds the shape; a site belongs to the
    cylinder when |axial| <= length/2 and radial distance <= diameter/2.
    """
    nl = max(1, int(math.ceil(length - 1e-9)))
    nd = max(1, int(math.ceil(diameter - 1e-9)))
    dims = [nd, nd, nd]
    dims[axis - 1] = nl
    nx, ny, nz = dims
    Z, Y, X = _centred_axes(nx, ny, nz)
    coords = [X, Y, Z]
    a = coords[axis - 1]
    others = [c for i, c in enumerate(coords) if i != axis - 1]
    rad2 = others[0] ** 2 + others[1] ** 2
    mask = (np.abs(a) <= 0.5 * length) & (rad2 <= 0.25 * diameter * diameter)
    return _as_target(mask)


def hex_prism(length: float, vertex_to_vertex: float, axis: int = 1):
    """HEX_PRISM: hexagonal prism, axis along x/y/z (axis = 1/2/3).

    The hexagon has side s = vertex_to_vertex/2 and one pair of vertices on the
    first remaining axis; a site is inside when it lies within all three pairs
    of parallel edges (distance <= s*sqrt(3)/2 from the centre along each edge
    normal) and |axial| <= length/2.
    """
    s = 0.5 * vertex_to_vertex
    apothem = s * math.sqrt(3.0) / 2.0
    nl = max(1, int(math.ceil(length - 1e-9)))
    nu = max(1, int(math.ceil(2.0 * s - 1e-9)))
    nv = max(1, int(math.ceil(2.0 * apothem - 1e-9)))
    dims = [0, 0, 0]
    rest = [i for i in range(3) if i != axis - 1]
    dims[axis - 1] = nl
    dims[rest[0]] = nu
    dims[rest[1]] = nv
    nx, ny, nz = dims
    Z, Y, X = _centred_axes(nx, ny, nz)
    coords = [X, Y, Z]
    a = coords[axis - 1]
    u = coords[rest[0]]
    v = coords[rest[1]]
    inside = np.abs(a) <= 0.5 * length
    for ang in (0.0, math.pi / 3.0, 2.0 * math.pi / 3.0):
        # edge normals of a hexagon with vertices on the u axis point at
        # 30, 90, 150 degrees from u
        nu_, nv_ = math.cos(ang + math.pi / 6.0), math.sin(ang + math.pi / 6.0)
        inside &= np.abs(u * nu_ + v * nv_) <= apothem + 1e-12
    return _as_target(inside)


def trim(occ: np.ndarray, comp: np.ndarray):
    """Crop occ/comp to the bounding box of the occupied sites."""
    idx = np.nonzero(occ)
    if len(idx[0]) == 0:
        return occ, comp
    sl = tuple(slice(int(i.min()), int(i.max()) + 1) for i in idx)
    return np.ascontiguousarray(occ[sl]), np.ascontiguousarray(comp[sl])


def num_dipoles(occ: np.ndarray) -> int:
    return int(np.count_nonzero(occ))


def effective_radius(n_dipoles: int) -> float:
    """a_eff / d = (3 N / 4 pi)^(1/3): the radius of the equal-volume sphere."""
    return (3.0 * n_dipoles / (4.0 * math.pi)) ** (1.0 / 3.0)
