"""The seeded synthetic workloads the library is tested and measured on.

Each workload is a target (occupancy + composition), refractive indices
relative to the ambient medium, k*d, the incident beams in the target frame and
the solver settings.  Sizes follow the DDSCAT 7.3 guide's workload shapes: a
sphere is an ELLIPSOID with equal axes, the size parameter is x = k a_eff with
a_eff = (3N/4pi)^(1/3) d (Sec. "Target Size and Validity Criteria"), so
kd = x / (a_eff/d).  No dataset is involved; the random pieces (the serving
stream, random test vectors) are drawn from numpy generators with fixed seeds.

This module holds no DDA arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import orientation as ori
from . import targets as tg


@dataclasses.dataclass
class Workload:
    name: str
    occ: np.ndarray            # (nz, ny, nx) uint8
    comp: np.ndarray           # (nz, ny, nx) uint8, 1..ncomp on occupied sites
    m: list                    # complex refractive index per composition
    kd: float
    khat: np.ndarray           # [n_inc, 3] incidence directions (TF)
    yhat: np.ndarray           # [n_inc, 3] y_LF in the TF
    e01: np.ndarray            # [n_inc, 3] complex first polarization (TF)
    npol: int = 2
    method: str = "LDR"        # CM | LDR | FCD
    tol: float = 1e-8
    x: float = 0.0             # size parameter k a_eff
    dirs: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros((0, 2)))  # [n_dirs, 2] (theta_s, phi_s) LF

    @property
    def shape(self):
        nz, ny, nx = self.occ.shape
        return nx, ny, nz

    @property
    def n_dipoles(self) -> int:
        return int(np.count_nonzero(self.occ))

    @property
    def n_rhs(self) -> int:
        return self.khat.shape[0] * self.npol


def kd_for_size_parameter(x: float, n_dipoles: int) -> float:
    return x / tg.effective_radius(n_dipoles)


def default_dirs():
    """A few scattering directions in the LF planes phi_s = 0 and 90 deg."""
    th = np.deg2rad(np.arange(0.0, 181.0, 30.0))
    d = [(t, 0.0) for t in th] + [(t, 0.5 * math.pi) for t in th]
    return np.array(d[1:])  # the forward direction is always added by the solver


def _lab_incidence(orientations):
    return ori.incident_set(orientations)


def sphere_workload(name, n, m, x, method="LDR", tol=1e-8, diameter=None):
    occ, comp = tg.sphere(n, diameter)
    N = int(np.count_nonzero(occ))
    kd = kd_for_size_parameter(x, N)
    kh, yh, e1 = _lab_incidence([(0.0, 0.0, 0.0)])
    return Workload(name, occ, comp, [complex(m)], kd, kh, yh, e1, 2, method,
                    tol, x, default_dirs())


def c1_sphere16():
    """Sphere on a 16^3 lattice, m = 1.33+0.01i, x = 1, LDR, FP64, tol 1e-8."""
    return sphere_workload("sphere16_m1.33_x1_LDR", 16, 1.33 + 0.01j, 1.0)


def c2_sphere64():
    """Sphere on a 64^3 lattice, m = 1.5+0.02i, x = 5, LDR, two polarizations."""
    return sphere_workload("sphere64_m1.5_x5_LDR", 64, 1.5 + 0.02j, 5.0)


def c5_sphere256():
    """Sphere on a 256^3 lattice, m = 1.33+0.01i, x = 25, LDR (grid 512^3)."""
    return sphere_workload("sphere256_m1.33_x25_LDR", 256, 1.33 + 0.01j, 25.0)


def c3_ellipsoid(nbeta=4, ntheta=8):
    """Ellipsoid 1:2:3 on 48x96x144, m = 1.7+0.1i, x = 8, FCD; NBETA x NTHETA
    orientations (beta midpoints over [0, 360), cos(Theta) midpoints over
    [0, 180] for even NTHETA, Phi = 0), two polarizations each."""
    occ, comp = tg.ellipsoid(48, 96, 144)
    N = int(np.count_nonzero(occ))
    kd = kd_for_size_parameter(8.0, N)
    orients = [(t, 0.0, b) for t in ori.sample_theta(0.0, math.pi, ntheta)
               for b in ori.sample_beta(0.0, 2.0 * math.pi, nbeta)]
    kh, yh, e1 = _lab_incidence(orients)
    return Workload("ellipsoid48x96x144_m1.7_x8_FCD", occ, comp, [1.7 + 0.1j], kd,
                    kh, yh, e1, 2, "FCD", 1e-8, 8.0, default_dirs())


def small_ellipsoid(nx=6, ny=10, nz=12, m=1.5 + 0.1j, kd=0.4, method="LDR",
                    n_orient=1, seed=7):
    """A small non-cubic ellipsoid with random orientations (parity cases)."""
    occ, comp = tg.ellipsoid(nx, ny, nz)
    rng = np.random.default_rng(seed)
    orients = [(0.0, 0.0, 0.0)] + ori.random_orientations(rng, n_orient - 1)
    kh, yh, e1 = _lab_incidence(orients)
    N = int(np.count_nonzero(occ))
    return Workload(f"ellipsoid{nx}x{ny}x{nz}", occ, comp, [complex(m)], kd, kh,
                    yh, e1, 2, method, 1e-10, kd * tg.effective_radius(N),
                    default_dirs())


def two_material_brick(nx=7, ny=5, nz=9, m=(1.5 + 0.1j, 2.0 + 0.5j), kd=0.5,
                       method="LDR", seed=3):
    """A brick with two compositions assigned at random (ragged, non-cubic)."""
    occ, comp = tg.rect_prism(nx, ny, nz)
    rng = np.random.default_rng(seed)
    comp = (1 + (rng.random(occ.shape) < 0.4)).astype(np.uint8)
    vac = rng.random(occ.shape) < 0.15
    occ = occ.copy()
    occ[vac] = 0
    comp[vac] = 0
    kh, yh, e1 = _lab_incidence([(0.3, 0.2, 0.1)])
    N = int(np.count_nonzero(occ))
    return Workload(f"brick{nx}x{ny}x{nz}_2mat", occ, comp, [complex(v) for v in m],
                    kd, kh, yh, e1, 2, method, 1e-10,
                    kd * tg.effective_radius(N), default_dirs())


def random_polarization(occ: np.ndarray, seed: int, n_rhs: int = 1):
    """Seeded complex normal vectors on occupied sites, zero on vacant ones.

    Shape [n_rhs, 3, nz, ny, nx] complex128 (the box layout).
    """
    rng = np.random.default_rng(seed)
    shp = (n_rhs, 3) + occ.shape
    v = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    v *= (occ != 0)[None, None]
    return v


def serving_stream(n_requests=400, seed=20261202, n_min=1e3, n_max=1e6,
                   rate_hz=1.0, burst=(0.5, 0.6, 4.0)):
    """The seeded serving stream: targets of mixed shape and size.

    Shape uniform over {sphere, CYLINDER1, HEX_PRISM, RCTGLPRSM}; N log-uniform
    in [n_min, n_max] (the generator scales the box to land within ~5%);
    Re m ~ U[1.2, 2.0], Im m ~ U[0, 0.3]; x log-uniform in [1, min(10, x_max)]
    with x_max = 62.04/|m| (N/1e6)^(1/3) so that |m| k d <= 1; LDR; random
    orientation.  Arrival times are Poisson at ``rate_hz``, with the rate
    multiplied by burst[2] between fractions burst[0] and burst[1] of the
    stream.  Returns a list of dicts.
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for i in range(n_requests):
        frac = i / max(1, n_requests)
        r = rate_hz * (burst[2] if burst[0] <= frac < burst[1] else 1.0)
        t += rng.exponential(1.0 / r)
        shape = ["sphere", "cylinder", "hex_prism", "rect"][int(rng.integers(4))]
        n_target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        ar = rng.uniform(0.5, 3.0)
        ratios = rng.uniform(1.0, 3.0, size=2)
        occ, comp = _shape_with_n(shape, n_target, ar, ratios)
        m = complex(rng.uniform(1.2, 2.0), rng.uniform(0.0, 0.3))
        N = int(np.count_nonzero(occ))
        x_max = 62.04 / abs(m) * (N / 1e6) ** (1.0 / 3.0)
        x_hi = max(1.0, min(10.0, x_max))
        x = math.exp(rng.uniform(0.0, math.log(x_hi)))
        kd = kd_for_size_parameter(x, N)
        orients = ori.random_orientations(rng, 1)
        kh, yh, e1 = _lab_incidence(orients)
        out.append(dict(id=i, t_arrival=t, shape=shape, occ=occ, comp=comp,
                        m=[m], kd=kd, x=x, khat=kh, yhat=yh, e01=e1,
                        method="LDR", npol=2))
    return out


def _shape_with_n(shape, n_target, ar, ratios):
    """Scale a shape so that its dipole count lands near n_target."""
    def build(s):
        if shape == "sphere":
            n = max(2, int(round(s)))
            return tg.sphere(n)
        if shape == "cylinder":
            return tg.cylinder(ar * s, s, 1)
        if shape == "hex_prism":
            return tg.hex_prism(ar * s, s, 1)
        nx = max(1, int(round(s)))
        return tg.rect_prism(nx, max(1, int(round(s * ratios[0]))),
                             max(1, int(round(s * ratios[1]))))

    # volume ~ c * s^3: two secant steps on log N vs log s
    s = n_target ** (1.0 / 3.0)
    for _ in range(6):
        occ, comp = build(s)
        n = max(1, int(np.count_nonzero(occ)))
        if abs(n / n_target - 1.0) < 0.05:
            break
        s *= (n_target / n) ** (1.0 / 3.0)
    return tg.trim(occ, comp)
