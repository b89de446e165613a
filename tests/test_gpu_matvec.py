"""GPU parity of the A.P product (the hot loop) against the CPU oracle.

FP64: max |y_gpu - y_oracle| / max |y_oracle| <= 1e-10 (the tolerance the
method is held to for A.P).  FP32: <= 2e-5 (single-precision FFT of lengths up
to a few hundred: ~log2(L) * 2^-24 per pass, times five passes, with margin).
Cases span several tiles, ragged edges, vacancies, two materials, degenerate
one-site and one-line boxes, 2/3/5-smooth grids and all four polarizability
prescriptions (GKDLDR's tensor: a different alpha^{-1} on each lattice axis).
"""
import numpy as np
import pytest

from dda_inputs import targets as tg
from dda_inputs import workloads as W
from oracle import dda as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


@pytest.fixture(scope="module")
def B():
    from paper_1305_6497_gb300 import binding
    return binding


def _case(occ, comp, m, kd, method, khat, e, seed=5):
    flat, pos = O.site_positions(occ)
    comp_s = comp.reshape(-1)[flat]
    ainv = O.site_alpha_inverse(comp_s, m, method, kd, khat, e)
    x = O.box_to_sites(W.random_polarization(occ, seed)[0], flat)
    return flat, pos, ainv, x


def _ref(occ, pos, ainv, x, kd, method, flat):
    if len(pos) <= 3000:
        return O.matvec_direct(x, pos, ainv, kd, method)
    ainv_box = np.zeros((3, occ.size), np.complex128)
    ainv_box[:, flat] = (np.repeat(ainv[:, None], 3, axis=1) if ainv.ndim == 1 else ainv).T
    op = O.FFTOperator(occ, ainv_box.reshape((3,) + occ.shape), kd, method)
    return O.box_to_sites(op(O.sites_to_box(x, flat, occ.shape)), flat)


def _err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


CASES = [
    ("ellipsoid6x10x12", lambda: tg.ellipsoid(6, 10, 12), [1.5 + 0.1j]),
    ("brick7x5x9_2mat", lambda: (W.two_material_brick().occ, W.two_material_brick().comp),
     [1.5 + 0.1j, 2.0 + 0.5j]),
    ("one_site", lambda: tg.rect_prism(1, 1, 1), [1.7 + 0.2j]),
    ("line_z5", lambda: tg.rect_prism(1, 1, 5), [1.7 + 0.2j]),
    ("line_x3", lambda: tg.rect_prism(3, 1, 1), [1.7 + 0.2j]),
    ("slab_24x20x9", lambda: tg.ellipsoid(24, 20, 9, 30, 30, 12), [1.33 + 0.05j]),
    ("sphere16", lambda: tg.sphere(16), [1.33 + 0.01j]),
    ("cyl_13x13x31", lambda: tg.cylinder(31, 13, 3), [1.6 + 0.3j]),
    # z lengths 64 and 128 (compile-time z kernel), ragged x tiles, nz < Lz/2
    ("ell_20x24x32", lambda: tg.ellipsoid(20, 24, 32), [1.5 + 0.1j]),
    ("ell_13x9x64", lambda: tg.ellipsoid(13, 9, 64), [1.33 + 0.05j]),
    ("ell_11x10x63", lambda: tg.ellipsoid(11, 10, 63), [1.7 + 0.2j]),
    # x lengths 64 and 128 (compile-time x kernels), ragged row tiles, nx < Lx/2
    ("ell_32x7x5", lambda: tg.ellipsoid(32, 7, 5), [1.5 + 0.1j]),
    ("ell_64x6x5", lambda: tg.ellipsoid(64, 6, 5), [1.33 + 0.05j]),
    ("ell_63x5x6", lambda: tg.ellipsoid(63, 5, 6), [1.7 + 0.2j]),
    # three- and four-stage compiled plans: 512 = 16x8x4 on each axis, and the
    # ellipsoid grid's 96 = 8x4x3 (x), 192 = 16x4x3 (y), 288 = 8x4x3x3 (z)
    ("ell_256x5x4", lambda: tg.ellipsoid(256, 5, 4), [1.33 + 0.01j]),
    ("ell_4x256x5", lambda: tg.ellipsoid(4, 256, 5), [1.33 + 0.01j]),
    ("ell_5x4x256", lambda: tg.ellipsoid(5, 4, 256), [1.33 + 0.01j]),
    ("ell_48x7x5", lambda: tg.ellipsoid(48, 7, 5), [1.7 + 0.1j]),
    ("ell_5x96x6", lambda: tg.ellipsoid(5, 96, 6), [1.7 + 0.1j]),
    ("ell_6x5x144", lambda: tg.ellipsoid(6, 5, 144), [1.7 + 0.1j]),
]


@pytest.mark.parametrize("name,mk,m", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("method", ["LDR", "CM", "FCD", "GKDLDR"])
def test_matvec_fp64_matches_oracle(B, name, mk, m, method):
    occ, comp = mk()
    kd = 0.37
    khat = np.array([0.36, 0.48, 0.8])
    e = np.array([0.8, -0.6, 0.0], np.complex128)
    flat, pos, ainv, x = _case(occ, comp, m, kd, method, khat, e)
    ref = _ref(occ, pos, ainv, x, kd, method, flat)
    t = B.Target(occ, comp, m, method=method)
    y = t.matvec(kd, x, khat, e, "fp64")
    assert _err(y, ref) <= TOL64, (name, method, _err(y, ref))
    # the refinement's residual operator: FP64 vectors, double-float FFT passes
    ydf = t.matvec(kd, x, khat, e, "df64")
    assert _err(ydf, ref) <= TOL64, (name, method, _err(ydf, ref))
    y32 = t.matvec(kd, x, khat, e, "fp32")
    assert _err(y32, ref) <= TOL32, (name, method, _err(y32, ref))
    t.close()


def test_matvec_grid_is_smooth_and_large_enough(B):
    occ, comp = tg.ellipsoid(7, 11, 13)
    t = B.Target(occ, comp, [1.5])
    L = t.grid
    for n, l in zip((7, 11, 13), L):
        assert l >= 2 * n - 1
        r = l
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        assert r == 1
    t.close()


def test_matvec_kd_change_rebuilds_green(B):
    occ, comp = tg.ellipsoid(6, 7, 8)
    flat, pos, ainv1, x = _case(occ, comp, [1.4 + 0.1j], 0.2, "CM", None, None)
    _, _, ainv2, _ = _case(occ, comp, [1.4 + 0.1j], 0.9, "CM", None, None)
    t = B.Target(occ, comp, [1.4 + 0.1j], method="CM")
    for kd, ai in ((0.2, ainv1), (0.9, ainv2), (0.2, ainv1)):
        y = t.matvec(kd, x)
        ref = O.matvec_direct(x, pos, ai, kd, "CM")
        assert _err(y, ref) <= TOL64
    t.close()


def test_matvec_is_deterministic(B):
    occ, comp = tg.sphere(12)
    flat, pos, ainv, x = _case(occ, comp, [1.5 + 0.02j], 0.3, "LDR", [1, 0, 0], [0, 1, 0])
    t = B.Target(occ, comp, [1.5 + 0.02j])
    a = t.matvec(0.3, x, [1, 0, 0], [0, 1, 0])
    b = t.matvec(0.3, x, [1, 0, 0], [0, 1, 0])
    assert np.array_equal(a, b)
    t.close()
