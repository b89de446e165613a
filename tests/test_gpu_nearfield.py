"""GPU near field (dda_nearfield) against the oracle's direct sums.

The oracle evaluates the same dipoles P (the GPU solve's) at every site of
the extended box, so the comparison isolates the near-field computation:
E_sca, E_macro and B_sca to 1e-10 of the largest value, E_inc and B_inc to
1e-13.  With a
converged P the identity P_j = alpha_j (E_inc + E_sca)_j holds at target sites
to the solve's tolerance.
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

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1305_6497_gb300 import binding
    return binding


def _max_rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("method", ["LDR", "CM", "FCD"])
def test_nearfield_matches_oracle_on_the_whole_extended_box(B, method):
    w = W.small_ellipsoid(5, 6, 4, m=1.6 + 0.2j, kd=0.5, method=method, n_orient=2, seed=4)
    ext = [0.4, 0.6, 0.3, 0.2, 0.5, 0.5]
    t = B.Target(w.occ, w.comp, w.m, method=method)
    sol = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-11, precision="fp64")
    nf = t.nearfield(w.kd, w.khat, w.e01, sol["P"], ext,
                     want=("E_inc", "E_sca", "E_macro", "B_inc", "B_sca"))
    assert nf["dims"] == O.nearfield_box(w.occ.shape, ext)[0]
    flat, _ = O.site_positions(w.occ)
    for i in range(2):
        e1, e2 = O.polarization_pair(w.khat[i], w.e01[i])
        for l, e in enumerate((e1, e2)):
            r = 2 * i + l
            ref = O.nearfield(w.occ, w.comp, w.m, w.kd, w.khat[i], e, method, sol["P"][r], ext)
            assert _max_rel(nf["E_sca"][r], ref["E_sca"]) < 1e-10
            assert np.abs(nf["E_inc"][r] - ref["E_inc"]).max() < 1e-13
            assert _max_rel(nf["E_macro"][r], ref["E_macro"]) < 1e-10
            assert _max_rel(nf["B_sca"][r], ref["B_sca"]) < 1e-10
            assert np.abs(nf["B_inc"][r] - ref["B_inc"]).max() < 1e-13
            # identity at target sites
            (nx, ny, nz), (lx, ly, lz) = nf["dims"], nf["lo"]
            tz, ty, tx = w.occ.shape
            ix, iy, iz = flat % tx, (flat // tx) % ty, flat // (tx * ty)
            etot = (nf["E_inc"][r] + nf["E_sca"][r])[:, iz + lz, iy + ly, ix + lx].T
            ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, method, w.kd,
                                        w.khat[i], e)
            P = sol["P"][r]
            assert np.abs(P - etot / ainv[:, None]).max() < 1e-8 * np.abs(P).max()
    t.close()


def test_nearfield_sphere32_sampled_points_and_cache(B):
    occ, comp = tg.sphere(32)
    m, kd = [1.33 + 0.01j], 0.2
    t = B.Target(occ, comp, m, method="LDR")
    khat, e01 = np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]])
    sol = t.solve(kd, khat, e01, yhat=[[0, 1.0, 0]], tol=1e-9, precision="fp32_refined")
    ext = [0.25] * 6
    nf = t.nearfield(kd, khat, e01, sol["P"], ext)
    dims, lo = nf["dims"], nf["lo"]
    assert dims == (48, 48, 48) and lo == (8, 8, 8)
    rng = np.random.default_rng(5)
    M = dims[0] * dims[1] * dims[2]
    pts = np.unique(np.concatenate([[0, M - 1], rng.choice(M, 40, replace=False)]))
    e1, e2 = O.polarization_pair(khat[0], e01[0])
    for l, e in enumerate((e1, e2)):
        ref = O.nearfield(occ, comp, m, kd, khat[0], e, "LDR", sol["P"][l], ext, points=pts)
        got = nf["E_sca"][l].reshape(3, -1)[:, pts].T
        assert _max_rel(got, ref["E_sca"]) < 1e-10
        got = nf["E_macro"][l].reshape(3, -1)[:, pts].T
        assert _max_rel(got, ref["E_macro"]) < 1e-10
    nb = t.nearfield(kd, khat, e01, sol["P"], ext, want=("B_sca",))
    for l, e in enumerate((e1, e2)):
        ref = O.nearfield(occ, comp, m, kd, khat[0], e, "LDR", sol["P"][l], ext, points=pts)
        got = nb["B_sca"][l].reshape(3, -1)[:, pts].T
        assert _max_rel(got, ref["B_sca"]) < 1e-10
    # the extended box is cached: a second call gives identical fields
    nf2 = t.nearfield(kd, khat, e01, sol["P"], ext, want=("E_sca",))
    assert np.array_equal(nf2["E_sca"], nf["E_sca"]) and nf2["E_inc"] is None
    # another extension rebuilds it
    nf3 = t.nearfield(kd, khat, e01, sol["P"], [0, 0, 0, 0, 0, 0.5], want=("E_sca",))
    assert nf3["dims"] == (32, 32, 48)
    a = nf3["E_sca"][:, :, :32, :, :]
    b = nf["E_sca"][:, :, 8:40, 8:40, 8:40]
    assert _max_rel(a, b) < 1e-12
    t.close()


def test_nearfield_rejects_bad_arguments(B):
    occ, comp = tg.sphere(6)
    t = B.Target(occ, comp, [1.5], method="LDR")
    sol = t.solve(0.3, [1, 0, 0], [0, 1, 0], tol=1e-8)
    with pytest.raises(B.DDAError):
        t.nearfield(0.3, [1, 0, 0], [0, 1, 0], sol["P"], [-0.1, 0, 0, 0, 0, 0])
    with pytest.raises(B.DDAError):
        t.nearfield(0.3, [1, 0, 0], [0, 1, 0], sol["P"], [0, 0, 0, 0, 0, 200])
    with pytest.raises(ValueError):
        t.nearfield(0.3, [1, 0, 0], [0, 1, 0], sol["P"][:1], [0] * 6)
    t.close()


def test_guide_nearfield_track_through_the_au_sphere(B):
    """The guide's ddpostprocess example on the GPU (59728-dipole Au
    pseudosphere, GKDLDR, 96^3 near-field box): the library's E on the sites
    around the x-axis track equals the oracle's direct sums for the same dipoles
    to 1e-9, and the interpolated E_y follows the printed track as in the
    oracle's test (4.5% of max |E| illuminated side and inside, 7% shadow side)."""
    import nearfield_track as T
    occ, comp = tg.sphere(48, T.DIAMETER)
    N = int(occ.sum())
    kd = T.X_SIZE / O.effective_radius(N)
    t = B.Target(occ, comp, [T.M_AU], method="GKDLDR")
    out = t.solve(kd, [1, 0, 0], [0, 1, 0], yhat=[0, 1, 0], npol=1, tol=1e-8,
                  precision="fp32_refined")
    nf = t.nearfield(kd, [1, 0, 0], [0, 1, 0], out["P"], T.EXT, npol=1,
                     want=("E_inc", "E_sca"))
    t.close()
    dims, lo = nf["dims"], nf["lo"]
    assert tuple(dims) == (96, 96, 96)
    etot = (nf["E_inc"] + nf["E_sca"])[0, 1].reshape(-1)
    d_um = T.LAMBDA_UM * kd / (2 * math.pi)
    x_um, e_pr = T.printed()
    pts = sorted({i for x in x_um for i, _ in T.corners(x / d_um, lo, 48, dims)})
    ref = O.nearfield(occ, comp, [T.M_AU], kd, [1, 0, 0], [0, 1, 0], "GKDLDR", out["P"][0],
                      T.EXT, points=np.array(pts))
    eref = (ref["E_inc"] + ref["E_sca"])[:, 1]
    assert np.abs(etot[pts] - eref).max() <= 1e-9 * np.abs(eref).max()
    inner, shadow = T.compare(x_um, e_pr, lambda xd: sum(w * etot[i] for i, w in
                                                         T.corners(xd, lo, 48, dims)),
                              d_um, 0.5 * T.DIAMETER)
    assert inner < 0.045, inner
    assert shadow < 0.07, shadow
