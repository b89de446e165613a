"""Orientation averages (dda_orient_average) against the oracle, which solves
each (beta, Theta, Phi) orientation on its own and applies the same
post-processing; and the guide's worked example on the GPU."""
import math

import numpy as np
import pytest

from dda_inputs import targets as tg
from oracle import dda as O
from oracle import scattering as S

pytestmark = pytest.mark.gpu
DEG = math.pi / 180


@pytest.fixture(scope="module")
def B():
    from paper_1305_6497_gb300 import binding
    return binding


def _compare(got, ref, tol):
    for k in ("Qext", "Qabs", "Qsca", "Qpha", "Qsca_int", "cos2", "Qbk"):
        assert np.allclose(got[k], ref[k], rtol=tol, atol=tol * 1e-3), (k, got[k], ref[k])
    assert np.allclose(got["g"], ref["g"], rtol=tol, atol=tol * np.abs(ref["g"]).max())
    mu, mr = got["mueller"], ref["mueller"]
    for s in range(len(mr)):
        assert np.abs(mu[s] - mr[s]).max() <= tol * np.abs(mr[s]).max()


@pytest.mark.parametrize("method,solver,e01", [("LDR", "bicgstab", (0, 1, 0)),
                                                ("FCD", "qmr", (0, 1, 1j)),
                                                ("CM", "bicgstab", (0, 0.6, -0.8))])
def test_orientation_average_matches_oracle(B, method, solver, e01):
    occ, comp = tg.ellipsoid(5, 6, 4)
    m, kd = [1.6 + 0.1j], 0.5
    grid = dict(beta=(0, math.pi), nbeta=2, theta=(0, math.pi), ntheta=3,
                phi=(0, 2 * math.pi), nphi=2)
    sel = [(0.0, 0.0), (35 * DEG, 10 * DEG), (90 * DEG, 90 * DEG), (160 * DEG, 300 * DEG)]
    t = B.Target(occ, comp, m, method=method)
    got = t.orient_average(kd, **grid, e01_lab=e01, tol=1e-11, precision="fp64", solver=solver,
                           eta=1.0, sel=sel)
    assert got["n_orient"] == 12 and got["status"] == B.DDA_OK
    e1 = np.asarray(e01, complex)
    ref = S.orientation_average(occ, comp, m, kd, ((0, math.pi), 2, (0, math.pi), 3,
                                                   (0, 2 * math.pi), 2),
                                method=method, e01_lab=e1, eta=1.0, sel=sel, tol=1e-12)
    assert got["n_sca"] == ref["n_sca"]
    _compare(got, ref, 1e-7)
    # the same averages when the orientations are solved in batches of 2 incidences
    got2 = t.orient_average(kd, **grid, e01_lab=e01, tol=1e-11, precision="fp64",
                            solver=solver, eta=1.0, sel=sel, max_rhs=4)
    _compare(got2, got, 1e-9)
    t.close()


def test_worked_example_on_the_gpu(B):
    """RCTGLPRSM 16 x 32 x 32 (the guide's Appendix): against the oracle at
    1e-6, and against the guide's printed values at the percent level."""
    occ, comp = tg.rect_prism(16, 32, 32)
    kd = 3.093665 * 0.06346821
    m = [0.9656 + 1.8628j]
    sel = [(20 * DEG, 0.0), (90 * DEG, 0.0), (180 * DEG, 0.0)]
    t = B.Target(occ, comp, m, method="LDR")
    got = t.orient_average(kd, tol=1e-10, precision="fp32_refined", eta=0.5, sel=sel)
    assert got["n_sca"] == 962
    ref = S.orientation_average(occ, comp, m, kd, ((0, 0), 1, (0, 0), 1, (0, 0), 1),
                                eta=0.5, sel=sel, tol=1e-10)
    _compare(got, ref, 1e-6)
    assert abs(np.mean(got["Qext"]) / 3.6134 - 1) < 0.01
    assert abs(np.mean(got["g"][:, 0]) / 0.41463 - 1) < 0.02
    assert abs(np.mean(got["cos2"]) / 0.75169 - 1) < 0.02
    assert abs(got["mueller"][2][0, 0] / 18.591 - 1) < 0.02
    t.close()
