"""Autotuned launch schedules give the same A.P (the schedule only changes how
the passes are tiled, never the arithmetic order within a transform line)."""
import numpy as np
import pytest

from dda_inputs import targets as tg
from dda_inputs import workloads as W
from oracle import dda as O

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results(tmp_path, monkeypatch):
    from paper_1305_6497_gb300 import binding as B
    monkeypatch.setenv("DDA_TUNE_FILE", str(tmp_path / "tune.txt"))
    occ, comp = tg.ellipsoid(20, 24, 28)
    flat, pos = O.site_positions(occ)
    x = O.box_to_sites(W.random_polarization(occ, 4)[0], flat)
    t = B.Target(occ, comp, [1.5 + 0.1j], method="CM")
    y0 = t.matvec(0.4, x)
    sched = t.autotune(0.4, 2)
    for p in ("fp32", "fp64"):
        assert set(sched[p]) == {"x_lines", "y_tile", "z_tile", "z_pitch", "z_stage_ghat"}
    y1 = t.matvec(0.4, x)
    assert np.abs(y1 - y0).max() <= 1e-12 * np.abs(y0).max()
    ainv = O.site_alpha_inverse(comp.reshape(-1)[flat], [1.5 + 0.1j], "CM", 0.4)
    ref = O.matvec_direct(x, pos, ainv, 0.4, "CM", rows=np.arange(0, len(flat), 97))
    assert np.abs(y1[::97] - ref).max() <= 1e-10 * np.abs(ref).max()
    t.close()
