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
        assert set(sched[p]) == set(B.SCHEDULE_KEYS)
    y1 = t.matvec(0.4, x)
    assert np.abs(y1 - y0).max() <= 1e-12 * np.abs(y0).max()
    ainv = O.site_alpha_inverse(comp.reshape(-1)[flat], [1.5 + 0.1j], "CM", 0.4)
    ref = O.matvec_direct(x, pos, ainv, 0.4, "CM", rows=np.arange(0, len(flat), 97))
    assert np.abs(y1[::97] - ref).max() <= 1e-10 * np.abs(ref).max()
    t.close()


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(13, 18, 22), (13, 32, 32), (32, 18, 64), (64, 7, 9),
                                   (48, 96, 9), (9, 7, 144), (5, 6, 256)])
def test_every_thread_count_gives_the_same_product(threads, precision, shape):
    """Explicit schedules with every thread count the tuner may pick (and odd
    line/tile counts) must reproduce the default schedule's product; box sides
    32 and 64 give the lengths 64 and 128 of the compile-time FP32 kernels."""
    from paper_1305_6497_gb300 import binding as B
    occ, comp = tg.ellipsoid(*shape)
    flat, pos = O.site_positions(occ)
    x = O.box_to_sites(W.random_polarization(occ, 5)[0], flat)
    t = B.Target(occ, comp, [1.5 + 0.1j], method="LDR")
    kh, e = [1.0, 0, 0], [0, 1.0, 0]
    y0 = t.matvec(0.4, x, kh, e, precision)
    for xl, yt, zt, gs in ((3, 5, 2, 0), (16, 8, 8, 1), (64, 32, 16, 0), (5, 16, 4, 1),
                           (8, 16, 16, 1)):
        try:
            t.set_schedule(dict(x_lines=xl, y_tile=yt, z_tile=zt, z_pitch=3 * zt + 1,
                                z_stage_ghat=gs, x_threads=threads, y_threads=threads,
                                z_threads=threads), precision)
        except B.DDAError as ex:  # e.g. 64 FP64 lines of 128 points: too big a CTA
            assert "shared memory" in str(ex)
            continue
        assert t.schedule(precision)["z_threads"] == threads
        y1 = t.matvec(0.4, x, kh, e, precision)
        tol = 1e-12 if precision == "fp64" else 1e-6
        assert np.abs(y1 - y0).max() <= tol * np.abs(y0).max(), (xl, yt, zt, gs)
    with pytest.raises(B.DDAError):
        t.set_schedule(dict(x_lines=8, y_tile=8, z_tile=3, z_pitch=9, z_stage_ghat=0,
                            x_threads=64, y_threads=64, z_threads=64), precision)
    with pytest.raises(B.DDAError):
        t.set_schedule(dict(x_lines=8, y_tile=8, z_tile=8, z_pitch=24, z_stage_ghat=0,
                            x_threads=48, y_threads=64, z_threads=64), precision)
    t.close()


@pytest.mark.parametrize("shape", [(13, 18, 64), (9, 7, 256)])
def test_compiled_z_pass_takes_384_threads(shape):
    """The FP32 z pass of a compiled radix plan accepts CTAs of 384 threads
    (same product); other z tiles and the FP64 pass keep the 256 limit."""
    from paper_1305_6497_gb300 import binding as B
    occ, comp = tg.ellipsoid(*shape)
    flat, pos = O.site_positions(occ)
    x = O.box_to_sites(W.random_polarization(occ, 5)[0], flat)
    t = B.Target(occ, comp, [1.5 + 0.1j], method="LDR")
    kh, e = [1.0, 0, 0], [0, 1.0, 0]
    y0 = t.matvec(0.4, x, kh, e, "fp32")
    for zt, gs in ((4, 1), (8, 0)):
        t.set_schedule(dict(x_lines=16, y_tile=16, z_tile=zt, z_pitch=3 * zt + 1,
                            z_stage_ghat=gs, x_threads=128, y_threads=128, z_threads=384),
                       "fp32")
        assert t.schedule("fp32")["z_threads"] == 384
        y1 = t.matvec(0.4, x, kh, e, "fp32")
        assert np.abs(y1 - y0).max() <= 1e-6 * np.abs(y0).max()
    with pytest.raises(B.DDAError):   # a 3-stage plan has no compiled 2-column tile
        if shape[2] == 256:
            t.set_schedule(dict(x_lines=16, y_tile=16, z_tile=2, z_pitch=7, z_stage_ghat=0,
                                x_threads=128, y_threads=128, z_threads=384), "fp32")
        else:
            t.set_schedule(dict(x_lines=16, y_tile=16, z_tile=8, z_pitch=25, z_stage_ghat=0,
                                x_threads=128, y_threads=128, z_threads=384), "fp64")
    t.close()


@pytest.mark.parametrize("shape", [(11, 18, 32), (12, 18, 64), (20, 7, 256), (10, 9, 144),
                                   (6, 40, 256)])
def test_column_pair_z_kernel_matches(shape):
    """z staging 2 and 3 select the column-pair z kernel (two columns per
    thread, both rows of an octant row and every right-hand side per CTA, its
    own radix-8 plan of the z length; Ghat read through L2, or staged once in
    shared memory), 6 and 7 the same with each pass's column tile loaded and
    stored by TMA (bit-identical to 2 and 3): the FP32 product equals the
    compiled-plan kernel's to FP32 rounding (another factorization of the same
    transform) and the oracle's, over ragged column tiles and odd Ly; batched
    solves (several right-hand sides, some converging first) give the same
    Q's."""
    from paper_1305_6497_gb300 import binding as B
    occ, comp = tg.ellipsoid(*shape)
    flat, pos = O.site_positions(occ)
    x = O.box_to_sites(W.random_polarization(occ, 7)[0], flat)
    t = B.Target(occ, comp, [1.5 + 0.1j], method="GKDLDR")
    kh, e = np.array([0.36, 0.48, 0.8]), [0.8, -0.6, 0]
    assert t.grid[0] % 2 == 0
    ainv = O.site_alpha_inverse(comp.reshape(-1)[flat], [1.5 + 0.1j], "GKDLDR", 0.4, kh)
    rows = np.arange(0, len(flat), 7)
    ref = O.matvec_direct(x, pos, ainv, 0.4, "GKDLDR", rows=rows)
    for zt in (4, 8):
        base = dict(x_lines=16, y_tile=16, z_tile=zt, z_pitch=3 * zt, x_threads=128,
                    y_threads=128, z_threads=256)
        t.set_schedule(dict(base, z_stage_ghat=0), "fp32")
        y0 = t.matvec(0.4, x, kh, e, "fp32")
        prev = {}
        for zg in (2, 3, 6, 7):
            t.set_schedule(dict(base, z_stage_ghat=zg, z_threads=384), "fp32")
            assert t.schedule("fp32")["z_stage_ghat"] == zg
            y1 = t.matvec(0.4, x, kh, e, "fp32")
            assert np.abs(y1 - y0).max() <= 2e-6 * np.abs(y0).max(), (zt, zg)
            assert np.abs(y1[rows] - ref).max() <= 2e-5 * np.abs(ref).max(), (zt, zg)
            if zg >= 6:   # TMA tiles: the same arithmetic as plain loads and stores
                assert np.array_equal(y1, prev[zg - 4]), (zt, zg)
            prev[zg] = y1
        with pytest.raises(B.DDAError):      # the pair kernel runs 384 threads
            t.set_schedule(dict(base, z_stage_ghat=2, z_threads=256), "fp32")
    w = W.small_ellipsoid(*shape, m=1.5 + 0.1j, kd=0.4, method="LDR", n_orient=3, seed=9)
    t2 = B.Target(w.occ, w.comp, w.m, method="LDR")
    kw = dict(yhat=w.yhat, npol=2, tol=1e-9, precision="fp32_refined", want_P=True)
    sched = dict(x_lines=16, y_tile=16, z_tile=8, z_pitch=24, x_threads=128, y_threads=128,
                 z_threads=256)
    t2.set_schedule(dict(sched, z_stage_ghat=0), "fp32")
    a = t2.solve(w.kd, w.khat, w.e01, **kw)
    for zg in (2, 3, 6, 7):
        t2.set_schedule(dict(sched, z_stage_ghat=zg, z_threads=384), "fp32")
        b = t2.solve(w.kd, w.khat, w.e01, **kw)
        assert b["status"] == B.DDA_OK
        assert np.all(np.abs(b["Qext"] / a["Qext"] - 1) < 1e-7)
        assert np.abs(b["P"] - a["P"]).max() <= 1e-7 * np.abs(a["P"]).max()
    t.close()
    t2.close()


def test_column_pair_z_kernel_needs_a_compiled_plan_and_even_x_length():
    from paper_1305_6497_gb300 import binding as B
    occ, comp = tg.ellipsoid(13, 10, 11)      # Lx = 25 (odd), Lz = 24: no pair plan
    t = B.Target(occ, comp, [1.5 + 0.1j], method="CM")
    with pytest.raises(B.DDAError):
        t.set_schedule(dict(x_lines=16, y_tile=16, z_tile=4, z_pitch=12, z_stage_ghat=2,
                            x_threads=128, y_threads=128, z_threads=384), "fp32")
    t.close()
