"""GPU parity of the whole solve (BiCGSTAB, refinement, observables) against
the CPU oracle.

The oracle solves to a relative residual of 1e-12; the GPU to the tolerance
given.  Q_ext and Q_abs must agree to 1e-6 relative (the method's FP64 bar),
P to 1e-6 in norm, f_ml to 1e-6 relative to max |f|.  The GPU's reported
residual is recomputed by the oracle from the returned P.
"""
import math

import numpy as np
import pytest

from dda_inputs import targets as tg
from dda_inputs import workloads as W
from oracle import dda as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1305_6497_gb300 import binding
    return binding


def _oracle(w, i=0, tol=1e-12):
    return O.solve_target(w.occ, w.comp, w.m, w.kd, w.khat[i], w.yhat[i], w.e01[i],
                          w.method, npol=w.npol, tol=tol, dirs=w.dirs)


def _check(out, ref, r0=0, tolq=1e-6, tolp=1e-6):
    for l in range(len(ref["Qext"])):
        r = r0 + l
        assert abs(out["Qext"][r] / ref["Qext"][l] - 1) < tolq, (r, out["Qext"][r], ref["Qext"][l])
        assert abs(out["Qabs"][r] / ref["Qabs"][l] - 1) < tolq
        assert abs(out["Qsca"][r] - (out["Qext"][r] - out["Qabs"][r])) < 1e-14
        perr = np.linalg.norm(out["P"][r] - ref["P"][l]) / np.linalg.norm(ref["P"][l])
        assert perr < tolp, (r, perr)


@pytest.mark.parametrize("method", ["LDR", "CM", "FCD", "GKDLDR"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_solve_small_ellipsoid(B, method, precision):
    w = W.small_ellipsoid(6, 10, 12, m=1.5 + 0.1j, kd=0.4, method=method)
    ref = _oracle(w)
    t = B.Target(w.occ, w.comp, w.m, method=method)
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=2, tol=1e-10, precision=precision,
                  dirs=w.dirs)
    assert out["status"] == B.DDA_OK
    _check(out, ref)
    assert np.all(out["resid"] <= 1e-10 * 1.01)
    fa, fr = out["famp"][0], ref["famp"]
    assert np.abs(fa - fr).max() < 1e-6 * np.abs(fr).max()
    t.close()


def test_solve_two_materials_with_vacancies(B):
    w = W.two_material_brick()
    ref = _oracle(w)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, dirs=w.dirs)
    _check(out, ref)
    t.close()


def test_solve_many_orientations_batched(B):
    """Several incidences x 2 polarizations solved as one batch of RHS; each
    one must equal the oracle's solve of that incidence alone."""
    w = W.small_ellipsoid(8, 6, 7, m=1.7 + 0.1j, kd=0.5, method="FCD", n_orient=4, seed=9)
    t = B.Target(w.occ, w.comp, w.m, method="FCD")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, precision="fp32_refined",
                  dirs=w.dirs)
    for i in range(4):
        ref = _oracle(w, i)
        _check(out, ref, r0=2 * i)
        assert np.abs(out["famp"][i] - ref["famp"]).max() < 1e-6 * np.abs(ref["famp"]).max()
    t.close()


def test_c1_sphere16_vs_oracle_and_mie(B):
    """Sphere 16^3, m = 1.33+0.01i, x = 1, LDR, FP64, tol 1e-8."""
    from oracle import mie
    w = W.c1_sphere16()
    ref = _oracle(w, tol=1e-12)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-8, precision="fp64", dirs=w.dirs)
    assert out["status"] == B.DDA_OK
    _check(out, ref, tolq=1e-6, tolp=1e-5)
    qe_mie = mie.mie_q(w.m[0], w.x)[0]
    assert abs(np.mean(out["Qext"]) / qe_mie - 1) < 0.02
    t.close()


def test_optical_theorem_on_gpu_outputs(B):
    w = W.small_ellipsoid(9, 7, 5, m=1.4 + 0.05j, kd=0.6, method="LDR", n_orient=3, seed=2)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-9, dirs=w.dirs)
    g = math.pi * O.effective_radius(w.n_dipoles) ** 2
    for i in range(3):
        for l in range(2):
            cext = 4 * math.pi / w.kd ** 2 * out["famp"][i, 0, l, l].imag
            assert abs(cext / g / out["Qext"][2 * i + l] - 1) < 1e-10
    t.close()


def test_reported_residual_matches_oracle_residual(B):
    w = W.small_ellipsoid(7, 8, 9, m=1.6 + 0.2j, kd=0.45, method="LDR")
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-6, precision="fp32_refined")
    flat, pos = O.site_positions(w.occ)
    e1, e2 = O.polarization_pair(w.khat[0], w.e01[0])
    for l, e in enumerate((e1, e2)):
        ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, "LDR", w.kd, w.khat[0], e)
        E = O.incident_field(pos, w.kd, w.khat[0], e)
        r = E - O.matvec_direct(out["P"][l], pos, ainv, w.kd, "LDR")
        res = np.linalg.norm(r) / np.linalg.norm(E)
        assert abs(res / out["resid"][l] - 1) < 1e-3
        assert res <= 1e-6
    t.close()


def test_warm_start_from_solution_needs_no_iterations(B):
    w = W.small_ellipsoid(6, 6, 6, m=1.5 + 0.1j, kd=0.4, method="CM")
    t = B.Target(w.occ, w.comp, w.m, method="CM")
    a = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-9)
    b = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-8, P0=a["P"])
    assert np.all(b["iters"] == 0)
    assert np.allclose(a["Qext"], b["Qext"], rtol=1e-12)
    t.close()


def test_noconv_reports_last_iterate(B):
    w = W.small_ellipsoid(8, 8, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    out = t.solve(w.kd, w.khat, w.e01, tol=1e-14, max_iter=2, precision="fp64")
    assert out["status"] == B.DDA_ERR_NOCONV
    assert np.all(out["iters"] == 2)
    assert np.all(np.isfinite(out["Qext"]))
    t.close()


def test_invalid_arguments_are_rejected(B):
    occ, comp = tg.sphere(4)
    with pytest.raises(B.DDAError):
        B.Target(np.zeros((3, 3, 3), np.uint8), None, [1.5])
    with pytest.raises(B.DDAError):
        B.Target(occ, comp * 3, [1.5])
    t = B.Target(occ, comp, [1.5 + 0.1j])
    with pytest.raises(B.DDAError):
        t.solve(-1.0, [1, 0, 0], [0, 1, 0])
    with pytest.raises(B.DDAError):
        t.solve(0.3, [1, 0, 0], [1, 0, 0])   # e01 not transverse
    t.set_polarizability("FCD")
    with pytest.raises(B.DDAError):
        t.solve(3.5, [1, 0, 0], [0, 1, 0])   # FCD needs kd < pi
    t.close()


# ---- QMR for complex-symmetric A (the guide's QMRCCG option) ------------------------
@pytest.mark.parametrize("method", ["LDR", "FCD"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_qmr_small_ellipsoid(B, method, precision):
    w = W.small_ellipsoid(6, 10, 12, m=1.5 + 0.1j, kd=0.4, method=method)
    ref = _oracle(w)
    t = B.Target(w.occ, w.comp, w.m, method=method)
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=2, tol=1e-10, precision=precision,
                  dirs=w.dirs, solver="qmr")
    assert out["status"] == B.DDA_OK
    _check(out, ref)
    assert np.all(out["resid"] <= 1e-10 * 1.01)
    assert np.abs(out["famp"][0] - ref["famp"]).max() < 1e-6 * np.abs(ref["famp"]).max()
    if precision == "fp64":
        # one matvec per iteration (plus the final true-residual matvec)
        assert out["matvecs"] == int(np.sum(out["iters"])) + 2
    t.close()


def test_qmr_batched_orientations_and_two_materials(B):
    w = W.small_ellipsoid(8, 6, 7, m=1.7 + 0.1j, kd=0.5, method="FCD", n_orient=4, seed=9)
    t = B.Target(w.occ, w.comp, w.m, method="FCD")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, precision="fp32_refined",
                  dirs=w.dirs, solver="qmr")
    for i in range(4):
        _check(out, _oracle(w, i), r0=2 * i)
    t.close()
    w = W.two_material_brick()
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, dirs=w.dirs, solver="qmr")
    _check(out, _oracle(w))
    t.close()


def test_qmr_and_bicgstab_agree_and_qmr_needs_fewer_matvecs(B):
    w = W.c1_sphere16()
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    a = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-8, precision="fp64")
    q = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-8, precision="fp64", solver="qmr")
    assert np.allclose(a["Qext"], q["Qext"], rtol=1e-6, atol=0)
    assert np.all(q["resid"] <= 1e-8)
    assert q["matvecs"] < a["matvecs"]
    # switching back and forth reuses nothing stale (graphs are per solver)
    a2 = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-8, precision="fp64")
    assert np.array_equal(a["Qext"], a2["Qext"])
    t.close()


def test_qmr_warm_start_and_noconv(B):
    w = W.small_ellipsoid(6, 6, 6, m=1.5 + 0.1j, kd=0.4, method="CM")
    t = B.Target(w.occ, w.comp, w.m, method="CM")
    a = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-9, solver="qmr")
    b = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-8, P0=a["P"], solver="qmr")
    assert np.all(b["iters"] == 0)
    out = t.solve(w.kd, w.khat, w.e01, tol=1e-14, max_iter=3, precision="fp64", solver="qmr")
    assert out["status"] == B.DDA_ERR_NOCONV
    assert np.all(out["iters"] == 3)
    assert np.all(np.isfinite(out["Qext"]))
    with pytest.raises(KeyError):
        t.solve(w.kd, w.khat, w.e01, solver="gmres")
    t.close()


def test_unknown_solver_code_is_rejected_by_the_library(B):
    import ctypes as ct
    w = W.small_ellipsoid(4, 4, 4, m=1.5 + 0.1j, kd=0.4, method="LDR")
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    prm, keep, _ = B._params(w.kd, w.khat, w.e01, None, 2, 1e-8, 10, "fp64", 0.0, None, None)
    prm.solver = 7
    res = B.SolveResult()
    assert B.lib.dda_solve(t.h, ct.byref(prm), ct.byref(res)) == B.DDA_ERR_INVALID_ARG
    assert "solver" in B.dda_last_error()
    t.close()


def test_qmr_circular_polarization_falls_back_and_converges(B):
    """Circularly polarized light has E_j . E_j = 0 at every site, so QMR's
    bilinear Lanczos process breaks down at once; the library finishes those
    right-hand sides with BiCGSTAB and the result equals BiCGSTAB's and the
    oracle's."""
    w = W.small_ellipsoid(5, 6, 4, m=1.6 + 0.1j, kd=0.5, method="FCD")
    x, y = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    e = np.array([0, 1, 1j]) / np.sqrt(2)
    t = B.Target(w.occ, w.comp, w.m, method="FCD")
    for precision in ("fp64", "fp32_refined"):
        q = t.solve(w.kd, x, e, yhat=y, tol=1e-10, precision=precision, solver="qmr")
        b = t.solve(w.kd, x, e, yhat=y, tol=1e-10, precision=precision)
        assert q["status"] == B.DDA_OK
        assert np.all(q["resid"] <= 1e-10)
        assert np.allclose(q["Qext"], b["Qext"], rtol=1e-8)
    ref = O.solve_target(w.occ, w.comp, w.m, w.kd, x, y, e, "FCD", npol=2, tol=1e-12)
    assert np.allclose(q["Qext"], ref["Qext"], rtol=1e-6)
    t.close()


def test_refined_residual_in_double_float_equals_fp64_residual(B):
    """The refinement's residuals computed with double-float FFT passes give the
    same converged solution as with FP64 passes (to the solve tolerance)."""
    w = W.small_ellipsoid(9, 10, 12, m=1.5 + 0.1j, kd=0.4, method="LDR", n_orient=2, seed=3)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    a = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, precision="fp32_refined")
    b = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, precision="fp32_refined",
                fp64_residual=True)
    assert np.all(a["resid"] <= 1e-10) and np.all(b["resid"] <= 1e-10)
    assert np.allclose(a["Qext"], b["Qext"], rtol=1e-8, atol=0)
    assert np.abs(a["P"] - b["P"]).max() <= 1e-8 * np.abs(b["P"]).max()
    # the reported residual is the true residual (checked in FP64 by the oracle)
    flat, pos = O.site_positions(w.occ)
    e1, _ = O.polarization_pair(w.khat[0], w.e01[0])
    ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, "LDR", w.kd, w.khat[0], e1)
    E = O.incident_field(pos, w.kd, w.khat[0], e1)
    r = E - O.matvec_direct(a["P"][0], pos, ainv, w.kd, "LDR")
    assert abs(np.linalg.norm(r) / np.linalg.norm(E) / a["resid"][0] - 1) < 1e-2
    t.close()


# ---- BiCGstab(2) (the guide's PBCGS2) ------------------------------------------------
@pytest.mark.parametrize("method", ["LDR", "FCD"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_bicgstab2_small_ellipsoid(B, method, precision):
    w = W.small_ellipsoid(6, 10, 12, m=1.5 + 0.1j, kd=0.4, method=method)
    ref = _oracle(w)
    t = B.Target(w.occ, w.comp, w.m, method=method)
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=2, tol=1e-10, precision=precision,
                  dirs=w.dirs, solver="bicgstab2")
    assert out["status"] == B.DDA_OK
    _check(out, ref)
    assert np.all(out["resid"] <= 1e-10 * 1.01)
    assert np.all(out["iters"] % 2 == 0)       # whole cycles of two iterations
    t.close()


def test_bicgstab2_batched_and_circular(B):
    w = W.small_ellipsoid(8, 6, 7, m=1.7 + 0.1j, kd=0.5, method="FCD", n_orient=4, seed=9)
    t = B.Target(w.occ, w.comp, w.m, method="FCD")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, precision="fp32_refined",
                  dirs=w.dirs, solver="bicgstab2")
    for i in range(4):
        _check(out, _oracle(w, i), r0=2 * i)
    x, y = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    e = np.array([0, 1, 1j]) / np.sqrt(2)
    q = t.solve(w.kd, x, e, yhat=y, tol=1e-10, precision="fp64", solver="bicgstab2")
    b = t.solve(w.kd, x, e, yhat=y, tol=1e-10, precision="fp64")
    assert q["status"] == B.DDA_OK
    assert np.allclose(q["Qext"], b["Qext"], rtol=1e-8)
    t.close()


# ---- GPBi-CG (the guide's GPBICG) and normal-equation CG (PETRKP) ------------------
@pytest.mark.parametrize("solver", ["gpbicg", "petrkp"])
@pytest.mark.parametrize("method", ["LDR", "FCD"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_gpbicg_petrkp_small_ellipsoid(B, solver, method, precision):
    w = W.small_ellipsoid(6, 10, 12, m=1.5 + 0.1j, kd=0.4, method=method)
    ref = _oracle(w)
    t = B.Target(w.occ, w.comp, w.m, method=method)
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=2, tol=1e-10, precision=precision,
                  dirs=w.dirs, solver=solver, max_iter=5000)
    assert out["status"] == B.DDA_OK
    _check(out, ref)
    assert np.all(out["resid"] <= 1e-10 * 1.01)
    fa, fr = out["famp"][0], ref["famp"]
    assert np.abs(fa - fr).max() < 1e-6 * np.abs(fr).max()
    t.close()


def _linear_system(w):
    """E and v -> A v (the oracle's direct sum) for the first incidence and
    polarization, as flat site-major vectors."""
    flat, pos = O.site_positions(w.occ)
    e1, _ = O.polarization_pair(w.khat[0], w.e01[0])
    ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, w.method, w.kd, w.khat[0], e1)
    E = O.incident_field(pos, w.kd, w.khat[0], e1)
    mv = lambda v: O.matvec_direct(v.reshape(-1, 3), pos, ainv, w.kd, w.method).reshape(-1)
    return E, mv


def test_gpbicg_first_iteration_is_bicgstab(B):
    """GPBi-CG's first iteration has eta = 0 by definition, so its iterate is
    BiCGSTAB's first iterate (the oracle's, from the same zero start and shadow
    vector); after three iterations eta != 0 and the two differ."""
    w = W.small_ellipsoid(6, 7, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    E, mv = _linear_system(w)
    x1, _, _ = O.bicgstab(mv, E.reshape(-1), tol=0.0, maxiter=1)
    x3, _, _ = O.bicgstab(mv, E.reshape(-1), tol=0.0, maxiter=3)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    g1 = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=1,
                 precision="fp64", solver="gpbicg")
    assert g1["status"] == B.DDA_ERR_NOCONV and g1["iters"][0] == 1
    assert np.abs(g1["P"][0].reshape(-1) - x1).max() <= 1e-10 * np.abs(x1).max()
    g3 = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=3,
                 precision="fp64", solver="gpbicg")
    assert np.abs(g3["P"][0].reshape(-1) - x3).max() > 1e-8 * np.abs(x3).max()
    t.close()


def test_petrkp_first_iterate_and_monotone_residual(B):
    """Normal-equation CG: the first iterate is alpha A^H E with
    alpha = ||A^H E||^2 / ||A A^H E||^2 (A^H v = conj(A conj v)), and the true
    residual never grows from one iteration to the next (CG on A^H A minimises
    ||E - A P|| over a growing Krylov space)."""
    w = W.small_ellipsoid(6, 7, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    E, mv = _linear_system(w)
    b = E.reshape(-1)
    z = np.conj(mv(np.conj(b)))
    az = mv(z)
    x1 = (np.vdot(z, z).real / np.vdot(az, az).real) * z
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    res = []
    for k in (1, 2, 3, 5, 8, 13):
        o = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=k,
                    precision="fp64", solver="petrkp")
        assert o["iters"][0] == k
        if k == 1:
            assert np.abs(o["P"][0].reshape(-1) - x1).max() <= 1e-10 * np.abs(x1).max()
        res.append(o["resid"][0])
    assert all(b2 <= b1 * (1 + 1e-12) for b1, b2 in zip(res, res[1:])), res
    t.close()


def test_gpbicg_batched_circular_and_fallback(B):
    """Four orientations x two polarizations in one batch; circular
    polarization (E . E = 0 breaks QMR, not GPBi-CG) agrees with BiCGSTAB."""
    w = W.small_ellipsoid(8, 6, 7, m=1.7 + 0.1j, kd=0.5, method="FCD", n_orient=4, seed=9)
    t = B.Target(w.occ, w.comp, w.m, method="FCD")
    out = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, tol=1e-10, precision="fp32_refined",
                  dirs=w.dirs, solver="gpbicg")
    for i in range(4):
        _check(out, _oracle(w, i), r0=2 * i)
    x, y = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    e = np.array([0, 1, 1j]) / np.sqrt(2)
    for solver in ("gpbicg", "petrkp"):
        q = t.solve(w.kd, x, e, yhat=y, tol=1e-10, precision="fp64", solver=solver,
                    max_iter=5000)
        b = t.solve(w.kd, x, e, yhat=y, tol=1e-10, precision="fp64")
        assert q["status"] == B.DDA_OK
        assert np.allclose(q["Qext"], b["Qext"], rtol=1e-8)
    t.close()


@pytest.mark.parametrize("k", [2, 5])
def test_gpbicg_iterates_match_oracle(B, k):
    """The GPU's k-th GPBi-CG iterate (FP64) equals the oracle's (oracle/krylov.py),
    the same recurrences from the same start, up to FFT rounding."""
    from oracle import krylov as K
    w = W.small_ellipsoid(6, 7, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    E, mv = _linear_system(w)
    xo, n = K.gpbicg(mv, E.reshape(-1), maxiter=k)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    g = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=k,
                precision="fp64", solver="gpbicg")
    assert n == k and g["iters"][0] == k
    assert np.abs(g["P"][0].reshape(-1) - xo).max() <= 1e-9 * np.abs(xo).max()
    t.close()


@pytest.mark.parametrize("k", [3, 8])
def test_petrkp_iterates_match_oracle(B, k):
    """The GPU's k-th normal-equation CG iterate (FP64) equals the oracle's."""
    from oracle import krylov as K
    w = W.small_ellipsoid(6, 7, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    E, mv = _linear_system(w)
    xo, n = K.cgnr(mv, E.reshape(-1), maxiter=k)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    g = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=k,
                precision="fp64", solver="petrkp")
    assert n == k and g["iters"][0] == k
    assert np.abs(g["P"][0].reshape(-1) - xo).max() <= 1e-9 * np.abs(xo).max()
    t.close()


@pytest.mark.parametrize("k", [3, 7])
def test_qmr_iterates_match_oracle(B, k):
    """The GPU's k-th QMR iterate (FP64; its pending d/x update flushed) equals
    the oracle's complex-symmetric QMR."""
    from oracle import krylov as K
    w = W.small_ellipsoid(6, 7, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    E, mv = _linear_system(w)
    xo, n, _ = K.qmr_sym(mv, E.reshape(-1), maxiter=k)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    g = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=k,
                precision="fp64", solver="qmr")
    assert n == k and g["iters"][0] == k
    assert np.abs(g["P"][0].reshape(-1) - xo).max() <= 1e-9 * np.abs(xo).max()
    t.close()


@pytest.mark.parametrize("cycles", [1, 3])
def test_bicgstab2_iterates_match_oracle(B, cycles):
    """The GPU's BiCGstab(2) iterate after k cycles (2k iterations, FP64) equals
    the oracle's."""
    from oracle import krylov as K
    w = W.small_ellipsoid(6, 7, 8, m=1.5 + 0.1j, kd=0.4, method="LDR")
    E, mv = _linear_system(w)
    xo, c, _ = K.bicgstab2(mv, E.reshape(-1), ncycles=cycles)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    g = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=2 * cycles,
                precision="fp64", solver="bicgstab2")
    assert c == cycles and g["iters"][0] == 2 * cycles
    assert np.abs(g["P"][0].reshape(-1) - xo).max() <= 1e-9 * np.abs(xo).max()
    t.close()


def test_solve_on_a_callers_stream_is_bit_identical(B):
    """dda_solve_params.cuda_stream: the solve runs on a caller's (torch) stream,
    after the caller's earlier work there, with the same results bit for bit."""
    import torch
    w = W.small_ellipsoid(8, 12, 32, m=1.5 + 0.1j, kd=0.4, method="LDR", n_orient=2)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    kw = dict(yhat=w.yhat, npol=2, tol=1e-10, precision="fp32_refined", dirs=w.dirs)
    ref = t.solve(w.kd, w.khat, w.e01, **kw)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # queue work ahead on the caller's stream; the solve must order after it
        a = torch.randn(4096, 4096, device="cuda")
        b = a @ a
    out = t.solve(w.kd, w.khat, w.e01, stream_ptr=s.cuda_stream, **kw)
    assert s.query()                       # the call returned after its work finished
    torch.cuda.synchronize()
    del a, b
    for key in ("Qext", "Qabs", "iters", "resid"):
        assert np.array_equal(out[key], ref[key]), key
    assert np.array_equal(out["P"], ref["P"])
    assert np.array_equal(out["famp"], ref["famp"])
    t.close()


@pytest.mark.parametrize("precision", ["fp32_refined", "fp64"])
def test_guide_worked_example_gkdldr(B, precision):
    """The guide's appendix example (RCTGLPRSM 16x32x32 Au brick, GKDLDR, k d =
    0.19635, m = 0.9656 + 1.8628i): Q_ext 3.6134, Q_abs 1.4308, Q_sca 2.1827,
    S_11(0) 75.115, S_11(180) 18.591 as printed, to 1e-4 relative, and the
    oracle's values to 1e-6."""
    occ, comp = tg.rect_prism(16, 32, 32)
    kd = 3.093665 * 0.06346821
    m = 0.9656 + 1.8628j
    t = B.Target(occ, comp, [m], method="GKDLDR")
    out = t.solve(kd, [1, 0, 0], [0, 1, 0], yhat=[0, 1, 0], npol=2, tol=1e-8,
                  precision=precision, dirs=np.array([(math.pi, 0.0)]), want_P=False)
    t.close()
    assert out["status"] == B.DDA_OK
    f = out["famp"][0]
    s11 = 0.5 * np.sum(np.abs(f) ** 2, axis=(1, 2))
    qext, qabs = np.mean(out["Qext"]), np.mean(out["Qabs"])
    got = dict(qext=qext, qabs=qabs, qsca=qext - qabs, s0=s11[0], s180=s11[1])
    printed = dict(qext=3.6134, qabs=1.4308, qsca=2.1827, s0=75.115, s180=18.591)
    for key, v in printed.items():
        assert abs(got[key] / v - 1) < 1e-4, (key, got[key], v)
    ref = O.solve_target(occ, comp, [m], kd, [1, 0, 0], [0, 1, 0], [0, 1, 0], "GKDLDR",
                         tol=1e-11)
    for l in range(2):
        assert abs(out["Qext"][l] / ref["Qext"][l] - 1) < 1e-6
        assert abs(out["Qabs"][l] / ref["Qabs"][l] - 1) < 1e-6


@pytest.mark.parametrize("solver", ["bicgstab", "qmr", "bicgstab2", "gpbicg", "petrkp"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_device_loop_equals_host_checked_blocks(B, solver, precision):
    """Without profiling a Krylov solve runs its blocks of iterations as one
    device-side loop (a CUDA-graph while-node that stops when every right-hand
    side is frozen); with per-pass profiling the host checks the flags after
    each block.  Both run the same kernels on the same data: bit-identical P,
    iterations and residuals, also when max_iter stops the solve mid-way (a
    remainder shorter than a block runs on the host)."""
    w = W.small_ellipsoid(8, 12, 32, m=1.5 + 0.1j, kd=0.4, method="LDR", n_orient=3)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    kw = dict(yhat=w.yhat, npol=2, tol=1e-9, precision=precision, solver=solver)
    a = t.solve(w.kd, w.khat, w.e01, profile=False, **kw)
    b = t.solve(w.kd, w.khat, w.e01, profile=True, **kw)
    assert a["status"] == B.DDA_OK
    for key in ("P", "iters", "resid", "Qext"):
        assert np.array_equal(a[key], b[key]), key
    if precision == "fp64":
        c = t.solve(w.kd, w.khat, w.e01, profile=False, max_iter=10, **dict(kw, tol=1e-14))
        d = t.solve(w.kd, w.khat, w.e01, profile=True, max_iter=10, **dict(kw, tol=1e-14))
        assert c["status"] == B.DDA_ERR_NOCONV
        assert np.array_equal(c["P"], d["P"]) and np.array_equal(c["iters"], d["iters"])
        assert np.all(c["iters"] <= 10 + (1 if solver == "bicgstab2" else 0))
    t.close()


@pytest.mark.parametrize("k", [1, 3])
def test_fp32_bicgstab_iterates_within_the_fp32_error_bound(B, k):
    """The FP32 Krylov solve -- FP32 vectors and FFT passes, inner products
    summed in FP32 within each thread (chunks of 8) and block (shuffle tree)
    and in FP64 across blocks -- follows the oracle's FP64 BiCGSTAB: after k
    iterations (from the same zero start and shadow vector) the GPU iterate
    differs from the oracle's by a relative amount set by FP32 rounding.  The
    inner products alone stay within (m/8 + 15) 2^-24 of sum |terms| for m
    terms per thread (a few 1e-7 here), a product through five FFT passes of
    length <= 64 within ~1e-6; through the k-th iterate these compound to a few
    1e-6 per iteration, so the bound asserted is 2e-5 k.  A reduction that lost
    a block or a chunk would move alpha and omega by ~1/(number of blocks), at
    the percent level on this size (~40 k vector elements, dozens of blocks per
    pass).  The FP64 solve meets the FP64 bar on the same iterates."""
    w = W.small_ellipsoid(20, 24, 28, m=1.5 + 0.1j, kd=0.3, method="LDR")
    flat, pos = O.site_positions(w.occ)
    e1, _ = O.polarization_pair(w.khat[0], w.e01[0])
    ainv = O.site_alpha_inverse(w.comp.reshape(-1)[flat], w.m, w.method, w.kd, w.khat[0], e1)
    E = O.incident_field(pos, w.kd, w.khat[0], e1).reshape(-1)
    ainv_box = np.zeros(w.occ.size, np.complex128)
    ainv_box[flat] = ainv
    op = O.FFTOperator(w.occ, ainv_box.reshape(w.occ.shape), w.kd, w.method)

    def mv(v):
        return O.box_to_sites(op(O.sites_to_box(v.reshape(-1, 3), flat, w.occ.shape)),
                              flat).reshape(-1)
    xo, it, _ = O.bicgstab(mv, E, tol=0.0, maxiter=k)
    assert it == k
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    for precision, bound in (("fp64", 1e-9), ("fp32", 2e-5 * k)):
        g = t.solve(w.kd, w.khat, w.e01, yhat=w.yhat, npol=1, tol=1e-14, max_iter=k,
                    precision=precision)
        assert g["iters"][0] == k
        rel = np.linalg.norm(g["P"][0].reshape(-1) - xo) / np.linalg.norm(xo)
        assert rel < bound, (precision, k, rel)
    t.close()
