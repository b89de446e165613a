"""ctypes binding of libdda.so (include/dda.h): argument marshalling only.

Every function here has the name of the C entry point it calls and converts
numpy arrays to the plain pointers and sizes of the C ABI; all computation
happens in the CUDA library.  Importing this module loads libdda.so and raises
if it is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdda.so")

DDA_OK, DDA_ERR_INVALID_ARG, DDA_ERR_OOM, DDA_ERR_CUDA, DDA_ERR_NOCONV, \
    DDA_ERR_BREAKDOWN, DDA_ERR_TIMEOUT = range(7)
POL = {"CM": 0, "LDR": 1, "FCD": 2, "GKDLDR": 3}
PREC = {"fp64": 0, "fp32": 1, "fp32_refined": 2, "df64": 3}
SOLVER = {"bicgstab": 0, "qmr": 1, "bicgstab2": 2, "gpbicg": 3, "petrkp": 4}

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


class SolveParams(ct.Structure):
    _fields_ = [("kd", ct.c_double), ("n_inc", ct.c_int), ("khat", _dp), ("yhat", _dp),
                ("e01", _dp), ("npol", ct.c_int), ("tol", ct.c_double),
                ("max_iter", ct.c_int), ("precision", ct.c_int), ("inner_tol", ct.c_double),
                ("n_dirs", ct.c_int), ("dirs", _dp), ("P0", _dp), ("profile", ct.c_int),
                ("solver", ct.c_int), ("fp64_residual", ct.c_int),
                ("cuda_stream", ct.c_void_p)]


class SolveResult(ct.Structure):
    _fields_ = [("P", _dp), ("Qext", _dp), ("Qabs", _dp), ("Qsca", _dp), ("famp", _dp),
                ("iters", _ip), ("resid", _dp), ("sweeps", _ip),
                ("t_setup_ms", ct.c_double), ("t_solve_ms", ct.c_double),
                ("matvecs", ct.c_int64), ("matvecs_fp64", ct.c_int64),
                ("kernel_ms", ct.c_double * 10), ("kernel_calls", ct.c_int64 * 10),
                ("launches", ct.c_int64)]

class OrientParams(ct.Structure):
    _fields_ = [("kd", ct.c_double), ("range", ct.c_double * 6), ("n", ct.c_int * 3),
                ("e01_lab", _dp), ("tol", ct.c_double), ("max_iter", ct.c_int),
                ("precision", ct.c_int), ("solver", ct.c_int), ("eta", ct.c_double),
                ("n_sel", ct.c_int), ("sel", _dp), ("max_rhs", ct.c_int)]


class OrientResult(ct.Structure):
    _fields_ = [("Qext", ct.c_double * 2), ("Qabs", ct.c_double * 2), ("Qsca", ct.c_double * 2),
                ("Qpha", ct.c_double * 2), ("Qsca_int", ct.c_double * 2),
                ("g", (ct.c_double * 3) * 2), ("cos2", ct.c_double * 2),
                ("Qbk", ct.c_double * 2), ("mueller", _dp), ("n_orient", ct.c_int),
                ("n_sca", ct.c_int64), ("iters", ct.c_int64), ("t_solve_ms", ct.c_double)]


PASSES = ("x_fwd", "y_fwd", "z_mul", "y_inv", "x_inv")


class DDAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(LIB_PATH)
    vp = ct.c_void_p
    lib.dda_target_create.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                      ct.c_int, _dp, ct.POINTER(vp)]
    lib.dda_target_create.restype = ct.c_int
    lib.dda_set_polarizability.argtypes = [vp, ct.c_int]
    lib.dda_set_polarizability.restype = ct.c_int
    lib.dda_matvec.argtypes = [vp, ct.c_double, _dp, _dp, _dp, _dp, ct.c_int]
    lib.dda_matvec.restype = ct.c_int
    lib.dda_solve.argtypes = [vp, ct.POINTER(SolveParams), ct.POINTER(SolveResult)]
    lib.dda_solve.restype = ct.c_int
    lib.dda_target_destroy.argtypes = [vp]
    lib.dda_target_destroy.restype = None
    lib.dda_status_string.argtypes = [ct.c_int]
    lib.dda_status_string.restype = ct.c_char_p
    lib.dda_last_error.argtypes = []
    lib.dda_last_error.restype = ct.c_char_p
    lib.dda_target_num_dipoles.argtypes = [vp]
    lib.dda_target_num_dipoles.restype = ct.c_int64
    lib.dda_solve_hbm_bytes.argtypes = [vp, ct.POINTER(SolveParams)]
    lib.dda_solve_hbm_bytes.restype = ct.c_int64
    lib.dda_estimate_solve_bytes.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int64,
                                             ct.c_int, ct.c_int, ct.POINTER(SolveParams)]
    lib.dda_estimate_solve_bytes.restype = ct.c_int64
    lib.dda_target_device_bytes.argtypes = [vp]
    lib.dda_target_device_bytes.restype = ct.c_int64
    lib.dda_target_grid.argtypes = [vp, _ip, _ip, _ip]
    lib.dda_target_grid.restype = ct.c_int
    lib.dda_launch_count.argtypes = []
    lib.dda_launch_count.restype = ct.c_int64
    lib.dda_autotune.argtypes = [vp, ct.c_double, ct.c_int]
    lib.dda_autotune.restype = ct.c_int
    lib.dda_target_schedule.argtypes = [vp, ct.c_int, _ip]
    lib.dda_target_schedule.restype = ct.c_int
    lib.dda_set_schedule.argtypes = [vp, ct.c_int, _ip]
    lib.dda_set_schedule.restype = ct.c_int
    lib.dda_matvec_noalloc.argtypes = [vp, ct.c_double, _dp, _dp, ct.c_void_p, ct.c_void_p,
                                       ct.c_int, ct.c_void_p]
    lib.dda_matvec_noalloc.restype = ct.c_int
    lib.dda_scattering_directions.argtypes = [ct.c_double, ct.c_double, ct.c_int64, _dp, _dp]
    lib.dda_scattering_directions.restype = ct.c_int64
    lib.dda_mueller.argtypes = [ct.c_int64, _dp, _dp, _dp, _dp, _dp]
    lib.dda_mueller.restype = ct.c_int
    lib.dda_orientation_grid.argtypes = [_dp, _ip, _dp, _dp, _dp, _dp, _dp]
    lib.dda_orientation_grid.restype = ct.c_int
    lib.dda_orient_average.argtypes = [vp, ct.POINTER(OrientParams), ct.POINTER(OrientResult)]
    lib.dda_orient_average.restype = ct.c_int
    lib.dda_nearfield_box.argtypes = [vp, _dp, _ip, _ip]
    lib.dda_nearfield_box.restype = ct.c_int
    lib.dda_nearfield.argtypes = [vp, ct.POINTER(SolveParams), _dp, _dp, _dp, _dp, _dp, _dp,
                                  _dp]
    lib.dda_nearfield.restype = ct.c_int
    return lib


lib = _load()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _check(status, allow=()):
    if status != DDA_OK and status not in allow:
        raise DDAError(status, f"{lib.dda_status_string(status).decode()}: "
                               f"{lib.dda_last_error().decode()}")
    return status


def dda_status_string(status: int) -> str:
    return lib.dda_status_string(status).decode()


def dda_last_error() -> str:
    return lib.dda_last_error().decode()


def dda_launch_count() -> int:
    return int(lib.dda_launch_count())


def dda_target_create(occ: np.ndarray, comp: np.ndarray | None, m) -> int:
    """occ/comp: (nz, ny, nx) arrays; m: complex refractive indices.  Returns a handle."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    nz, ny, nx = occ.shape
    if comp is not None:
        comp = np.ascontiguousarray(comp, dtype=np.uint8)
    mm = np.ascontiguousarray(np.array(m, dtype=np.complex128).view(np.float64))
    h = ct.c_void_p()
    _check(lib.dda_target_create(nx, ny, nz, occ.ctypes.data,
                                 None if comp is None else comp.ctypes.data,
                                 len(m), _ptr(mm), ct.byref(h)))
    return h.value


def dda_set_polarizability(h, method: str) -> None:
    _check(lib.dda_set_polarizability(h, POL[method]))


def dda_target_destroy(h) -> None:
    lib.dda_target_destroy(h)


def dda_target_num_dipoles(h) -> int:
    return int(lib.dda_target_num_dipoles(h))


def dda_target_grid(h):
    a, b, c = ct.c_int(), ct.c_int(), ct.c_int()
    _check(lib.dda_target_grid(h, ct.byref(a), ct.byref(b), ct.byref(c)))
    return a.value, b.value, c.value


def dda_matvec(h, kd: float, x: np.ndarray, khat=None, e=None, precision="fp64") -> np.ndarray:
    """y = A x; x: [N, 3] complex on the occupied sites (flat-index order)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(x)
    kh = None if khat is None else np.ascontiguousarray(khat, dtype=np.float64)
    ee = None if e is None else np.ascontiguousarray(np.asarray(e, np.complex128).view(np.float64))
    _check(lib.dda_matvec(h, float(kd), _ptr(kh), _ptr(ee), _ptr(x.view(np.float64)),
                          _ptr(y.view(np.float64)), PREC[precision]))
    return y


def dda_autotune(h, kd: float, n_rhs: int) -> None:
    _check(lib.dda_autotune(h, float(kd), int(n_rhs)))


def dda_target_schedule(h, precision="fp32") -> dict:
    out = (ct.c_int * 8)()
    _check(lib.dda_target_schedule(h, PREC[precision], out))
    return dict(x_lines=out[0], y_tile=out[1], z_tile=out[2], z_pitch=out[3],
                z_stage_ghat=out[4], x_threads=out[5], y_threads=out[6], z_threads=out[7])


SCHEDULE_KEYS = ("x_lines", "y_tile", "z_tile", "z_pitch", "z_stage_ghat", "x_threads",
                 "y_threads", "z_threads")


def dda_set_schedule(h, schedule: dict, precision="fp32") -> None:
    vals = (ct.c_int * 8)(*[int(schedule[k]) for k in SCHEDULE_KEYS])
    _check(lib.dda_set_schedule(h, PREC[precision], vals))


def dda_matvec_noalloc(h, kd: float, x_dev_ptr: int, y_dev_ptr: int, khat=None, e=None,
                       precision="fp64", stream_ptr: int = 0) -> None:
    """y = A x on caller-owned DEVICE buffers (box layout [3][nz][ny][nx], complex
    FP32 or FP64), without any device allocation by the library."""
    kh = None if khat is None else np.ascontiguousarray(khat, dtype=np.float64)
    ee = None if e is None else np.ascontiguousarray(np.asarray(e, np.complex128).view(np.float64))
    _check(lib.dda_matvec_noalloc(h, float(kd), _ptr(kh), _ptr(ee), ct.c_void_p(x_dev_ptr),
                                  ct.c_void_p(y_dev_ptr), PREC[precision],
                                  ct.c_void_p(stream_ptr) if stream_ptr else None))


def _params(kd, khat, e01, yhat, npol, tol, max_iter, precision, inner_tol, dirs, P0,
            profile=False, solver="bicgstab", fp64_residual=False, stream_ptr=0):
    keep = []

    def arr(a, dtype=np.float64):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        return a

    khat = arr(np.atleast_2d(khat))
    n_inc = khat.shape[0]
    e = arr(np.atleast_2d(np.asarray(e01, np.complex128)), np.complex128)
    yh = arr(None if yhat is None else np.atleast_2d(yhat))
    d = arr(None if dirs is None or len(dirs) == 0 else np.asarray(dirs).reshape(-1, 2))
    p0 = arr(None if P0 is None else np.asarray(P0, np.complex128), np.complex128)
    prm = SolveParams(kd=float(kd), n_inc=n_inc, khat=_ptr(khat), yhat=_ptr(yh),
                      e01=_ptr(e.view(np.float64)), npol=int(npol), tol=float(tol),
                      max_iter=int(max_iter), precision=PREC[precision],
                      inner_tol=float(inner_tol), n_dirs=0 if d is None else d.shape[0],
                      dirs=_ptr(d), P0=None if p0 is None else _ptr(p0.view(np.float64)),
                      profile=1 if profile else 0, solver=SOLVER[solver],
                      fp64_residual=1 if fp64_residual else 0,
                      cuda_stream=ct.c_void_p(stream_ptr) if stream_ptr else None)
    return prm, keep, n_inc


def dda_solve_hbm_bytes(h, kd, khat, e01, npol=2, precision="fp64", dirs=None,
                       solver="bicgstab") -> int:
    prm, keep, _ = _params(kd, khat, e01, None, npol, 1e-8, 1, precision, 0.0, dirs, None,
                           solver=solver)
    return int(lib.dda_solve_hbm_bytes(h, ct.byref(prm)))


def dda_estimate_solve_bytes(occ, ncomp, method, kd, khat, e01, npol=2,
                             precision="fp64", dirs=None, solver="bicgstab") -> int:
    """Device bytes a new target of this occupancy needs at the peak of its first
    solve (host-only: nothing is allocated)."""
    nz, ny, nx = np.asarray(occ).shape
    prm, keep, _ = _params(kd, khat, e01, None, npol, 1e-8, 1, precision, 0.0, dirs, None,
                           solver=solver)
    b = int(lib.dda_estimate_solve_bytes(nx, ny, nz, int(np.count_nonzero(occ)), int(ncomp),
                                         POL[method], ct.byref(prm)))
    if b < 0:
        raise DDAError(DDA_ERR_INVALID_ARG, "bad arguments to dda_estimate_solve_bytes")
    return b


def dda_target_device_bytes(h) -> int:
    return int(lib.dda_target_device_bytes(h))


def dda_solve(h, kd, khat, e01, yhat=None, npol=2, tol=1e-8, max_iter=2000,
              precision="fp64", inner_tol=0.0, dirs=None, P0=None, want_P=True,
              want_famp=True, raise_on_noconv=False, profile=False,
              solver="bicgstab", fp64_residual=False, stream_ptr: int = 0) -> dict:
    """Solve for every incidence x polarization.  Returns a dict of numpy arrays.
    solver: "bicgstab" (two matvecs per iteration), "qmr" (complex-symmetric
    QMR, one matvec per iteration), "bicgstab2" (BiCGstab(2), four matvecs per
    two-iteration cycle), "gpbicg" (GPBi-CG, two matvecs per iteration) or
    "petrkp" (conjugate gradients on the normal equations, two matvecs per
    iteration).  stream_ptr: a cudaStream_t (e.g. torch.cuda.Stream().cuda_stream)
    on which the library runs the solve; 0 = the target's own stream."""
    prm, keep, n_inc = _params(kd, khat, e01, yhat, npol, tol, max_iter, precision,
                               inner_tol, dirs, P0, profile, solver, fp64_residual,
                               stream_ptr)
    N = dda_target_num_dipoles(h)
    R = n_inc * npol
    D = prm.n_dirs + 1
    out = dict(P=np.empty((R, N, 3), np.complex128) if want_P else None,
               Qext=np.empty(R), Qabs=np.empty(R), Qsca=np.empty(R),
               famp=np.empty((n_inc, D, 2, npol), np.complex128) if want_famp else None,
               iters=np.empty(R, np.int32), resid=np.empty(R), sweeps=np.empty(R, np.int32))
    res = SolveResult(
        P=None if out["P"] is None else _ptr(out["P"].view(np.float64)),
        Qext=_ptr(out["Qext"]), Qabs=_ptr(out["Qabs"]), Qsca=_ptr(out["Qsca"]),
        famp=None if out["famp"] is None else _ptr(out["famp"].view(np.float64)),
        iters=out["iters"].ctypes.data_as(_ip), resid=_ptr(out["resid"]),
        sweeps=out["sweeps"].ctypes.data_as(_ip))
    st = lib.dda_solve(h, ct.byref(prm), ct.byref(res))
    allow = () if raise_on_noconv else (DDA_ERR_NOCONV,)
    _check(st, allow)
    out["status"] = st
    out["t_setup_ms"] = res.t_setup_ms
    out["t_solve_ms"] = res.t_solve_ms
    out["matvecs"] = res.matvecs
    out["matvecs_fp64"] = res.matvecs_fp64
    out["launches"] = res.launches
    if profile:
        out["kernel_ms"] = {(p, PASSES[i]): res.kernel_ms[5 * k + i]
                            for k, p in enumerate(("fp32", "fp64")) for i in range(5)}
        out["kernel_calls"] = {(p, PASSES[i]): res.kernel_calls[5 * k + i]
                               for k, p in enumerate(("fp32", "fp64")) for i in range(5)}
    return out


def dda_nearfield_box(h, ext):
    """(dims, lo): extended box (nx', ny', nz') and the target's offset in it."""
    e = np.ascontiguousarray(ext, np.float64)
    if e.shape != (6,):
        raise ValueError("ext must hold 6 values (-x, +x, -y, +y, -z, +z)")
    dims = (ct.c_int * 3)()
    lo = (ct.c_int * 3)()
    _check(lib.dda_nearfield_box(h, _ptr(e), dims, lo))
    return tuple(dims), tuple(lo)


def dda_nearfield(h, kd, khat, e01, P, ext, npol=2, want=("E_inc", "E_sca", "E_macro")):
    """Near field of the dipoles P (as returned by dda_solve for the same
    incidences) on the extended box.  Arrays have shape (n_rhs, 3, nz', ny', nx')."""
    prm, keep, n_inc = _params(kd, khat, e01, None, npol, 1e-8, 1, "fp64", 0.0, None, None)
    dims, lo = dda_nearfield_box(h, ext)
    R = n_inc * npol
    P = np.ascontiguousarray(P, np.complex128)
    N = dda_target_num_dipoles(h)
    if P.shape != (R, N, 3):
        raise ValueError(f"P must have shape {(R, N, 3)}")
    e = np.ascontiguousarray(ext, np.float64)
    shape = (R, 3, dims[2], dims[1], dims[0])
    keys = ("E_inc", "E_sca", "E_macro", "B_inc", "B_sca")
    bad = set(want) - set(keys)
    if bad:
        raise ValueError(f"unknown near-field outputs {sorted(bad)}")
    out = {k: np.empty(shape, np.complex128) if k in want else None for k in keys}
    _check(lib.dda_nearfield(h, ct.byref(prm), _ptr(P.view(np.float64)), _ptr(e),
                             *[None if out[k] is None else _ptr(out[k].view(np.float64))
                               for k in keys]))
    out["dims"], out["lo"] = dims, lo
    return out


def dda_scattering_directions(x, eta):
    """(theta [n], phi [n], omega [n]) of the averaging direction set."""
    n = lib.dda_scattering_directions(float(x), float(eta), 0, None, None)
    if n < 0:
        raise DDAError(DDA_ERR_INVALID_ARG, "x must be > 0 and eta >= 1e-3")
    tp = np.empty((n, 2))
    om = np.empty(n)
    lib.dda_scattering_directions(float(x), float(eta), n, _ptr(tp), _ptr(om))
    return tp[:, 0].copy(), tp[:, 1].copy(), om


def dda_mueller(f, e01_lab, phi_s):
    """f [n, 2 (m), 2 (l)] complex, e01_lab [3] complex, phi_s [n] ->
    (S [n, 4] complex S_1..S_4, M [n, 4, 4])."""
    f = np.ascontiguousarray(f, np.complex128)
    n = f.shape[0]
    e = np.ascontiguousarray(e01_lab, np.complex128)
    ph = np.ascontiguousarray(phi_s, np.float64)
    S = np.empty((n, 4), np.complex128)
    M = np.empty((n, 4, 4))
    _check(lib.dda_mueller(n, _ptr(f.view(np.float64)), _ptr(e.view(np.float64)), _ptr(ph),
                           _ptr(S.view(np.float64)), _ptr(M)))
    return S, M


def dda_orientation_grid(beta, nbeta, theta, ntheta, phi, nphi):
    rng = np.array([beta[0], beta[1], theta[0], theta[1], phi[0], phi[1]], np.float64)
    n = (ct.c_int * 3)(nbeta, ntheta, nphi)
    b, t, p = np.empty(nbeta), np.empty(ntheta), np.empty(nphi)
    wb, wa = np.empty(nbeta), np.empty((ntheta, nphi))
    _check(lib.dda_orientation_grid(_ptr(rng), n, _ptr(b), _ptr(t), _ptr(p), _ptr(wb), _ptr(wa)))
    return b, t, p, wb, wa


def dda_orient_average(h, kd, beta=(0.0, 0.0), nbeta=1, theta=(0.0, 0.0), ntheta=1,
                       phi=(0.0, 0.0), nphi=1, e01_lab=(0, 1, 0), tol=1e-8, max_iter=2000,
                       precision="fp32_refined", solver="bicgstab", eta=0.0, sel=(),
                       max_rhs=0) -> dict:
    """Orientation-averaged efficiencies, angular averages and Mueller matrix."""
    e = np.ascontiguousarray(e01_lab, np.complex128)
    sl = np.ascontiguousarray(np.asarray(sel, np.float64).reshape(-1, 2))
    prm = OrientParams(kd=float(kd), e01_lab=_ptr(e.view(np.float64)), tol=float(tol),
                       max_iter=int(max_iter), precision=PREC[precision],
                       solver=SOLVER[solver], eta=float(eta), n_sel=sl.shape[0],
                       sel=_ptr(sl) if sl.shape[0] else None, max_rhs=int(max_rhs))
    prm.range[:] = [beta[0], beta[1], theta[0], theta[1], phi[0], phi[1]]
    prm.n[:] = [nbeta, ntheta, nphi]
    mu = np.empty((sl.shape[0], 4, 4))
    res = OrientResult(mueller=_ptr(mu) if sl.shape[0] else None)
    st = lib.dda_orient_average(h, ct.byref(prm), ct.byref(res))
    _check(st, (DDA_ERR_NOCONV,))
    out = {k: np.array(getattr(res, k)[:]) for k in ("Qext", "Qabs", "Qsca", "Qpha",
                                                      "Qsca_int", "cos2", "Qbk")}
    out["g"] = np.array([list(res.g[0]), list(res.g[1])])
    out["mueller"] = mu
    out.update(status=st, n_orient=res.n_orient, n_sca=res.n_sca, iters=res.iters,
               t_solve_ms=res.t_solve_ms)
    return out


class Target:
    """Owning wrapper around a dda_target handle."""

    def __init__(self, occ, comp=None, m=(1.5 + 0j,), method="LDR"):
        self.h = dda_target_create(occ, comp, list(m))
        self.shape = tuple(np.asarray(occ).shape[::-1])
        dda_set_polarizability(self.h, method)

    def close(self):
        if self.h:
            dda_target_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_dipoles(self):
        return dda_target_num_dipoles(self.h)

    @property
    def grid(self):
        return dda_target_grid(self.h)

    def set_polarizability(self, method):
        dda_set_polarizability(self.h, method)

    def matvec(self, kd, x, khat=None, e=None, precision="fp64"):
        return dda_matvec(self.h, kd, x, khat, e, precision)

    def solve(self, kd, khat, e01, **kw):
        return dda_solve(self.h, kd, khat, e01, **kw)

    def hbm_bytes(self, kd, khat, e01, **kw):
        return dda_solve_hbm_bytes(self.h, kd, khat, e01, **kw)

    @property
    def device_bytes(self):
        return dda_target_device_bytes(self.h)

    def orient_average(self, kd, **kw):
        return dda_orient_average(self.h, kd, **kw)

    def nearfield(self, kd, khat, e01, P, ext, **kw):
        return dda_nearfield(self.h, kd, khat, e01, P, ext, **kw)

    def set_schedule(self, schedule, precision="fp32"):
        dda_set_schedule(self.h, schedule, precision)

    def schedule(self, precision="fp32"):
        return dda_target_schedule(self.h, precision)

    def autotune(self, kd, n_rhs):
        dda_autotune(self.h, kd, n_rhs)
        return {p: dda_target_schedule(self.h, p) for p in ("fp32", "fp64")}
