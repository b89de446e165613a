"""The allocation-free matvec entry point against the ordinary one.

dda_matvec_noalloc serves callers that must not allocate device memory (a host
framework that owns the device heap, serving loops that cannot afford the
device-wide synchronization of cudaFree, real-time loops).  It runs the same
FFT-convolution kernels with the scratch in a fixed static device array, on
buffers the caller provides.  Here the caller's buffers come from torch; the
results must match dda_matvec (the existing entry point) to the tolerances the
matvec parity tests use, on two calls in a row (the second sees the first
call's leftovers in the shared array).  The calls must also leave the device's
free memory unchanged, and a call that follows one which filled the shared
array with NaN must still return finite, matching values.  This file is
collected last.
"""
import numpy as np
import pytest

from dda_inputs import targets as tg
from dda_inputs import workloads as W
from oracle import dda as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


def _box(x_sites, flat, occ, dtype):
    import torch
    b = O.sites_to_box(x_sites, flat, occ.shape)
    return torch.from_numpy(np.ascontiguousarray(b.astype(dtype))).cuda()


def _err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("method", ["LDR", "FCD", "GKDLDR"])
def test_noalloc_matvec_matches_matvec_twice(method):
    import torch
    from paper_1305_6497_gb300 import binding as B
    w = W.two_material_brick(9, 7, 11, method=method)
    flat, _ = O.site_positions(w.occ)
    khat = np.array([0.36, 0.48, 0.8])
    e = np.array([0.8, -0.6, 0.0], np.complex128)
    t = B.Target(w.occ, w.comp, w.m, method=method)
    for call, seed in enumerate((21, 22)):
        x = O.box_to_sites(W.random_polarization(w.occ, seed)[0], flat)
        for prec, dt, tol in (("fp64", np.complex128, TOL64), ("fp32", np.complex64, TOL32)):
            ref = t.matvec(w.kd, x, khat, e, prec)       # existing entry point
            xd = _box(x, flat, w.occ, dt)
            yd = torch.full_like(xd, complex(7.0, -3.0))  # stale values must be overwritten
            torch.cuda.synchronize()
            B.dda_matvec_noalloc(t.h, w.kd, xd.data_ptr(), yd.data_ptr(), khat, e, prec)
            y = O.box_to_sites(yd.cpu().numpy().astype(np.complex128), flat)
            assert _err(y, ref) <= tol, (method, prec, call, _err(y, ref))
            vac = (w.occ == 0)
            assert np.all(yd.cpu().numpy()[:, vac] == 0)
    t.close()


def test_noalloc_rejects_missing_green_transform_and_oversize():
    from paper_1305_6497_gb300 import binding as B
    import torch
    occ, comp = tg.sphere(8)
    t = B.Target(occ, comp, [1.5 + 0.1j], method="CM")
    xd = torch.zeros((3, 8, 8, 8), dtype=torch.complex128, device="cuda")
    yd = torch.zeros_like(xd)
    with pytest.raises(B.DDAError):        # no transform built for this kd yet
        B.dda_matvec_noalloc(t.h, 0.3, xd.data_ptr(), yd.data_ptr())
    t.close()
    occ, comp = tg.rect_prism(96, 96, 96)   # 3*96*192*192 FP64 values > 64 MiB
    t = B.Target(occ, comp, [1.5 + 0.1j], method="CM")
    with pytest.raises(B.DDAError) as ei:
        B.dda_matvec_noalloc(t.h, 0.3, xd.data_ptr(), yd.data_ptr())
    assert "static area" in str(ei.value)
    t.close()


def test_noalloc_allocates_nothing_and_ignores_leftovers():
    """Free device memory is the same before and after every call, the first
    one included (the static array was committed when the target was created;
    the warm-up dda_matvec built the Green transform and launched the kernels);
    a NaN-filled shared array from another target's call changes nothing."""
    import torch
    from paper_1305_6497_gb300 import binding as B
    w = W.two_material_brick(9, 7, 11, method="LDR")
    flat, _ = O.site_positions(w.occ)
    khat = np.array([0.0, 0.6, 0.8])
    e = np.array([1.0, 0.0, 0.0], np.complex128)
    x = O.box_to_sites(W.random_polarization(w.occ, 31)[0], flat)
    t = B.Target(w.occ, w.comp, w.m, method="LDR")
    # a second, larger target whose call fills more of the shared array with NaN
    occ2, comp2 = tg.rect_prism(20, 18, 16)
    t2 = B.Target(occ2, comp2, [1.4 + 0.05j], method="LDR")
    flat2, _ = O.site_positions(occ2)
    refs, bufs = {}, {}
    for prec, dt in (("fp64", np.complex128), ("fp32", np.complex64)):
        refs[prec] = t.matvec(w.kd, x, khat, e, prec)
        t2.matvec(w.kd, np.ones((len(flat2), 3), np.complex128), khat, e, prec)
        xd = _box(x, flat, w.occ, dt)
        nd = torch.full((3,) + occ2.shape, complex(np.nan, np.nan),
                        dtype=torch.complex128 if prec == "fp64" else torch.complex64,
                        device="cuda") * torch.from_numpy(
                            (occ2 != 0).astype(np.float32)).cuda()
        bufs[prec] = (xd, torch.empty_like(xd), nd, torch.empty_like(nd))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for rnd in range(2):
        for prec, tol in (("fp64", TOL64), ("fp32", TOL32)):
            xd, yd, nd, nyd = bufs[prec]
            B.dda_matvec_noalloc(t2.h, w.kd, nd.data_ptr(), nyd.data_ptr(), khat, e, prec)
            assert torch.cuda.mem_get_info()[0] == free0, (prec, rnd)
            B.dda_matvec_noalloc(t.h, w.kd, xd.data_ptr(), yd.data_ptr(), khat, e, prec)
            assert torch.cuda.mem_get_info()[0] == free0, (prec, rnd)
            y = O.box_to_sites(yd.cpu().numpy().astype(np.complex128), flat)
            assert np.all(np.isfinite(y)), (prec, rnd)
            assert _err(y, refs[prec]) <= tol, (prec, rnd, _err(y, refs[prec]))
    t.close()
    t2.close()
