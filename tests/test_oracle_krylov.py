"""Pins of the oracle's GPBi-CG and normal-equation CG (oracle/krylov.py)
against what the mathematics fixes: the solution of a small dense
complex-symmetric system (numpy.linalg.solve), GPBi-CG's first step being
BiCGSTAB's (eta = 0 at n = 0), the first CGNR iterate's closed form, CGNR's
monotone residual and its termination in at most n steps on an n x n system."""
import numpy as np
import pytest

from oracle import dda as O
from oracle import krylov as K


def _system(n, shift, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = a + a.T + shift * np.eye(n)        # complex symmetric, like the DDA matrix
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return a, b


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gpbicg_solves_complex_symmetric_system(seed):
    a, b = _system(40, 12.0, seed)
    x, it = K.gpbicg(lambda v: a @ v, b, maxiter=400, tol=1e-12)
    ref = np.linalg.solve(a, b)
    assert np.linalg.norm(b - a @ x) <= 1e-11 * np.linalg.norm(b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    assert it < 400


@pytest.mark.parametrize("seed", [0, 1])
def test_cgnr_solves_complex_symmetric_system(seed):
    a, b = _system(30, 10.0, seed)
    x, it = K.cgnr(lambda v: a @ v, b, maxiter=2000, tol=1e-12)
    ref = np.linalg.solve(a, b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()


def test_gpbicg_first_step_is_bicgstab():
    a, b = _system(25, 8.0, 3)
    mv = lambda v: a @ v
    x1, n1 = K.gpbicg(mv, b, maxiter=1)
    y1, _, _ = O.bicgstab(mv, b, tol=0.0, maxiter=1)
    assert n1 == 1
    assert np.abs(x1 - y1).max() <= 1e-13 * np.abs(y1).max()
    # from the second step on eta != 0 and the iterates differ
    x2, _ = K.gpbicg(mv, b, maxiter=2)
    y2, _, _ = O.bicgstab(mv, b, tol=0.0, maxiter=2)
    assert np.abs(x2 - y2).max() > 1e-8 * np.abs(y2).max()


def test_cgnr_first_iterate_closed_form():
    a, b = _system(20, 6.0, 4)
    x1, _ = K.cgnr(lambda v: a @ v, b, maxiter=1)
    s = a.conj().T @ b                      # A^H b
    w = a @ s
    ref = (np.vdot(s, s).real / np.vdot(w, w).real) * s
    assert np.abs(x1 - ref).max() <= 1e-13 * np.abs(ref).max()


def test_cgnr_monotone_residual_and_n_step_termination():
    n = 12
    a, b = _system(n, 9.0, 5)
    res = []
    for k in range(1, n + 1):
        x, _ = K.cgnr(lambda v: a @ v, b, maxiter=k)
        res.append(np.linalg.norm(b - a @ x))
    assert all(r2 <= r1 * (1 + 1e-12) for r1, r2 in zip(res, res[1:]))
    # CG on the n x n normal equations reaches the solution in n steps
    assert res[-1] <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qmr_solves_and_keeps_its_residual_bound(seed):
    """QMR for A = A^T reaches the dense solution, and after every iteration k
    the true residual stays below tau_k sqrt(k + 1), the bound its stopping
    rule relies on."""
    a, b = _system(30, 10.0, seed)
    mv = lambda v: a @ v
    x, it, _ = K.qmr_sym(mv, b, maxiter=400, tol=1e-12)
    ref = np.linalg.solve(a, b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    for k in range(1, 25):
        xk, _, taus = K.qmr_sym(mv, b, maxiter=k)
        assert np.linalg.norm(b - a @ xk) <= taus[-1] * np.sqrt(k + 1) * (1 + 1e-10)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bicgstab2_solves_and_its_recursive_residual_is_true(seed):
    """BiCGstab(2) reaches the dense solution, and after every cycle the
    recursively updated residual equals b - A x (a dropped or mis-signed term in
    any of the updates breaks this identity)."""
    a, b = _system(30, 10.0, seed)
    mv = lambda v: a @ v
    x, c, _ = K.bicgstab2(mv, b, ncycles=300, tol=1e-12)
    ref = np.linalg.solve(a, b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    for k in range(1, 6):
        xk, _, rk = K.bicgstab2(mv, b, ncycles=k)
        assert np.abs(rk - (b - a @ xk)).max() <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("seed", [0, 1])
def test_gpbicg_recursive_residual_is_true(seed):
    """GPBi-CG's coupled x, z, u and r updates keep r = b - A x after every
    iteration."""
    a, b = _system(30, 10.0, seed)
    mv = lambda v: a @ v
    for k in range(1, 8):
        xk, _, rk = K.gpbicg(mv, b, maxiter=k, return_r=True)
        assert np.abs(rk - (b - a @ xk)).max() <= 1e-11 * np.linalg.norm(b)
