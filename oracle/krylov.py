"""More Krylov methods for the oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy restatements of four more of the guide's iterative options
(Sec. "Choice of Iterative Algorithm"), each written from its published
definition, so that tests can compare the GPU iterates with them step by step.
Only the tests may import this module; the CUDA library never does.

  qmr_sym -- QMR for complex-symmetric A (Freund 1992; coupled two-term
            recurrences, Freund & Nachtigal 1994), the guide's QMRCCG option
  bicgstab2 -- BiCGstab(l) with l = 2 (Sleijpen & van der Vorst 1993), the
            guide's PBCGS2 option
  gpbicg -- GPBi-CG (Zhang 1997), the guide's GPBICG option
  cgnr   -- conjugate gradients on the normal equations A^H A x = A^H b
            (Petravic & Kuo-Petravic 1979), the guide's PETRKP option

Each takes the matrix as a function v -> A v.  <a, b> = sum conj(a) b.
"""
import numpy as np


def _dot(a, b):
    return np.vdot(a, b)


def gpbicg(matvec, b, maxiter, tol=0.0, return_r=False):
    """GPBi-CG from x0 = 0 with shadow vector rt = r0 = b.

    Iteration n (t, u, z, A t, A p start at zero and beta at 0):
      p = r + beta (p - u);  w = A t_{n-1} + beta A p_{n-1}
      alpha = <rt, r> / <rt, A p>
      y = t_{n-1} - r - alpha w + alpha A p;  t = r - alpha A p
      (zeta, eta) minimise ||t - zeta A t - eta y|| (eta = 0 at n = 0):
        the 2x2 normal equations [<At,At> <At,y>; <y,At> <y,y>] (zeta, eta)
        = (<At,t>, <y,t>)
      u = zeta A p + eta (t_{n-1} - r + beta u);  z = zeta r + eta z - alpha u
      x = x + alpha p + z;  r = t - eta y - zeta A t
      beta = (alpha / zeta) <rt, r_new> / <rt, r>
    Stops after `maxiter` iterations or when ||r|| <= tol ||b||.
    Returns (x, iterations), and the recursively updated r when return_r."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    rt = r.copy()
    p = np.zeros_like(b)
    u = np.zeros_like(b)
    z = np.zeros_like(b)
    t_old = np.zeros_like(b)
    at_old = np.zeros_like(b)
    ap_old = np.zeros_like(b)
    beta = 0.0
    rho = _dot(rt, r)
    bn = np.linalg.norm(b)
    n = 0
    while n < maxiter and np.linalg.norm(r) > tol * bn:
        p = r + beta * (p - u)
        w = at_old + beta * ap_old
        ap = matvec(p)
        alpha = rho / _dot(rt, ap)
        y = t_old - r - alpha * w + alpha * ap
        t = r - alpha * ap
        at = matvec(t)
        aa = _dot(at, at).real
        if n == 0:
            zeta, eta = _dot(at, t) / aa, 0.0
        else:
            yy = _dot(y, y).real
            ay = _dot(at, y)
            m = np.array([[aa, ay], [np.conj(ay), yy]])
            zeta, eta = np.linalg.solve(m, np.array([_dot(at, t), _dot(y, t)]))
        u = zeta * ap + eta * (t_old - r + beta * u)
        z = zeta * r + eta * z - alpha * u
        x = x + alpha * p + z
        r_new = t - eta * y - zeta * at
        rho_new = _dot(rt, r_new)
        beta = (alpha / zeta) * rho_new / rho
        r, rho = r_new, rho_new
        t_old, at_old, ap_old = t, at, ap
        n += 1
    return (x, n, r) if return_r else (x, n)


def cgnr(matvec, b, maxiter, tol=0.0):
    """Conjugate gradients on A^H A x = A^H b from x0 = 0, for complex-symmetric
    A (A^T = A), so that A^H v = conj(A conj(v)):
      r = b;  p = A^H r;  gamma = ||A^H r||^2
      w = A p;  alpha = gamma / ||w||^2;  x += alpha p;  r -= alpha w
      s = A^H r;  beta = ||s||^2 / gamma;  gamma = ||s||^2;  p = s + beta p
    Stops after `maxiter` iterations or when ||r|| <= tol ||b||.
    Returns (x, iterations)."""
    b = np.asarray(b, dtype=np.complex128)
    ah = lambda v: np.conj(matvec(np.conj(v)))
    x = np.zeros_like(b)
    r = b.copy()
    p = ah(r)
    gamma = _dot(p, p).real
    bn = np.linalg.norm(b)
    n = 0
    while n < maxiter and np.linalg.norm(r) > tol * bn:
        w = matvec(p)
        alpha = gamma / _dot(w, w).real
        x = x + alpha * p
        r = r - alpha * w
        n += 1
        if np.linalg.norm(r) <= tol * bn:
            break
        s = ah(r)
        g_new = _dot(s, s).real
        p = s + (g_new / gamma) * p
        gamma = g_new
    return x, n


def qmr_sym(matvec, b, maxiter, tol=0.0):
    """QMR for A = A^T from x0 = 0: the Lanczos process on the bilinear form
    x^T y, whose vectors are the BiCG residuals, with the quasi-residual
    minimised by Givens rotations in the coupled two-term form:
      r = b;  q = r;  tau = ||r||;  theta = 0;  rho = r^T r;  d = 0
      t = A q;  alpha = rho / (q^T t);  r -= alpha t
      theta' = ||r|| / tau;  c^2 = 1 / (1 + theta'^2);  tau = tau theta' c
      d = c^2 theta^2 d + c^2 alpha q;  x += d;  theta = theta'
      rho' = r^T r;  beta = rho' / rho;  q = r + beta q
    Stops after `maxiter` iterations or when tau sqrt(k + 1) <= tol ||b||.
    Returns (x, iterations, taus) with taus[k] the tau after iteration k + 1."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    q = r.copy()
    d = np.zeros_like(b)
    tau = np.linalg.norm(r)
    theta = 0.0
    rho = np.sum(r * r)
    bn = np.linalg.norm(b)
    taus = []
    n = 0
    while n < maxiter:
        t = matvec(q)
        alpha = rho / np.sum(q * t)
        r = r - alpha * t
        th = np.linalg.norm(r) / tau
        c2 = 1.0 / (1.0 + th * th)
        tau = tau * th * np.sqrt(c2)
        d = c2 * theta * theta * d + c2 * alpha * q
        x = x + d
        theta = th
        n += 1
        taus.append(tau)
        if tau * np.sqrt(n + 1) <= tol * bn:
            break
        rho_new = np.sum(r * r)
        q = r + (rho_new / rho) * q
        rho = rho_new
    return x, n, taus


def bicgstab2(matvec, b, ncycles, tol=0.0):
    """BiCGstab(2) from x0 = 0 with shadow vector rt = r0 = b.  Each cycle
    (four matvecs, counted as two iterations):
      rho0 = -omega rho0
      for j = 0, 1:
        rho1 = <rt, r_j>;  beta = alpha rho1 / rho0;  rho0 = rho1
        u_i = r_i - beta u_i (i <= j);  u_{j+1} = A u_j
        alpha = rho0 / <rt, u_{j+1}>
        r_i = r_i - alpha u_{i+1} (i <= j);  r_{j+1} = A r_j;  x = x + alpha u_0
      (g1, g2) minimise ||r_0 - g1 r_1 - g2 r_2|| (2x2 normal equations)
      u_0 -= g1 u_1 + g2 u_2;  x += g1 r_0 + g2 r_1;  r_0 -= g1 r_1 + g2 r_2;
      omega = g2
    Starts from rho0 = 1, alpha = 0, omega = 1, u_0 = 0.  Stops after
    `ncycles` cycles or when ||r_0|| <= tol ||b||.  Returns (x, cycles, r0),
    r0 the recursively updated residual."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = [b.copy(), None, None]
    u = [np.zeros_like(b), None, None]
    rt = b.copy()
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    bn = np.linalg.norm(b)
    c = 0
    while c < ncycles and np.linalg.norm(r[0]) > tol * bn:
        rho0 = -omega * rho0
        for j in range(2):
            rho1 = _dot(rt, r[j])
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = matvec(u[j])
            alpha = rho0 / _dot(rt, u[j + 1])
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = matvec(r[j])
            x = x + alpha * u[0]
        m = np.array([[_dot(r[1], r[1]), _dot(r[1], r[2])],
                      [_dot(r[2], r[1]), _dot(r[2], r[2])]])
        g1, g2 = np.linalg.solve(m, np.array([_dot(r[1], r[0]), _dot(r[2], r[0])]))
        u[0] = u[0] - g1 * u[1] - g2 * u[2]
        x = x + g1 * r[0] + g2 * r[1]
        r[0] = r[0] - g1 * r[1] - g2 * r[2]
        omega = g2
        c += 1
    return x, c, r[0]
