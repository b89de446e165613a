"""CPU oracle for the discrete-dipole solve -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 numpy/scipy code that computes what the DDSCAT 7.3 guide's
method computes, written from its definitions so that a reader can check each
step against the paper.  Only the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this package; the CUDA library never does,
and nothing here imports the CUDA library.

Units: lattice units, d = 1, so "k" below is k*d.  Time dependence exp(-i w t),
Gaussian units (the guide follows Draine 1988).

Contents, each citing the passage it follows:
  site_positions           -- targets as lists of occupied lattice sites (Sec.
                              "Target Geometry: The Target Frame")
  alpha_cm / polarizability -- Clausius-Mossotti, CM with radiative reaction,
                              LATTDR and FLTRCD (Sec. "Choice of DDA Method")
  incident_field           -- E_inc,j = e exp(i k khat.r_j) (Sec. "Incident
                              Polarization State", "Target Orientation")
  green_point, green_fcd   -- the interaction tensors entering A (eq. AP=E)
  matvec_direct, dense_matrix, fft_matvec -- A.P by direct summation, as a
                              dense matrix, and by the FFT convolution the
                              guide's ESELF uses (Sec. "Choice of FFT Algorithm")
  bicgstab                 -- BiCGSTAB (van der Vorst 1992), the PIM method the
                              guide's PBCGST option runs (Sec. "Choice of
                              Iterative Algorithm")
  cross_sections           -- Q_ext, Q_abs, Q_sca (Sec. "What Does It Calculate?")
  scattering_amplitudes    -- f_ml (eq. f_ml_def)
  nearfield_box, nearfield -- E_inc, E_sca, E_macro, B_inc, B_sca in and
                              around the target on an extended box (Sec.
                              "Near-Field Calculations", eq. macro_vs_micro)

Readings where the guide is silent or garbled are stated at each function and
collected in the design notes.  LATTDR's coefficients b1, b2, b3 (Draine &
Goodman 1993, cited by the guide without printing them) and the GKDLDR tensor
form are pinned by the dispersion relation of the infinite lattice, evaluated
by Ewald summation in the tests; everything else is pinned by tests against
closed forms, invariants or independent library routines.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

# LATTDR coefficients of Draine & Goodman (1993), cited by the guide (Sec.
# "Point Dipoles: Options LATTDR and GKDLDR") without printing them.  They are
# the (kd)^2 coefficients of the infinite cubic lattice's dipole sum for a wave
# of index m (tests/test_oracle_lattice_dispersion.py derives them).
LDR_B1 = -1.8915316
LDR_B2 = 0.1648469
LDR_B3 = -1.7700004

METHODS = ("CM", "LDR", "FCD", "GKDLDR")


# --------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------
def site_positions(occ: np.ndarray):
    """Occupied sites of an (nz, ny, nx) occupancy grid, in flat-index order.

    Returns (flat_index [N], pos [N, 3]) with pos = (ix, iy, iz) - (n - 1)/2:
    lattice sites x_j = [(i, j, k) + x0] d with the origin at the box centre.
    """
    nz, ny, nx = occ.shape
    iz, iy, ix = np.nonzero(occ)
    flat = ix + nx * (iy + ny * iz)
    pos = np.stack([ix - 0.5 * (nx - 1), iy - 0.5 * (ny - 1), iz - 0.5 * (nz - 1)],
                   axis=1).astype(np.float64)
    return flat.astype(np.int64), pos


def effective_radius(n_dipoles: int) -> float:
    """a_eff = (3 V / 4 pi)^(1/3) with V = N d^3 (Sec. "Applicability of the DDA")."""
    return (3.0 * n_dipoles / (4.0 * math.pi)) ** (1.0 / 3.0)


# --------------------------------------------------------------------------
# Polarizabilities (Sec. "Choice of DDA Method")
# --------------------------------------------------------------------------
def alpha_cm(m: complex) -> complex:
    """Clausius-Mossotti polarizability 3 d^3/(4 pi) (m^2 - 1)/(m^2 + 2)."""
    m2 = complex(m) ** 2
    return 3.0 / (4.0 * math.pi) * (m2 - 1.0) / (m2 + 2.0)


def ldr_s(khat, e) -> float:
    """S = sum_j (khat_j e_j)^2 for a unit propagation vector and unit
    polarization; for a complex e the squared modulus |e_j|^2 is used (the
    guide does not print S; for linear polarization both readings agree)."""
    khat = np.asarray(khat, dtype=np.float64)
    e = np.asarray(e, dtype=np.complex128)
    e = e / np.linalg.norm(e)
    return float(np.sum(khat ** 2 * np.abs(e) ** 2))


def polarizability(method: str, m: complex, kd: float, khat=None, e=None) -> complex:
    """Dipole polarizability alpha (units d^3) for refractive index m.

    CM:  alpha_CM / [1 - (2/3) i (kd)^3 alpha_CM]   (Clausius-Mossotti with the
         radiative-reaction correction; without it C_abs < 0 for real m).
    LDR: alpha_CM / {1 + alpha_CM [(b1 + m^2 b2 + m^2 b3 S)(kd)^2 - (2/3) i (kd)^3]}
         (LATTDR, Draine & Goodman 1993).
    FCD: alpha_CM / {1 - alpha_CM [(4/3)(kd)^2 + (2/(3 pi)) ln((pi-kd)/(pi+kd)) (kd)^3
                                  + (2/3) i (kd)^3]}
         (FLTRCD).  The guide prints "1 + D" and omits (kd)^3 on the log term;
         read literally, C_abs < 0 for real m and Re(1/alpha) is odd in k.  The
         reading here restores C_abs = 0 for real m and alpha(-k) = conj(alpha(k)).
    """
    a0 = alpha_cm(m)
    k = float(kd)
    m2 = complex(m) ** 2
    if method == "CM":
        return a0 / (1.0 - (2.0 / 3.0) * 1j * k ** 3 * a0)
    if method == "LDR":
        S = ldr_s(khat, e)
        return a0 / (1.0 + a0 * ((LDR_B1 + m2 * LDR_B2 + m2 * LDR_B3 * S) * k ** 2
                                 - (2.0 / 3.0) * 1j * k ** 3))
    if method == "GKDLDR":
        raise ValueError("GKDLDR is a tensor: use polarizability_tensor")
    if method == "FCD":
        logt = math.log((math.pi - k) / (math.pi + k))
        return a0 / (1.0 - a0 * ((4.0 / 3.0) * k ** 2
                                 + (2.0 / (3.0 * math.pi)) * logt * k ** 3
                                 + (2.0 / 3.0) * 1j * k ** 3))
    raise ValueError(f"unknown polarizability method {method!r}")


def polarizability_tensor(method: str, m: complex, kd: float, khat=None, e=None):
    """Diagonal of the polarizability tensor on the lattice axes x, y, z.

    GKDLDR (Sec. "Point Dipoles: Options LATTDR and GKDLDR": the lattice
    dispersion relation as corrected by Gutkowicz-Krusin & Draine 2004; the
    guide does not print it):
        alpha_a = alpha_CM / {1 + alpha_CM [(b1 + m^2 b2 + m^2 b3 khat_a^2)(kd)^2
                                           - (2/3) i (kd)^3]},   a = x, y, z.
    Reading: the lattice must carry a wave of index m along khat for BOTH
    transverse polarizations, so the transverse block of 1/alpha must equal
    that of the lattice's dipole sum; its (kd)^2 term is
    (b1 + m^2 b2) I + m^2 b3 diag(khat_a^2) there (the Ewald test), which a
    tensor diagonal on the lattice axes matches with khat_a^2 in place of
    LATTDR's S = sum_a (khat_a e_a)^2 (S = e . diag(khat_a^2) . e for real e).
    It does not depend on the polarization.  The scalar methods return their
    alpha on all three axes.  Returns a complex [3] array (units d^3)."""
    if method != "GKDLDR":
        return np.full(3, polarizability(method, m, kd, khat, e), dtype=np.complex128)
    a0 = alpha_cm(m)
    k = float(kd)
    m2 = complex(m) ** 2
    kh = np.asarray(khat, dtype=np.float64)
    kh = kh / np.linalg.norm(kh)
    return np.array([a0 / (1.0 + a0 * ((LDR_B1 + m2 * LDR_B2 + m2 * LDR_B3 * kh[a] ** 2)
                                       * k ** 2 - (2.0 / 3.0) * 1j * k ** 3))
                     for a in range(3)])


def site_alpha_inverse(comp_sites: np.ndarray, m_list, method, kd, khat=None, e=None):
    """1/alpha_j for each occupied site (comp_sites in 1..ncomp): [N] for the
    scalar methods, [N, 3] (the tensor's diagonal) for GKDLDR."""
    idx = np.asarray(comp_sites, dtype=np.int64) - 1
    if method == "GKDLDR":
        inv = np.array([1.0 / polarizability_tensor(method, mm, kd, khat, e) for mm in m_list])
        return inv[idx]
    inv = np.array([1.0 / polarizability(method, mm, kd, khat, e) for mm in m_list])
    return inv[idx]


def _per_axis(ainv: np.ndarray) -> np.ndarray:
    """[N] or [N, 3] inverse polarizabilities as [N, 3]."""
    ainv = np.asarray(ainv)
    return np.repeat(ainv[:, None], 3, axis=1) if ainv.ndim == 1 else ainv


# --------------------------------------------------------------------------
# Incident wave
# --------------------------------------------------------------------------
def polarization_pair(khat, e01):
    """(e01, e02) with e01 normalized and e02 = khat x conj(e01)."""
    khat = np.asarray(khat, dtype=np.float64)
    e1 = np.asarray(e01, dtype=np.complex128)
    e1 = e1 / np.sqrt(np.sum(np.abs(e1) ** 2))
    e2 = np.cross(khat, np.conj(e1))
    return e1, e2


def incident_field(pos: np.ndarray, kd: float, khat, e) -> np.ndarray:
    """E_inc,j = e exp(i k khat . r_j), |E_0| = 1 at the origin.  [N, 3]."""
    phase = np.exp(1j * kd * (pos @ np.asarray(khat, dtype=np.float64)))
    return phase[:, None] * np.asarray(e, dtype=np.complex128)[None, :]


# --------------------------------------------------------------------------
# Interaction tensors
# --------------------------------------------------------------------------
def green_point(dr: np.ndarray, kd: float) -> np.ndarray:
    """Field tensor of a point dipole: E(r) = G(r) . P with

        G(r) P = e^{ikr}/r^3 { k^2 r^2 (rhat x P) x rhat + (1 - ikr)[3 rhat(rhat.P) - P] }

    i.e. G = (k^2 I + grad grad) e^{ikr}/r at r != 0 (Draine 1988).  dr [..., 3]
    nonzero; returns [..., 3, 3] complex.
    """
    dr = np.asarray(dr, dtype=np.float64)
    r = np.sqrt(np.sum(dr * dr, axis=-1))
    n = dr / r[..., None]
    nn = n[..., :, None] * n[..., None, :]
    eye = np.eye(3)
    k = float(kd)
    kr = np.asarray(k * r)
    pref = np.asarray(np.exp(1j * kr) / r ** 3)
    t = (kr ** 2)[..., None, None] * (eye - nn) + \
        np.asarray(1.0 - 1j * kr)[..., None, None] * (3.0 * nn - eye)
    return pref[..., None, None] * t


def filtered_scalar_green(r, kd, kf=math.pi):
    """Band-limited outgoing scalar Green function and its first two r-derivatives.

    g_F(r) = (2/(pi r)) int_0^{kF} q sin(q r) / (q^2 - k^2 - i0) dq, the field of a
    point source with spatial frequencies |q| > kF = pi/d removed (the filtered
    coupled dipole idea, Sec. "Filtered Coupled Dipole").  Splitting
    q/(q^2-k^2) into partial fractions gives the closed form

        r g_F = i sin(kr) + (1/pi)[cos(kr) S(r) + sin(kr) C(r)],
        S = Si((kF-k) r) + Si((kF+k) r),  C = Ci((kF-k) r) - Ci((kF+k) r),

    which tends to e^{ikr} as kF -> infinity.  Returns (g, g', g'').
    """
    r = np.asarray(r, dtype=np.float64)
    k = float(kd)
    a, b = kf - k, kf + k
    si_a, ci_a = special.sici(a * r)
    si_b, ci_b = special.sici(b * r)
    S = si_a + si_b
    C = ci_a - ci_b
    S1 = (np.sin(a * r) + np.sin(b * r)) / r
    C1 = (np.cos(a * r) - np.cos(b * r)) / r
    S2 = (a * np.cos(a * r) + b * np.cos(b * r)) / r - S1 / r
    C2 = (-a * np.sin(a * r) + b * np.sin(b * r)) / r - C1 / r
    c, s = np.cos(k * r), np.sin(k * r)
    h = 1j * s + (c * S + s * C) / math.pi
    h1 = 1j * k * c + (-k * s * S + c * S1 + k * c * C + s * C1) / math.pi
    h2 = -1j * k * k * s + (-k * k * c * S - 2 * k * s * S1 + c * S2
                            - k * k * s * C + 2 * k * c * C1 + s * C2) / math.pi
    g = h / r
    g1 = h1 / r - h / r ** 2
    g2 = h2 / r - 2.0 * h1 / r ** 2 + 2.0 * h / r ** 3
    return g, g1, g2


def green_fcd(dr: np.ndarray, kd: float) -> np.ndarray:
    """Filtered interaction tensor G_F = (k^2 I + grad grad) g_F at r != 0.

    For a radial g: d_a d_b g = n_a n_b g'' + (delta_ab - n_a n_b) g'/r.
    """
    dr = np.asarray(dr, dtype=np.float64)
    r = np.sqrt(np.sum(dr * dr, axis=-1))
    n = dr / r[..., None]
    nn = n[..., :, None] * n[..., None, :]
    eye = np.eye(3)
    g, g1, g2 = filtered_scalar_green(r, kd)
    k = float(kd)
    return (np.asarray(k * k * g + g1 / r)[..., None, None] * eye
            + np.asarray(g2 - g1 / r)[..., None, None] * nn)


def green(kind: str):
    """Interaction tensor for a polarizability method: FCD uses the filtered
    one, the others (CM, LDR, GKDLDR) the point-dipole tensor."""
    return green_fcd if kind == "FCD" else green_point


def magnetic_vector(dr: np.ndarray, kd: float, kind: str = "LDR") -> np.ndarray:
    """h(r) with B(r) = h(r) x P for a dipole P at the origin (Gaussian units,
    mu = 1): the vector potential of an oscillating dipole is A = -i k P g, so
    B = curl A = -i k g'(r) rhat x P.  g = e^{ikr}/r (g' = e^{ikr}(ikr - 1)/r^2),
    or the filtered g_F for FCD.  dr [..., 3] nonzero; returns [..., 3]."""
    dr = np.asarray(dr, dtype=np.float64)
    r = np.sqrt(np.sum(dr * dr, axis=-1))
    k = float(kd)
    if kind == "FCD":
        _, g1, _ = filtered_scalar_green(r, kd)
    else:
        g1 = np.exp(1j * k * r) * (1j * k * r - 1.0) / r ** 2
    return np.asarray(-1j * k * g1)[..., None] * (dr / r[..., None])


# --------------------------------------------------------------------------
# The matrix A of eq. (AP=E):  (A P)_j = alpha_j^{-1} P_j - sum_{l != j} G(r_j - r_l) P_l
# --------------------------------------------------------------------------
def matvec_direct(P: np.ndarray, pos: np.ndarray, ainv: np.ndarray, kd: float,
                  method: str = "LDR", rows=None, block: int = 256,
                  col_block: int | None = None) -> np.ndarray:
    """A.P by direct O(N^2) summation.  P [N, 3] complex; returns [len(rows), 3].

    The interaction sum over l runs over all sites at once, or in chunks of
    `col_block` sites (for very large N; only the grouping of the sum changes).
    """
    G = green(method)
    N = pos.shape[0]
    ai = _per_axis(ainv)
    rows = np.arange(N) if rows is None else np.asarray(rows)
    cb = N if col_block is None else int(col_block)
    out = np.empty((len(rows), 3), dtype=np.complex128)
    for s in range(0, len(rows), block):
        rb = rows[s:s + block]
        field = np.zeros((len(rb), 3), dtype=np.complex128)
        for c0 in range(0, N, cb):
            cols = np.arange(c0, min(N, c0 + cb))
            dr = pos[rb, None, :] - pos[None, cols, :]          # [b, n, 3]
            self_mask = (rb[:, None] == cols[None, :])
            dr[self_mask] = 1.0                                 # placeholder, zeroed below
            T = G(dr, kd)                                       # [b, n, 3, 3]
            T[self_mask] = 0.0
            field += np.einsum("bnij,nj->bi", T, P[cols])
        out[s:s + block] = ai[rb] * P[rb] - field
    return out


def dense_matrix(pos: np.ndarray, ainv: np.ndarray, kd: float, method: str = "LDR"):
    """The full 3N x 3N matrix A (index 3 j + a)."""
    N = pos.shape[0]
    dr = pos[:, None, :] - pos[None, :, :]
    eye_mask = np.eye(N, dtype=bool)
    dr[eye_mask] = 1.0
    T = -green(method)(dr, kd)
    T[eye_mask] = 0.0
    ai = _per_axis(ainv)
    for j in range(N):
        T[j, j] = np.diag(ai[j])
    return T.transpose(0, 2, 1, 3).reshape(3 * N, 3 * N)


def fft_grid_green(shape_box, grid, kd, method="LDR", z_range=None):
    """The 6 unique components (xx, xy, xz, yy, yz, zz) of G(Delta) laid on the
    periodic FFT grid: entry (i, j, l) holds G at the lattice offset
    Delta = (i or i - Lx, ...) when |Delta| fits the target box, else 0; Delta =
    0 is 0 (the self term sits in alpha^{-1}).  Returns [6, Lz, Ly, Lx], or the
    grid planes z0 <= i_z < z1 only for z_range = (z0, z1)."""
    nx, ny, nz = shape_box
    Lx, Ly, Lz = grid
    z0, z1 = (0, Lz) if z_range is None else z_range

    def offs(n, L):
        o = np.arange(L)
        d = np.where(o < n, o, o - L).astype(np.float64)
        valid = (o < n) | (o > L - n)
        return d, valid

    dx, vx = offs(nx, Lx)
    dy, vy = offs(ny, Ly)
    dz, vz = offs(nz, Lz)
    dz, vz = dz[z0:z1], vz[z0:z1]
    DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
    valid = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
    valid &= ~((DX == 0) & (DY == 0) & (DZ == 0))
    dr = np.stack([DX, DY, DZ], axis=-1)
    dr[~valid] = 1.0
    T = green(method)(dr, kd)
    T[~valid] = 0.0
    comps = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    return np.stack([T[..., a, b] for (a, b) in comps])


def default_grid(shape_box):
    """(2nx, 2ny, 2nz): the zero-padded grid of the guide's FFT method."""
    return tuple(2 * n for n in shape_box)


class FFTOperator:
    """A.P through the circulant embedding: the interaction sum is a discrete
    convolution of P with G over lattice offsets, evaluated by 3-D FFTs on a
    grid of at least (2nx-1)(2ny-1)(2nz-1) points (Sec. "Choice of FFT
    Algorithm"; Goodman, Draine & Flatau 1990).  numpy's FFT is the primitive."""

    def __init__(self, occ, ainv_box, kd, method="LDR", grid=None):
        nz, ny, nx = occ.shape
        self.occ = occ != 0
        self.box = (nx, ny, nz)
        self.grid = tuple(grid) if grid is not None else default_grid(self.box)
        for n, L in zip(self.box, self.grid):
            if L < 2 * n - 1:
                raise ValueError("FFT grid smaller than 2n-1 wraps the convolution")
        # [nz, ny, nx] complex (0 on vacant sites), or [3, nz, ny, nx] per axis
        self.ainv = ainv_box if np.ndim(ainv_box) == 4 else np.asarray(ainv_box)[None]
        gg = fft_grid_green(self.box, self.grid, kd, method)
        self.ghat = np.fft.fftn(gg, axes=(1, 2, 3))

    def __call__(self, Pbox: np.ndarray) -> np.ndarray:
        """Pbox [3, nz, ny, nx] complex (zero on vacant sites) -> A.P, same shape."""
        nx, ny, nz = self.box
        Lx, Ly, Lz = self.grid
        pad = np.zeros((3, Lz, Ly, Lx), dtype=np.complex128)
        pad[:, :nz, :ny, :nx] = Pbox
        ph = np.fft.fftn(pad, axes=(1, 2, 3))
        g = self.ghat
        full = [[g[0], g[1], g[2]], [g[1], g[3], g[4]], [g[2], g[4], g[5]]]
        eh = np.stack([sum(full[a][b] * ph[b] for b in range(3)) for a in range(3)])
        field = np.fft.ifftn(eh, axes=(1, 2, 3))[:, :nz, :ny, :nx]
        out = self.ainv * Pbox - field
        return out * self.occ[None]


class FFTOperatorLowMem:
    """The same A.P as FFTOperator, for grids where FFTOperator's arrays holding
    all components at once do not fit in host memory (the 512^3 grid of a 256^3
    box: its [3, 3] tensor on the grid alone is 19 GB).  Only the grouping of
    the work changes, not the arithmetic of any element:
      * G is laid on the grid a few z-planes at a time (fft_grid_green with a
        z_range) and each of its six components is transformed on its own;
      * each polarization component is padded and transformed on its own, and
        each output component's sum_b Ghat_ab Phat_b is formed and inverted on
        its own;
      * the FFTs are scipy.fft's (the library primitive, on `workers` host
        threads) and the element-wise products run over z-slabs on host
        threads.
    Memory: 6 + 3 + 2 grid arrays of complex128 (26 GB on a 512^3 grid)."""

    def __init__(self, occ, ainv_box, kd, method="LDR", grid=None, workers=None,
                 slab=8):
        import os
        from concurrent.futures import ThreadPoolExecutor
        from scipy import fft as sfft
        self._sfft = sfft
        nz, ny, nx = occ.shape
        self.occ = occ != 0
        self.box = (nx, ny, nz)
        self.grid = tuple(grid) if grid is not None else default_grid(self.box)
        for n, L in zip(self.box, self.grid):
            if L < 2 * n - 1:
                raise ValueError("FFT grid smaller than 2n-1 wraps the convolution")
        self.ainv = ainv_box if np.ndim(ainv_box) == 4 else np.asarray(ainv_box)[None]
        self.workers = workers or os.cpu_count() or 1
        self._pool = ThreadPoolExecutor(self.workers)
        Lx, Ly, Lz = self.grid
        self.ghat = np.empty((6, Lz, Ly, Lx), dtype=np.complex128)
        for z0 in range(0, Lz, slab):
            z1 = min(Lz, z0 + slab)
            self.ghat[:, z0:z1] = fft_grid_green(self.box, self.grid, kd, method, (z0, z1))
        for c in range(6):
            self.ghat[c] = sfft.fftn(self.ghat[c], workers=self.workers, overwrite_x=True)
        self._slabs = [(z0, min(Lz, z0 + slab)) for z0 in range(0, Lz, slab)]

    def _pointwise_sum(self, out, pairs):
        """out = sum over (g, p) in pairs of g * p, z-slab by z-slab."""
        def work(zr):
            z0, z1 = zr
            g, p = pairs[0]
            np.multiply(g[z0:z1], p[z0:z1], out=out[z0:z1])
            for g, p in pairs[1:]:
                out[z0:z1] += g[z0:z1] * p[z0:z1]
        list(self._pool.map(work, self._slabs))

    def __call__(self, Pbox: np.ndarray) -> np.ndarray:
        """Pbox [3, nz, ny, nx] complex (zero on vacant sites) -> A.P, same shape."""
        nx, ny, nz = self.box
        Lx, Ly, Lz = self.grid
        sfft = self._sfft
        ph = np.empty((3, Lz, Ly, Lx), dtype=np.complex128)
        for b in range(3):
            pad = np.zeros((Lz, Ly, Lx), dtype=np.complex128)
            pad[:nz, :ny, :nx] = Pbox[b]
            ph[b] = sfft.fftn(pad, workers=self.workers, overwrite_x=True)
            del pad
        g = self.ghat
        full = [[g[0], g[1], g[2]], [g[1], g[3], g[4]], [g[2], g[4], g[5]]]
        out = np.empty((3, nz, ny, nx), dtype=np.complex128)
        eh = np.empty((Lz, Ly, Lx), dtype=np.complex128)
        for a in range(3):
            self._pointwise_sum(eh, [(full[a][b], ph[b]) for b in range(3)])
            field = sfft.ifftn(eh, workers=self.workers)[:nz, :ny, :nx]
            out[a] = self.ainv[a if len(self.ainv) == 3 else 0] * Pbox[a] - field
            del field
        return out * self.occ[None]


# --------------------------------------------------------------------------
# BiCGSTAB (van der Vorst 1992) -- the PIM method behind the PBCGST option
# --------------------------------------------------------------------------
def bicgstab(matvec, b: np.ndarray, tol: float = 1e-11, maxiter: int = 10000, x0=None):
    """Solve A x = b.  Stops when ||b - A x|| / ||b|| <= tol (the recursively
    updated residual, re-checked against the true residual at exit).
    Returns (x, iterations, true relative residual)."""
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - matvec(x) if x0 is not None else b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    while it < maxiter:
        if np.linalg.norm(r) / bnorm <= tol:
            break
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        it += 1
        if np.linalg.norm(s) / bnorm <= tol:
            x = x + alpha * p
            r = s
            break
        t = matvec(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
    res = np.linalg.norm(b - matvec(x)) / bnorm
    return x, it, float(res)


# --------------------------------------------------------------------------
# Observables
# --------------------------------------------------------------------------
def cross_sections(P: np.ndarray, E: np.ndarray, ainv: np.ndarray, kd: float):
    """(Q_ext, Q_abs, Q_sca) for one incident polarization with |E_0| = 1.

    C_ext = 4 pi k sum_j Im(E_inc,j^* . P_j)
    C_abs = 4 pi k sum_j sum_a |P_ja|^2 [-Im(1/alpha_ja) - (2/3) k^3]
    (the work done on each dipole component; for a scalar alpha the familiar
    |P_j|^2 [-Im(1/alpha_j) - (2/3) k^3])
    Q = C / (pi a_eff^2), Q_sca = Q_ext - Q_abs (Sec. "What Does It
    Calculate?": Q_ext = Q_sca + Q_abs).
    """
    k = float(kd)
    N = P.shape[0]
    aeff = effective_radius(N)
    cext = 4.0 * math.pi * k * float(np.sum(np.imag(np.conj(E) * P)))
    cabs = 4.0 * math.pi * k * float(np.sum(np.abs(P) ** 2 * (-np.imag(_per_axis(ainv))
                                                              - (2.0 / 3.0) * k ** 3)))
    g = math.pi * aeff * aeff
    qext, qabs = cext / g, cabs / g
    return qext, qabs, qext - qabs


def scattering_frame(khat, yhat, theta, phi):
    """(n_s, theta_hat, phi_hat) in TF coordinates for a Lab-Frame direction.

    The Lab Frame has x_LF = khat and y_LF = yhat; n_s = x cos(theta) +
    y sin(theta) cos(phi) + z sin(theta) sin(phi) (Sec. "Scattering Directions", "Isolated Finite Targets",
    LFRAME), theta_hat = dn/dtheta, phi_hat = (dn/dphi)/sin(theta).
    """
    x = np.asarray(khat, dtype=np.float64)
    y = np.asarray(yhat, dtype=np.float64)
    z = np.cross(x, y)
    ct, st = math.cos(theta), math.sin(theta)
    cp, sp = math.cos(phi), math.sin(phi)
    n = x * ct + y * st * cp + z * st * sp
    th = -x * st + y * ct * cp + z * ct * sp
    ph = -y * sp + z * cp
    return n, th, ph


def scattering_amplitudes(P_l, pos, kd, khat, yhat, dirs):
    """f_ml for each direction (eq. f_ml_def with Draine 1988's convention).

    The far field of the dipoles is E_s = k^2 e^{ikr}/r sum_j [P_j - n(n.P_j)]
    e^{-ik n.r_j}; projecting on e_1 = theta_hat, e_2 = phi_hat and matching
    E_s.e_m = e^{ikr}/(kr) f_ml (E_inc(0).e_0l^* = 1 for the l-th solve) gives
    f_ml = k^3 e_m . sum_j P_j^{(l)} e^{-ik n.r_j}.

    P_l: list of [N, 3] arrays (one per incident polarization l).
    dirs: [D, 2] (theta_s, phi_s) radians.  Returns [D, 2 (m), npol (l)] complex.
    """
    k = float(kd)
    out = np.empty((len(dirs), 2, len(P_l)), dtype=np.complex128)
    for d, (th_s, ph_s) in enumerate(dirs):
        n, th, ph = scattering_frame(khat, yhat, th_s, ph_s)
        w = np.exp(-1j * k * (pos @ n))
        for l, P in enumerate(P_l):
            F = np.sum(P * w[:, None], axis=0)
            out[d, 0, l] = k ** 3 * np.dot(th, F)
            out[d, 1, l] = k ** 3 * np.dot(ph, F)
    return out


# --------------------------------------------------------------------------
# Whole solve for one target
# --------------------------------------------------------------------------
def box_to_sites(vbox: np.ndarray, flat: np.ndarray) -> np.ndarray:
    """[3, nz, ny, nx] -> [N, 3] on the occupied sites (flat-index order)."""
    return vbox.reshape(3, -1)[:, flat].T.copy()


def sites_to_box(v: np.ndarray, flat: np.ndarray, shape) -> np.ndarray:
    out = np.zeros((3, int(np.prod(shape))), dtype=np.complex128)
    out[:, flat] = v.T
    return out.reshape((3,) + tuple(shape))


def solve_target(occ, comp, m_list, kd, khat, yhat, e01, method="LDR", npol=2,
                 tol=1e-11, dirs=None, operator="fft", maxiter=20000, grid=None,
                 workers=None, on_matvec=None):
    """Solve A P = E_inc for each incident polarization of one incidence.

    operator: 'fft' (FFT convolution), 'fft_lowmem' (the same with
    FFTOperatorLowMem), 'direct' (O(N^2) sum) or 'dense' (LU).
    workers: host threads of FFTOperatorLowMem; on_matvec: optional callable
    invoked after every product (progress reporting only).
    Returns a dict with P (list of [N,3]), Qext/Qabs/Qsca, iters, resid, famp.
    """
    flat, pos = site_positions(occ)
    comp_sites = comp.reshape(-1)[flat]
    e1, e2 = polarization_pair(khat, e01)
    pols = [e1, e2][:npol]
    out = dict(P=[], Qext=[], Qabs=[], Qsca=[], iters=[], resid=[])
    for e in pols:
        ainv = site_alpha_inverse(comp_sites, m_list, method, kd, khat, e)
        E = incident_field(pos, kd, khat, e)
        if operator == "dense":
            A = dense_matrix(pos, ainv, kd, method)
            P = np.linalg.solve(A, E.reshape(-1)).reshape(-1, 3)
            it = 0
            res = float(np.linalg.norm(E.reshape(-1) - A @ P.reshape(-1))
                        / np.linalg.norm(E))
        elif operator == "direct":
            def mv(x):
                return matvec_direct(x.reshape(-1, 3), pos, ainv, kd, method).reshape(-1)
            x, it, res = bicgstab(mv, E.reshape(-1), tol, maxiter)
            P = x.reshape(-1, 3)
        elif operator in ("fft", "fft_lowmem"):
            ainv_box = np.zeros((3, occ.size), dtype=np.complex128)
            ainv_box[:, flat] = _per_axis(ainv).T
            if operator == "fft":
                op = FFTOperator(occ, ainv_box.reshape((3,) + occ.shape), kd, method, grid)
            else:
                op = FFTOperatorLowMem(occ, ainv_box.reshape((3,) + occ.shape), kd, method,
                                       grid, workers)
            shape = occ.shape

            def mv(x):
                xb = sites_to_box(x.reshape(-1, 3), flat, shape)
                y = box_to_sites(op(xb), flat).reshape(-1)
                if on_matvec is not None:
                    on_matvec()
                return y
            x, it, res = bicgstab(mv, E.reshape(-1), tol, maxiter)
            P = x.reshape(-1, 3)
        else:
            raise ValueError(operator)
        qe, qa, qs = cross_sections(P, E, ainv, kd)
        out["P"].append(P)
        out["Qext"].append(qe)
        out["Qabs"].append(qa)
        out["Qsca"].append(qs)
        out["iters"].append(it)
        out["resid"].append(res)
    d_all = np.concatenate([np.zeros((1, 2)), np.asarray(dirs if dirs is not None
                                                          else np.zeros((0, 2)))])
    out["famp"] = scattering_amplitudes(out["P"], pos, kd, khat, yhat, d_all)
    return out


# --------------------------------------------------------------------------
# Near field (Sec. "Near-Field Calculations")
# --------------------------------------------------------------------------
def nearfield_box(shape_zyx, ext):
    """Extended box of the NRFLD option: the target's box (nz, ny, nx) grown by
    r1 n_x sites below and r2 n_x above along x, r3, r4 along y, r5, r6 along z
    (Sec. "Additional Nearfield Calculation?"), each rounded to the nearest
    integer (halves away from zero).  Returns (dims (nx', ny', nz'), lo (x, y, z))."""
    nz, ny, nx = shape_zyx
    n = (nx, ny, nz)
    lo, dims = [], []
    for a in range(3):
        rl, rh = float(ext[2 * a]), float(ext[2 * a + 1])
        l = int(math.floor(rl * n[a] + 0.5))
        h = int(math.floor(rh * n[a] + 0.5))
        lo.append(l)
        dims.append(n[a] + l + h)
    return tuple(dims), tuple(lo)


def nearfield(occ, comp, m_list, kd, khat, e, method, P, ext, points=None):
    """Fields of the dipoles P [N, 3] (target sites in flat-index order) at the
    sites of the extended box, by direct summation:

      E_sca(r) = sum over target sites l with r_l != r of G(r - r_l) P_l
                 (G = green_point, or green_fcd for FCD: the tensor of the solve),
      E_inc(r) = e exp(i k khat . r), with r measured from the target's centre,
      E_macro  = 3 / (eps + 2) (E_inc + E_sca) on target sites of refractive
                 index m (eps = m^2, eq. macro_vs_micro), E_inc + E_sca in vacuum,
      B_sca(r) = sum over target sites l with r_l != r of h(r - r_l) x P_l,
      B_inc    = khat x E_inc (the plane wave's magnetic field).

    Returns a dict of arrays [3, nz', ny', nx'] (or [n_points, 3] for the flat
    indices `points` of the extended box), plus dims and lo.
    """
    dims, lo = nearfield_box(occ.shape, ext)
    nxe, nye, nze = dims
    nz, ny, nx = occ.shape
    flat, pos = site_positions(occ)
    comp_sites = comp.reshape(-1)[flat]
    G = green(method)
    allpts = np.arange(nxe * nye * nze) if points is None else np.asarray(points)
    ix = allpts % nxe
    iy = (allpts // nxe) % nye
    iz = allpts // (nxe * nye)
    r = np.stack([ix - lo[0] - 0.5 * (nx - 1), iy - lo[1] - 0.5 * (ny - 1),
                  iz - lo[2] - 0.5 * (nz - 1)], axis=1).astype(np.float64)
    esca = np.zeros((len(allpts), 3), np.complex128)
    bsca = np.zeros((len(allpts), 3), np.complex128)
    for s0 in range(0, len(allpts), 64):
        rb = r[s0:s0 + 64]
        dr = rb[:, None, :] - pos[None, :, :]
        same = np.all(dr == 0.0, axis=-1)
        dr[same] = 1.0
        T = G(dr, kd)
        T[same] = 0.0
        esca[s0:s0 + 64] = np.einsum("bnij,nj->bi", T, P)
        hv = magnetic_vector(dr, kd, method)
        hv[same] = 0.0
        bsca[s0:s0 + 64] = np.cross(hv, P[None, :, :]).sum(axis=1)
    einc = incident_field(r, kd, khat, e)
    binc = np.cross(np.asarray(khat, np.float64)[None, :], einc)
    # composition at each point (0 = vacuum)
    inside = (ix >= lo[0]) & (ix < lo[0] + nx) & (iy >= lo[1]) & (iy < lo[1] + ny) & \
             (iz >= lo[2]) & (iz < lo[2] + nz)
    cpt = np.zeros(len(allpts), np.int64)
    cpt[inside] = comp[iz[inside] - lo[2], iy[inside] - lo[1], ix[inside] - lo[0]]
    fac = np.ones(len(allpts), np.complex128)
    for c, m in enumerate(m_list, start=1):
        fac[cpt == c] = 3.0 / (complex(m) ** 2 + 2.0)
    emacro = fac[:, None] * (einc + esca)
    out = dict(dims=dims, lo=lo, comp=cpt)
    for k, v in (("E_inc", einc), ("E_sca", esca), ("E_macro", emacro), ("B_inc", binc),
                 ("B_sca", bsca)):
        out[k] = v if points is not None else v.T.reshape(3, nze, nye, nxe)
    return out
