// The lattice Green tensor and its transform on the padded FFT grid.
//
// A_jl = -G(r_j - r_l) for j != l (eq. AP=E).  CM and LDR use the point-dipole
// tensor G = (k^2 I + grad grad) e^{ikr}/r, i.e.
//   G_ab = A(r) delta_ab + B(r) n_a n_b,
//   A = e^{ikr}/r^3 ((kr)^2 - 1 + ikr),  B = e^{ikr}/r^3 (3 - (kr)^2 - 3ikr).
// FCD (Sec. "Filtered Coupled Dipole") uses (k^2 I + grad grad) g_F with g_F
// the outgoing scalar Green function with spatial frequencies above kF = pi/d
// removed; splitting q/(q^2-k^2) into partial fractions gives
//   r g_F = i sin(kr) + [cos(kr) S(r) + sin(kr) C(r)] / pi,
//   S = Si((kF-k)r) + Si((kF+k)r),  C = Ci((kF-k)r) - Ci((kF+k)r),
// and for a radial g: d_a d_b g = n_a n_b g'' + (delta_ab - n_a n_b) g'/r.
//
// G is laid on the periodic grid at offsets |Delta_x| < nx etc. (zero
// elsewhere, zero at Delta = 0), transformed by the same Stockham kernels as
// the matvec (FP64), and one octant of the transform is kept: components xx,
// yy, zz are even in every axis, xy is odd in x and y, xz in x and z, yz in y
// and z, so Ghat(L - k) = +/- Ghat(k) per axis.
#include <cmath>

#include "dda_ops.h"
#include "fft_core.cuh"

namespace dda {

// Si(x), Ci(x) for x > 0: power series below x = 2, and above it the
// continued fraction of E1(ix) = -Ci(x) + i (Si(x) - pi/2) (modified Lentz),
// E1(z) = e^{-z} / (z + 1 - 1/(z + 3 - 4/(z + 5 - ...))).
__device__ void sici(double x, double& si, double& ci) {
  const double kEuler = 0.57721566490153286061;
  const double kPiHalf = 1.57079632679489661923;
  if (x <= 2.0) {
    // Si = sum (-1)^n x^(2n+1) / ((2n+1)(2n+1)!), Ci = gamma + ln x + sum_{n>=1} (-1)^n x^(2n)/(2n (2n)!)
    double term = x;  // x^(2n+1)/(2n+1)! with sign
    double s = x;
    double fact_term = 1.0;  // x^(2n)/(2n)! with sign
    double c = 0.0;
    const double x2 = x * x;
    for (int n = 1; n < 40; ++n) {
      fact_term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n));
      c += fact_term / (2.0 * n);
      term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
      const double add = term / (2.0 * n + 1.0);
      s += add;
      if (fabs(add) < 1e-18 * fabs(s) && fabs(fact_term) < 1e-18) break;
    }
    si = s;
    ci = kEuler + log(x) + c;
    return;
  }
  // modified Lentz on b0 + a1/(b1 + a2/(b2 + ...)), b_n = z + 2n + 1, a_n = -n^2
  const double tiny = 1e-300;
  double2 b = make_double2(1.0, x);               // z + 1, z = i x
  double2 cc = make_double2(1.0 / tiny, 0.0);
  double2 d = make_double2(b.x / (b.x * b.x + b.y * b.y), -b.y / (b.x * b.x + b.y * b.y));
  double2 h = d;
  for (int n = 1; n < 400; ++n) {
    const double a = -(double)n * n;
    b.x += 2.0;
    // d = 1/(a d + b), c = b + a/c
    double2 ad = make_double2(a * d.x + b.x, a * d.y + b.y);
    const double dn = ad.x * ad.x + ad.y * ad.y;
    d = make_double2(ad.x / dn, -ad.y / dn);
    const double cn = cc.x * cc.x + cc.y * cc.y;
    cc = make_double2(b.x + a * cc.x / cn, b.y - a * cc.y / cn);
    const double2 del = cmul(cc, d);
    h = cmul(h, del);
    if (fabs(del.x - 1.0) + fabs(del.y) < 1e-16) break;
  }
  // E1(ix) = e^{-ix} h
  double sx, cx;
  sincos(x, &sx, &cx);
  const double2 e1 = cmul(make_double2(cx, -sx), h);
  ci = -e1.x;
  si = kPiHalf + e1.y;
}

// The scalar Green function at r > 0 and its first two radial derivatives:
// point g = e^{ikr}/r, or the filtered g_F (FCD).
__device__ void scalar_green(double r, double k, int filtered, double2& g, double2& g1,
                             double2& g2) {
  const double kr = k * r;
  double skr, ckr;
  sincos(kr, &skr, &ckr);
  const double ir = 1.0 / r, ir2 = ir * ir, ir3 = ir2 * ir;
  if (!filtered) {
    const double2 e = make_double2(ckr, skr);  // e^{ikr}
    g = cscale(e, ir);
    g1 = cscale(cmul(e, make_double2(-1.0, kr)), ir2);                        // (ikr - 1)/r^2
    g2 = cscale(cmul(e, make_double2(2.0 - kr * kr, -2.0 * kr)), ir3);        // (2 - 2ikr - k^2r^2)/r^3
    return;
  }
  const double kf = 3.14159265358979323846;  // pi / d
  const double a = kf - k, b = kf + k;
  double sia, cia, sib, cib;
  sici(a * r, sia, cia);
  sici(b * r, sib, cib);
  double sar, car, sbr, cbr;
  sincos(a * r, &sar, &car);
  sincos(b * r, &sbr, &cbr);
  const double S = sia + sib, Cc = cia - cib;
  const double S1 = (sar + sbr) / r, C1 = (car - cbr) / r;
  const double S2 = (a * car + b * cbr) / r - S1 / r;
  const double C2 = (-a * sar + b * sbr) / r - C1 / r;
  const double ip = 0.31830988618379067154;  // 1/pi
  // h = r g, h', h''
  const double2 h = make_double2(ip * (ckr * S + skr * Cc), skr);
  const double2 h1 = make_double2(ip * (-k * skr * S + ckr * S1 + k * ckr * Cc + skr * C1),
                                  k * ckr);
  const double2 h2 = make_double2(ip * (-k * k * ckr * S - 2.0 * k * skr * S1 + ckr * S2 -
                                        k * k * skr * Cc + 2.0 * k * ckr * C1 + skr * C2),
                                  -k * k * skr);
  g = cscale(h, ir);
  g1 = csub(cscale(h1, ir), cscale(h, ir2));
  g2 = cadd(csub(cscale(h2, ir), cscale(h1, 2.0 * ir2)), cscale(h, 2.0 * ir3));
}

// Tensor at offset (dx, dy, dz) != 0 : out[0..5] = xx, xy, xz, yy, yz, zz
__device__ void green_tensor(double dx, double dy, double dz, double k, int filtered,
                             double2 out[6]) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double r = sqrt(r2);
  const double n[3] = {dx / r, dy / r, dz / r};
  double2 A, B;
  if (!filtered) {
    const double kr = k * r;
    double skr, ckr;
    sincos(kr, &skr, &ckr);
    const double inv3 = 1.0 / (r2 * r);
    const double2 e = make_double2(ckr * inv3, skr * inv3);  // e^{ikr}/r^3
    A = cmul(e, make_double2(kr * kr - 1.0, kr));
    B = cmul(e, make_double2(3.0 - kr * kr, -3.0 * kr));
  } else {
    double2 g, g1, g2;
    scalar_green(r, k, 1, g, g1, g2);
    const double ir = 1.0 / r;
    A = cadd(cscale(g, k * k), cscale(g1, ir));
    B = csub(g2, cscale(g1, ir));
  }
  out[0] = cadd(A, cscale(B, n[0] * n[0]));
  out[1] = cscale(B, n[0] * n[1]);
  out[2] = cscale(B, n[0] * n[2]);
  out[3] = cadd(A, cscale(B, n[1] * n[1]));
  out[4] = cscale(B, n[1] * n[2]);
  out[5] = cadd(A, cscale(B, n[2] * n[2]));
}

// Magnetic field of a dipole P at offset r (Gaussian units): B = h(r) x P with
// h = -i k g'(r) rhat (from B = curl A, A = -i k P g), i.e. for the point
// dipole h = k^2 (e^{ikr}/r)(1 + i/(kr)) rhat; FCD uses the filtered g_F.
// out[0..2] = h_x, h_y, h_z.
__device__ void magnetic_vector(double dx, double dy, double dz, double k, int filtered,
                                double2 out[3]) {
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double2 g, g1, g2;
  scalar_green(r, k, filtered, g, g1, g2);
  const double2 m = make_double2(k * g1.y, -k * g1.x);  // -i k g'
  out[0] = cscale(m, dx / r);
  out[1] = cscale(m, dy / r);
  out[2] = cscale(m, dz / r);
}

// One thread per non-negative offset (dx, dy, dz) in the box; writes the up to
// 8 mirrored grid points with the parity signs.  grid6: [6][Lz][Ly][Lx], zeroed.
__global__ void k_green_fill(int nx, int ny, int nz, int Lx, int Ly, int Lz, double k,
                             int filtered, double2* __restrict__ grid6) {
  const int64_t nb = (int64_t)nx * ny * nz;
  const int64_t M = (int64_t)Lx * Ly * Lz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int dx = (int)(i % nx);
    const int64_t q = i / nx;
    const int dy = (int)(q % ny), dz = (int)(q / ny);
    if (dx == 0 && dy == 0 && dz == 0) continue;
    double2 g[6];
    const bool mag = (filtered & 2) != 0;
    if (mag) {
      magnetic_vector((double)dx, (double)dy, (double)dz, k, filtered & 1, g);
      g[3] = g[4] = g[5] = make_double2(0.0, 0.0);
    } else {
      green_tensor((double)dx, (double)dy, (double)dz, k, filtered & 1, g);
    }
    // parity of each component under the reflection of x, y, z: G xx..zz, or
    // h_x, h_y, h_z (odd in their own axis) for the magnetic vector
    const int pg[6][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 0, 0}, {0, 1, 1}, {0, 0, 0}};
    const int ph[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const int (*par)[3] = mag ? ph : pg;
    for (int mz = 0; mz < 2; ++mz) {
      if (mz && dz == 0) continue;
      const int iz = mz ? Lz - dz : dz;
      for (int my = 0; my < 2; ++my) {
        if (my && dy == 0) continue;
        const int iy = my ? Ly - dy : dy;
        for (int mx = 0; mx < 2; ++mx) {
          if (mx && dx == 0) continue;
          const int ix = mx ? Lx - dx : dx;
          const int64_t o = ((int64_t)iz * Ly + iy) * Lx + ix;
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const int flips = (mx & par[c][0]) + (my & par[c][1]) + (mz & par[c][2]);
            double2 v = g[c];
            if (flips & 1) { v.x = -v.x; v.y = -v.y; }
            grid6[c * M + o] = v;
          }
        }
      }
    }
  }
}

cudaError_t launch_green_fill(int nx, int ny, int nz, int Lx, int Ly, int Lz, double kd,
                              int filtered, double2* grid6, cudaStream_t st) {
  const int64_t M = (int64_t)Lx * Ly * Lz;
  cudaError_t e = cudaMemsetAsync(grid6, 0, sizeof(double2) * 6 * M, st);
  if (e != cudaSuccess) return e;
  const int64_t nb = (int64_t)nx * ny * nz;
  int blocks = (int)((nb + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_green_fill<<<blocks, 256, 0, st>>>(nx, ny, nz, Lx, Ly, Lz, kd, filtered, grid6);
  note_launch();
  return cudaGetLastError();
}

// Generic strided transform (used for the unpruned setup transforms along y and z).
// Lines are columns of a row-major plane: element (p, col) at base + p*row_stride + col.
template <typename T, bool INV>
__global__ void __launch_bounds__(512) k_fft_strided(cplx_t<T>* __restrict__ buf, AxisPlan P, const cplx_t<T>* tw,
                              int64_t ncols, int64_t row_stride, int64_t plane_stride,
                              int tile) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int64_t col0 = (int64_t)blockIdx.x * tile;
  const int ncol = (int)min((int64_t)tile, ncols - col0);
  C* base = buf + (int64_t)blockIdx.y * plane_stride + col0;
  const int L = P.L;
  for (int e = threadIdx.x; e < L * tile; e += blockDim.x) {
    const int p = e / tile, t = e - p * tile;
    s[p * tile + t] = t < ncol ? base[p * row_stride + t] : mk<C>(0, 0);
  }
  __syncthreads();
  fft_smem<C, INV>(s, tile, tile, P, tw);
  for (int e = threadIdx.x; e < L * tile; e += blockDim.x) {
    const int p = e / tile, t = e - p * tile;
    if (t < ncol) base[p * row_stride + t] = s[p * tile + t];
  }
}

static cudaError_t strided_pass(double2* buf, const AxisPlan& P, const double2* tw,
                                int64_t ncols, int64_t row_stride, int64_t plane_stride,
                                int nplanes, cudaStream_t st) {
  int tile = 8;
  while (tile > 1 && (size_t)tile * P.L * sizeof(double2) > 64 * 1024) tile >>= 1;
  int th = ((tile * P.L / 4 + 31) / 32) * 32;
  th = th < 64 ? 64 : (th > 512 ? 512 : th);
  const size_t smem = (size_t)tile * P.L * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_fft_strided<double, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e != cudaSuccess) return e;
  dim3 g((unsigned)((ncols + tile - 1) / tile), nplanes);
  k_fft_strided<double, false><<<g, th, smem, st>>>(buf, P, tw, ncols, row_stride,
                                                     plane_stride, tile);
                                                     note_launch();
  return cudaGetLastError();
}

// Forward unpruned 3-D transform of `count` (a multiple of 3) grids
// [count][Lz][Ly][Lx] into tmp.  `op` describes the full grid as its box
// (nx = Lx, ny = Ly, nz = Lz), so the x pass prunes nothing.
cudaError_t launch_fft3d_full(const OpView<double>& op, const MatvecLaunch& L, int count,
                              double2* grids, double2* tmp, cudaStream_t st) {
  cudaError_t e = launch_x_fwd<double>(op, L, count / 3, grids, tmp, st);
  if (e != cudaSuccess) return e;
  const int64_t Lx = op.Lx, Ly = op.Ly, Lz = op.Lz;
  // y: columns x of each (grid, z) plane
  e = strided_pass(tmp, op.py, op.twy, Lx, Lx, Ly * Lx, (int)(count * Lz), st);
  if (e != cudaSuccess) return e;
  // z: columns (y, x) of each grid
  return strided_pass(tmp, op.pz, op.twz, Ly * Lx, Ly * Lx, Lz * Ly * Lx, count, st);
}

// The forward transforms leave frequency k of each axis at position pos[k].
__global__ void k_green_octant(int Lx, int Ly, int Lz, const int* __restrict__ posx,
                               const int* __restrict__ posy, const int* __restrict__ posz,
                               const double2* __restrict__ full, double2* __restrict__ g64,
                               float2* __restrict__ g32) {
  const int Hx = Lx / 2 + 1, Hy = Ly / 2 + 1, Hz = Lz / 2 + 1;
  const int64_t H = (int64_t)Hx * Hy * Hz;
  const int64_t M = (int64_t)Lx * Ly * Lz;
  const double inv = 1.0 / (double)M;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 6 * H;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / H);
    const int64_t o = i - c * H;
    const int hx = (int)(o % Hx);
    const int64_t q = o / Hx;
    const int hy = (int)(q % Hy), hz = (int)(q / Hy);
    const double2 v = full[c * M + ((int64_t)posz[hz] * Ly + posy[hy]) * Lx + posx[hx]];
    const double2 w = make_double2(v.x * inv, v.y * inv);
    g64[6 * o + c] = w;  // the six components of a point side by side
    if (g32) g32[6 * o + c] = make_float2((float)w.x, (float)w.y);
  }
}

cudaError_t launch_green_octant(int Lx, int Ly, int Lz, const int* posx, const int* posy,
                                const int* posz, const double2* grid6, double2* g64,
                                float2* g32, cudaStream_t st) {
  const int64_t H = (int64_t)(Lx / 2 + 1) * (Ly / 2 + 1) * (Lz / 2 + 1);
  int blocks = (int)((6 * H + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_green_octant<<<blocks, 256, 0, st>>>(Lx, Ly, Lz, posx, posy, posz, grid6, g64, g32);
  note_launch();
  return cudaGetLastError();
}

}  // namespace dda
