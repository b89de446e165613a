// Cross sections and scattering amplitudes from the solved dipole moments.
//
//  C_ext = 4 pi k sum_j Im(E_inc,j^* . P_j)
//  C_abs = 4 pi k sum_j sum_a |P_ja|^2 [-Im(1/alpha_ja) - (2/3) k^3]  (a: lattice
//          axis; alpha's diagonal, equal on the axes except for GKDLDR)
//  (Sec. "What Does It Calculate?": Q = C / (pi a_eff^2), Q_ext = Q_sca + Q_abs)
//  F(n) = sum_j P_j exp(-i k n . r_j), f_ml = k^3 e_m . F  (eq. f_ml_def)
//
// On the lattice exp(-i k n.r_j) = ex(ix) ey(iy) ez(iz), so the phases come
// from three short per-axis tables and no transcendental is evaluated per site.
// All sums are FP64, two-stage and deterministic.
#include <algorithm>

#include "dda_ops.h"
#include "reduce.cuh"

namespace dda {

__global__ void k_cross_sections(int nx, int ny, int nz, const uint8_t* __restrict__ comp,
                                 RhsTables tb, const double2* __restrict__ P,
                                 const double* __restrict__ wabs, int ncomp1,
                                 double* partials) {
  const int r = blockIdx.y;
  const int64_t nbox = (int64_t)nx * ny * nz;
  const double2 e0 = tb.pol[r * 3 + 0], e1 = tb.pol[r * 3 + 1], e2 = tb.pol[r * 3 + 2];
  double acc[2] = {0.0, 0.0};
  GRID_LOOP(i, nbox) {
    const int cm = comp[i];
    if (cm) {
      const int ix = (int)(i % nx);
      const int64_t q = i / nx;
      const int iy = (int)(q % ny), iz = (int)(q / ny);
      const double2 ph = cmul(cmul(tb.phx[(int64_t)r * nx + ix], tb.phy[(int64_t)r * ny + iy]),
                              tb.phz[(int64_t)r * nz + iz]);
      const double2 p0 = P[((int64_t)r * 3 + 0) * nbox + i];
      const double2 p1 = P[((int64_t)r * 3 + 1) * nbox + i];
      const double2 p2 = P[((int64_t)r * 3 + 2) * nbox + i];
      // E^* . P = conj(ph) * (conj(e) . P)
      double2 ep = cadd(cadd(cmulc(e0, p0), cmulc(e1, p1)), cmulc(e2, p2));
      ep = cmulc(ph, ep);
      acc[0] += ep.y;
      const double* wa = wabs + ((int64_t)r * ncomp1 + cm) * 3;
      acc[1] += (p0.x * p0.x + p0.y * p0.y) * wa[0] + (p1.x * p1.x + p1.y * p1.y) * wa[1] +
                (p2.x * p2.x + p2.y * p2.y) * wa[2];
    }
  }
  write_partials<2>(acc, partials);
}

cudaError_t launch_cross_sections(int nx, int ny, int nz, const uint8_t* comp, RhsTables tb,
                                  int R, const double2* P, const double* wabs, int ncomp1,
                                  double* partials, int nblk, cudaStream_t st) {
  dim3 g(nblk, R);
  k_cross_sections<<<g, kThreads, 0, st>>>(nx, ny, nz, comp, tb, P, wabs, ncomp1, partials);
  note_launch();
  return cudaGetLastError();
}

// grid: (nblk, R, D); partials [(d*R + r)*nblk + blk][6]
__global__ void k_farfield(int nx, int ny, int nz, const uint8_t* __restrict__ comp,
                           const double2* __restrict__ P, const double2* __restrict__ fphx,
                           const double2* __restrict__ fphy, const double2* __restrict__ fphz,
                           double* partials, int d0) {
  const int r = blockIdx.y, d = d0 + (int)blockIdx.z, R = gridDim.y;
  const int64_t nbox = (int64_t)nx * ny * nz;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  GRID_LOOP(i, nbox) {
    if (comp[i]) {
      const int ix = (int)(i % nx);
      const int64_t q = i / nx;
      const int iy = (int)(q % ny), iz = (int)(q / ny);
      const double2 ph = cmul(cmul(fphx[(int64_t)d * nx + ix], fphy[(int64_t)d * ny + iy]),
                              fphz[(int64_t)d * nz + iz]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double2 t = cmul(P[((int64_t)r * 3 + c) * nbox + i], ph);
        acc[2 * c] += t.x;
        acc[2 * c + 1] += t.y;
      }
    }
  }
  double tot[6];
  block_sum<6>(acc, tot);
  if (threadIdx.x == 0) {
    double* o = partials + (((int64_t)d * R + r) * gridDim.x + blockIdx.x) * 6;
#pragma unroll
    for (int i = 0; i < 6; ++i) o[i] = tot[i];
  }
}

cudaError_t launch_farfield(int nx, int ny, int nz, const uint8_t* comp, int R, int D,
                            const double2* P, const double2* fphx, const double2* fphy,
                            const double2* fphz, double* partials, int nblk,
                            cudaStream_t st) {
  // grid.z is limited to 65535 directions per launch
  for (int d0 = 0; d0 < D; d0 += 65535) {
    dim3 g(nblk, R, std::min(65535, D - d0));
    k_farfield<<<g, kThreads, 0, st>>>(nx, ny, nz, comp, P, fphx, fphy, fphz, partials, d0);
    note_launch();
  }
  return cudaGetLastError();
}

// ---- near field (the guide's NRFLD option, Sec. "Near-Field Calculations") ---------
// E_sca is the field of all dipoles at each box site without the site's own
// dipole; the total microscopic field is E_inc + E_sca, and inside the target
// the macroscopic field is E_macro = 3 / (eps + 2) E_micro (eq. macro_vs_micro),
// in vacuum the two are equal.
// The incident magnetic field of the plane wave is B_inc = khat x E_inc.
__global__ void k_nearfield_post(int nx, int ny, int nz, const uint8_t* __restrict__ comp,
                                 RhsTables tb, const double2* __restrict__ esca,
                                 const double2* __restrict__ fac, const double* __restrict__ khat,
                                 double2* __restrict__ einc, double2* __restrict__ emacro,
                                 double2* __restrict__ binc) {
  const int r = blockIdx.y;
  const int64_t nbox = (int64_t)nx * ny * nz;
  GRID_LOOP(i, nbox) {
    const int ix = (int)(i % nx);
    const int64_t q = i / nx;
    const int iy = (int)(q % ny), iz = (int)(q / ny);
    const double2 ph = cmul(cmul(tb.phx[(int64_t)r * nx + ix], tb.phy[(int64_t)r * ny + iy]),
                            tb.phz[(int64_t)r * nz + iz]);
    const double2 f = fac[comp[i]];
    double2 ei[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t o = ((int64_t)r * 3 + c) * nbox + i;
      ei[c] = cmul(tb.pol[r * 3 + c], ph);
      if (einc) einc[o] = ei[c];
      if (emacro) {
        const double2 es = esca[o];
        emacro[o] = cmul(f, make_double2(ei[c].x + es.x, ei[c].y + es.y));
      }
    }
    if (binc) {
      const double* k = khat + 3 * r;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        binc[((int64_t)r * 3 + c) * nbox + i] =
            csub(cscale(ei[c2], k[c1]), cscale(ei[c1], k[c2]));
      }
    }
  }
}

cudaError_t launch_nearfield_post(int nx, int ny, int nz, const uint8_t* comp, RhsTables tb,
                                  int R, const double2* esca, const double2* fac,
                                  const double* khat, double2* einc, double2* emacro,
                                  double2* binc, cudaStream_t st) {
  const int64_t nbox = (int64_t)nx * ny * nz;
  dim3 g(reduce_blocks(nbox), R);
  k_nearfield_post<<<g, kThreads, 0, st>>>(nx, ny, nz, comp, tb, esca, fac, khat, einc,
                                           emacro, binc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace dda
