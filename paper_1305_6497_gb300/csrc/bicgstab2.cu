// BiCGstab(l) with l = 2 (Sleijpen & van der Vorst 1993; Sleijpen, van der
// Vorst & Fokkema 1994) -- the guide's PBCGS2 option, its recommended method
// (Sec. "Choice of Iterative Algorithm").  Vector and scalar kernels for R
// right-hand sides in lockstep; the driver is in api.cu.
//
// One cycle (four matvecs) with residuals r0, r1, r2, directions u0, u1, u2 and
// shadow vector rt:
//   rho0 <- -omega rho0
//   j = 0:  rho1 = <rt, r0>, beta = alpha rho1 / rho0, rho0 = rho1
//           u0 = r0 - beta u0;  u1 = A u0;  alpha = rho0 / <rt, u1>
//           r0 = r0 - alpha u1; r1 = A r0;  x = x + alpha u0 (deferred)
//   j = 1:  rho1 = <rt, r1>, beta = alpha rho1 / rho0, rho0 = rho1
//           u0 = r0 - beta u0, u1 = r1 - beta u1; u2 = A u1; alpha = rho0/<rt, u2>
//           r0 = r0 - alpha u1, r1 = r1 - alpha u2; r2 = A r1; x = x + alpha u0
//   minimal residual over span(r1, r2): (g1, g2) solves the 2x2 normal
//           equations [<r_i, r_j>] g = [<r_i, r0>], i, j = 1, 2; omega = g2
//           u0 = u0 - g1 u1 - g2 u2, x = x + g1 r0 + g2 r1, r0 = r0 - g1 r1 - g2 r2
// (<a, b> = sum conj(a) b).  A cycle counts as two iterations (four matvecs,
// as two BiCGSTAB iterations).
#include "dda_ops.h"
#include "reduce.cuh"

namespace dda {

namespace {
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C d2c(double2 a) { return mk<C>(a.x, a.y); }
}  // namespace

// u0 = r0 - beta u0
template <typename T>
__global__ void k_bs2_a(int64_t n, const cplx_t<T>* __restrict__ r0, cplx_t<T>* __restrict__ u0,
                        const KState* __restrict__ ks, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].beta}, sc);
  const C beta = sc[0];
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) u0[off + i] = csub(r0[off + i], cmul(beta, u0[off + i]));
}

// r0 = r0 - alpha u1
template <typename T>
__global__ void k_bs2_b(int64_t n, cplx_t<T>* __restrict__ r0, const cplx_t<T>* __restrict__ u1,
                        const KState* __restrict__ ks, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].alpha}, sc);
  const C alpha = sc[0];
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) r0[off + i] = csub(r0[off + i], cmul(alpha, u1[off + i]));
}

// x += alpha u0 (alpha of j = 0); u0 = r0 - beta u0; u1 = r1 - beta u1
template <typename T>
__global__ void k_bs2_c(int64_t n, cplx_t<T>* __restrict__ x, const cplx_t<T>* __restrict__ r0,
                        const cplx_t<T>* __restrict__ r1, cplx_t<T>* __restrict__ u0,
                        cplx_t<T>* __restrict__ u1, const KState* __restrict__ ks,
                        const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[2];
  block_scalars<C, 2>({ks[rr].alpha, ks[rr].beta}, sc);
  const C alpha = sc[0], beta = sc[1];
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    const C a0 = u0[g];
    x[g] = cadd(x[g], cmul(alpha, a0));
    u0[g] = csub(r0[g], cmul(beta, a0));
    u1[g] = csub(r1[g], cmul(beta, u1[g]));
  }
}

// r0 -= alpha u1; r1 -= alpha u2; x += alpha u0
template <typename T>
__global__ void k_bs2_d(int64_t n, cplx_t<T>* __restrict__ x, cplx_t<T>* __restrict__ r0,
                        cplx_t<T>* __restrict__ r1, const cplx_t<T>* __restrict__ u0,
                        const cplx_t<T>* __restrict__ u1, const cplx_t<T>* __restrict__ u2,
                        const KState* __restrict__ ks, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].alpha}, sc);
  const C alpha = sc[0];
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    r0[g] = csub(r0[g], cmul(alpha, u1[g]));
    r1[g] = csub(r1[g], cmul(alpha, u2[g]));
    x[g] = cadd(x[g], cmul(alpha, u0[g]));
  }
}

// Gram entries: ||r1||^2, ||r2||^2, <r1, r2>, <r1, r0>, <r2, r0>  ([R][nblk][8])
template <typename T>
__global__ void k_bs2_gram(int64_t n, const cplx_t<T>* __restrict__ r0,
                           const cplx_t<T>* __restrict__ r1, const cplx_t<T>* __restrict__ r2,
                           double* partials, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 8> acc;
  GRID_LOOP(i, n) {
    const C a = r0[off + i], b = r1[off + i], c = r2[off + i];
    acc.add(0, b.x * b.x + b.y * b.y);
    acc.add(1, c.x * c.x + c.y * c.y);
    acc.add(2, b.x * c.x + b.y * c.y);   // conj(r1) r2
    acc.add(3, b.x * c.y - b.y * c.x);
    acc.add(4, b.x * a.x + b.y * a.y);   // conj(r1) r0
    acc.add(5, b.x * a.y - b.y * a.x);
    acc.add(6, c.x * a.x + c.y * a.y);   // conj(r2) r0
    acc.add(7, c.x * a.y - c.y * a.x);
    acc.step();
  }
  acc.template write<8>(partials);
}

// minimal-residual update: u0 -= g1 u1 + g2 u2; x += g1 r0 + g2 r1;
// r0 -= g1 r1 + g2 r2; partials <rt, r0>, ||r0||^2  ([R][nblk][4])
template <typename T>
__global__ void k_bs2_e(int64_t n, cplx_t<T>* __restrict__ x, cplx_t<T>* __restrict__ r0,
                        const cplx_t<T>* __restrict__ r1, const cplx_t<T>* __restrict__ r2,
                        cplx_t<T>* __restrict__ u0, const cplx_t<T>* __restrict__ u1,
                        const cplx_t<T>* __restrict__ u2, const cplx_t<T>* __restrict__ rt,
                        double* partials, const KState* __restrict__ ks,
                        const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[2];
  block_scalars<C, 2>({ks[rr].qa1, ks[rr].qa2}, sc);
  const C g1 = sc[0], g2 = sc[1];
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 4> acc;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    const C a1 = r1[g];
    u0[g] = csub(u0[g], cadd(cmul(g1, u1[g]), cmul(g2, u2[g])));
    const C a0 = r0[g];
    x[g] = cadd(x[g], cadd(cmul(g1, a0), cmul(g2, a1)));
    const C rn = csub(a0, cadd(cmul(g1, a1), cmul(g2, r2[g])));
    r0[g] = rn;
    const C h = rt[g];
    acc.add(0, h.x * rn.x + h.y * rn.y);
    acc.add(1, h.x * rn.y - h.y * rn.x);
    acc.add(2, rn.x * rn.x + rn.y * rn.y);
    acc.step();
  }
  acc.template write<4>(partials);
}

// Scalar steps, one block per RHS.  KState use: rho = rho0, rho_old = the
// pending rho1 = <rt, r0> of the next cycle, qa1, qa2 = g1, g2.
//  phase 6: after the shared BiCGSTAB set-up (rho = ||r||^2 = <rt, r0>):
//           rho1 pending = rho, rho0 = 1, omega = 1
//  phase 0: cycle start: rho0 = -omega rho0; beta = alpha rho1 / rho0; rho0 = rho1
//  phase 2: rho1 = <rt, r1> (matvec partials, 2 values); beta, rho0 = rho1
//  phase 4: 2x2 minimal residual from the Gram partials (8 values)
//  phase 5: <rt, r0>, ||r0||^2 (4 values): convergence, iterations += 2
__global__ void k_bs2_scalar(int phase, int nblk, const double* partials, KState* ks,
                             int* active) {
  const int r = blockIdx.x;
  if (!active[r]) return;
  double tot[8];
  if (phase == 2) {
    double t2[2];
    sum_partials<2>(partials, nblk, r, t2);
    tot[0] = t2[0]; tot[1] = t2[1];
  } else if (phase == 4) {
    sum_partials<8>(partials, nblk, r, tot);
  } else if (phase == 5) {
    double t4[4];
    sum_partials<4>(partials, nblk, r, t4);
    for (int i = 0; i < 4; ++i) tot[i] = t4[i];
  }
  if (threadIdx.x != 0) return;
  KState& k = ks[r];
  auto breakdown = [&]() { k.status = KS_BREAKDOWN; active[r] = 0; };
  if (phase == 6) {
    k.rho_old = k.rho;
    k.rho = make_double2(1.0, 0.0);
    k.alpha = make_double2(0.0, 0.0);
    k.omega = make_double2(1.0, 0.0);
    k.beta = make_double2(0.0, 0.0);
    k.qa1 = k.qa2 = make_double2(0.0, 0.0);
    return;
  }
  if (phase == 0 || phase == 2) {
    double2 rho0 = k.rho;
    if (phase == 0) {
      rho0 = cmuld(make_double2(-k.omega.x, -k.omega.y), rho0);
    }
    const double2 rho1 = phase == 0 ? k.rho_old : make_double2(tot[0], tot[1]);
    if (!finite2(rho1) || (rho0.x == 0.0 && rho0.y == 0.0)) { breakdown(); return; }
    k.beta = cmuld(k.alpha, cdiv(rho1, rho0));
    k.rho = rho1;
    return;
  }
  if (phase == 4) {
    const double z11 = tot[0], z22 = tot[1];
    const double2 z12 = make_double2(tot[2], tot[3]);      // <r1, r2>
    const double2 b1 = make_double2(tot[4], tot[5]);       // <r1, r0>
    const double2 b2 = make_double2(tot[6], tot[7]);       // <r2, r0>
    // [[z11, z12], [conj z12, z22]] g = b
    const double det = z11 * z22 - (z12.x * z12.x + z12.y * z12.y);
    if (!(det > 1e-14 * z11 * z22) || !isfinite(det)) { breakdown(); return; }
    const double2 t1 = cmuld(z12, b2), t2 = cmuld(make_double2(z12.x, -z12.y), b1);
    k.qa1 = make_double2((z22 * b1.x - t1.x) / det, (z22 * b1.y - t1.y) / det);
    k.qa2 = make_double2((z11 * b2.x - t2.x) / det, (z11 * b2.y - t2.y) / det);
    k.omega = k.qa2;
    return;
  }
  // phase 5
  const double2 rho1 = make_double2(tot[0], tot[1]);
  k.rnorm2 = tot[2];
  k.iters += 2;
  if (k.rnorm2 <= k.tol2 * k.bnorm2) { k.status = KS_CONV; active[r] = 0; return; }
  if (!isfinite(k.rnorm2) || !finite2(rho1) || (rho1.x == 0.0 && rho1.y == 0.0) ||
      (k.omega.x == 0.0 && k.omega.y == 0.0)) {
    breakdown();
    return;
  }
  if (k.iters >= k.max_iter) { k.status = KS_NOCONV; active[r] = 0; return; }
  k.rho_old = rho1;
}

// ---- launchers -------------------------------------------------------------------
template <typename T>
cudaError_t launch_bs2_vec(int which, int64_t n, int R, cplx_t<T>* x, cplx_t<T>* r0,
                           cplx_t<T>* r1, cplx_t<T>* r2, cplx_t<T>* u0, cplx_t<T>* u1,
                           cplx_t<T>* u2, const cplx_t<T>* rt, double* partials,
                           const KState* ks, const int* active, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  switch (which) {
    case 0: k_bs2_a<T><<<g, kThreads, 0, st>>>(n, r0, u0, ks, active); break;
    case 1: k_bs2_b<T><<<g, kThreads, 0, st>>>(n, r0, u1, ks, active); break;
    case 2: k_bs2_c<T><<<g, kThreads, 0, st>>>(n, x, r0, r1, u0, u1, ks, active); break;
    case 3: k_bs2_d<T><<<g, kThreads, 0, st>>>(n, x, r0, r1, u0, u1, u2, ks, active); break;
    case 4: k_bs2_gram<T><<<g, kThreads, 0, st>>>(n, r0, r1, r2, partials, active); break;
    default:
      k_bs2_e<T><<<g, kThreads, 0, st>>>(n, x, r0, r1, r2, u0, u1, u2, rt, partials, ks,
                                          active);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bs2_scalar(int phase, int R, int nblk, const double* partials, KState* ks,
                              int* active, cudaStream_t st) {
  k_bs2_scalar<<<R, kThreads, 0, st>>>(phase, nblk, partials, ks, active);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_bs2_vec<float>(int, int64_t, int, float2*, float2*, float2*, float2*,
                                           float2*, float2*, float2*, const float2*, double*,
                                           const KState*, const int*, cudaStream_t);
template cudaError_t launch_bs2_vec<double>(int, int64_t, int, double2*, double2*, double2*,
                                            double2*, double2*, double2*, double2*,
                                            const double2*, double*, const KState*, const int*,
                                            cudaStream_t);

}  // namespace dda
