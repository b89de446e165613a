// Two more of the guide's Krylov options (Sec. "Choice of Iterative
// Algorithm"), vector and scalar kernels for R right-hand sides in lockstep;
// the drivers are in api.cu.  <a, b> = sum conj(a) b; rt is the shadow vector.
//
// GPBICG -- GPBi-CG (Zhang 1997).  t, u, z, At, q start at zero, beta at 0;
// iteration n:
//   p = r + beta (p - u);  w = At + beta q        (A t_{n-1} + beta A p_{n-1})
//   q = A p;  alpha = <rt, r> / <rt, q>
//   t' = r - alpha q;  y = t - t' - alpha w;  u = t - r + beta u;  t = t'
//   At = A t
//   (zeta, eta) minimise ||t - zeta At - eta y||, i.e. solve
//       [<At, At>  <At, y>] [zeta]   [<At, t>]
//       [<y, At>   <y, y> ] [eta ] = [<y, t> ]
//   (eta = 0 at n = 0, and wherever the 2x2 system is singular)
//   u = zeta q + eta u;  z = zeta r + eta z - alpha u;  x = x + alpha p + z
//   r' = t - eta y - zeta At;  beta = (alpha / zeta) <rt, r'> / <rt, r>
// With eta = 0 throughout this is BiCGSTAB with omega = zeta; so the scalar
// step that closes an iteration (beta, convergence) is BiCGSTAB's, with
// KState.omega = zeta and KState.qa1 = eta.
//
// PETRKP -- conjugate gradients on the normal equations A^H A x = A^H b
// (Petravic & Kuo-Petravic 1979; the guide's PETRKP, the method of the first
// DDA codes), with A^H v = conj(A conj(v)) because A = A^T:
//   init: r = b - A x;  p = A^H r;  gamma = ||p||^2
//   w = A p;  alpha = gamma / ||w||^2;  x = x + alpha p;  r = r - alpha w
//   m = A conj(r);  beta = ||m||^2 / gamma;  gamma = ||m||^2;  p = conj(m) + beta p
// All its scalars are real; KState.rho.x holds gamma.
#include "dda_ops.h"
#include "reduce.cuh"

namespace dda {

namespace {
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C conjc(C a) { return mk<C>(a.x, -a.y); }
}  // namespace

// ---- GPBi-CG ---------------------------------------------------------------------
// p = r + beta (p - u);  w = At + beta q
template <typename T>
__global__ void k_gp_p(int64_t n, const cplx_t<T>* __restrict__ r, cplx_t<T>* __restrict__ p,
                       const cplx_t<T>* __restrict__ u, const cplx_t<T>* __restrict__ at,
                       const cplx_t<T>* __restrict__ q, cplx_t<T>* __restrict__ w,
                       const KState* __restrict__ ks, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].beta}, sc);
  const C beta = sc[0];
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    p[g] = cadd(r[g], cmul(beta, csub(p[g], u[g])));
    w[g] = cadd(at[g], cmul(beta, q[g]));
  }
}

// t' = r - alpha q;  y = t - t' - alpha w;  u = t - r + beta u;  t = t'
template <typename T>
__global__ void k_gp_t(int64_t n, const cplx_t<T>* __restrict__ r,
                       const cplx_t<T>* __restrict__ q, cplx_t<T>* __restrict__ t,
                       const cplx_t<T>* __restrict__ w, cplx_t<T>* __restrict__ u,
                       cplx_t<T>* __restrict__ y, const KState* __restrict__ ks,
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
    const C ri = r[g], to = t[g];
    const C tn = csub(ri, cmul(alpha, q[g]));
    y[g] = csub(csub(to, tn), cmul(alpha, w[g]));
    u[g] = cadd(csub(to, ri), cmul(beta, u[g]));
    t[g] = tn;
  }
}

// partials ([R][nblk][8]): <At, t> (2), <At, At>, <y, y>, <At, y> (2), <y, t> (2)
template <typename T>
__global__ void k_gp_dots(int64_t n, const cplx_t<T>* __restrict__ at,
                          const cplx_t<T>* __restrict__ t, const cplx_t<T>* __restrict__ y,
                          double* partials, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 8> acc;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    const C a = at[g], b = t[g], c = y[g];
    acc.add(0, a.x * b.x + a.y * b.y);
    acc.add(1, a.x * b.y - a.y * b.x);
    acc.add(2, a.x * a.x + a.y * a.y);
    acc.add(3, c.x * c.x + c.y * c.y);
    acc.add(4, a.x * c.x + a.y * c.y);
    acc.add(5, a.x * c.y - a.y * c.x);
    acc.add(6, c.x * b.x + c.y * b.y);
    acc.add(7, c.x * b.y - c.y * b.x);
    acc.step();
  }
  acc.template write<8>(partials);
}

// u = zeta q + eta u;  z = zeta r + eta z - alpha u;  x += alpha p + z;
// r = t - eta y - zeta At;  partials ([R][nblk][4]): <rt, r> (2), ||r||^2, 0
template <typename T>
__global__ void k_gp_x(int64_t n, cplx_t<T>* __restrict__ x, cplx_t<T>* __restrict__ r,
                       const cplx_t<T>* __restrict__ p, const cplx_t<T>* __restrict__ q,
                       cplx_t<T>* __restrict__ u, cplx_t<T>* __restrict__ z,
                       const cplx_t<T>* __restrict__ t, const cplx_t<T>* __restrict__ y,
                       const cplx_t<T>* __restrict__ at, const cplx_t<T>* __restrict__ rt,
                       double* partials, const KState* __restrict__ ks,
                       const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[3];
  block_scalars<C, 3>({ks[rr].alpha, ks[rr].omega, ks[rr].qa1}, sc);
  const C alpha = sc[0], zeta = sc[1], eta = sc[2];
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 4> acc;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    const C un = cadd(cmul(zeta, q[g]), cmul(eta, u[g]));
    u[g] = un;
    const C zn = csub(cadd(cmul(zeta, r[g]), cmul(eta, z[g])), cmul(alpha, un));
    z[g] = zn;
    x[g] = cadd(x[g], cadd(cmul(alpha, p[g]), zn));
    const C rn = csub(csub(t[g], cmul(eta, y[g])), cmul(zeta, at[g]));
    r[g] = rn;
    const C h = rt[g];
    acc.add(0, h.x * rn.x + h.y * rn.y);
    acc.add(1, h.x * rn.y - h.y * rn.x);
    acc.add(2, rn.x * rn.x + rn.y * rn.y);
    acc.step();
  }
  acc.template write<4>(partials);
}

// zeta (-> KState.omega) and eta (-> KState.qa1) from the k_gp_dots partials
__global__ void k_gp_zeta(int nblk, const double* partials, KState* ks, int* active) {
  const int r = blockIdx.x;
  if (!active[r]) return;
  double tot[8];
  sum_partials<8>(partials, nblk, r, tot);
  if (threadIdx.x != 0) return;
  KState& k = ks[r];
  const double2 at = make_double2(tot[0], tot[1]);
  const double aa = tot[2], yy = tot[3];
  const double2 ay = make_double2(tot[4], tot[5]);
  const double2 yt = make_double2(tot[6], tot[7]);
  if (!(aa > 0.0) || !isfinite(aa) || !finite2(at)) {
    // At = 0 means t = 0: the next residual is zero and the scalar step that
    // follows reports convergence (or a breakdown for non-finite sums)
    k.omega = make_double2(0.0, 0.0);
    k.qa1 = make_double2(0.0, 0.0);
    return;
  }
  const double det = aa * yy - (ay.x * ay.x + ay.y * ay.y);
  if (k.iters == 0 || !(det > 1e-14 * aa * yy) || !isfinite(det) || !finite2(ay) ||
      !finite2(yt)) {
    k.omega = make_double2(at.x / aa, at.y / aa);
    k.qa1 = make_double2(0.0, 0.0);
    return;
  }
  // zeta = (yy <At,t> - <At,y> <y,t>) / det;  eta = (aa <y,t> - conj(<At,y>) <At,t>) / det
  const double2 a1 = cmuld(ay, yt), a2 = cmuld(make_double2(ay.x, -ay.y), at);
  k.omega = make_double2((yy * at.x - a1.x) / det, (yy * at.y - a1.y) / det);
  k.qa1 = make_double2((aa * yt.x - a2.x) / det, (aa * yt.y - a2.y) / det);
}

// ---- conjugate gradients on the normal equations ------------------------------------
// c = conj(r)
template <typename T>
__global__ void k_cg_conj(int64_t n, const cplx_t<T>* __restrict__ r, cplx_t<T>* __restrict__ c,
                          const int* __restrict__ active) {
  const int rr = blockIdx.y;
  if (active && !active[rr]) return;
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) c[off + i] = conjc(r[off + i]);
}

// partials ([R][nblk][1]): ||v||^2
template <typename T>
__global__ void k_cg_norm(int64_t n, const cplx_t<T>* __restrict__ v, double* partials,
                          const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 1> acc;
  GRID_LOOP(i, n) {
    const C a = v[off + i];
    acc.add(0, a.x * a.x + a.y * a.y);
    acc.step();
  }
  acc.template write<1>(partials);
}

// x += alpha p;  r -= alpha w;  c = conj(r);  partials: ||r||^2
template <typename T>
__global__ void k_cg_xr(int64_t n, cplx_t<T>* __restrict__ x, cplx_t<T>* __restrict__ r,
                        const cplx_t<T>* __restrict__ p, const cplx_t<T>* __restrict__ w,
                        cplx_t<T>* __restrict__ c, double* partials,
                        const KState* __restrict__ ks, const int* __restrict__ active) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].alpha}, sc);
  const T alpha = sc[0].x;  // real
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 1> acc;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    const C pv = p[g], wv = w[g], xv = x[g], rv = r[g];
    x[g] = mk<C>(xv.x + alpha * pv.x, xv.y + alpha * pv.y);
    const C rn = mk<C>(rv.x - alpha * wv.x, rv.y - alpha * wv.y);
    r[g] = rn;
    c[g] = conjc(rn);
    acc.add(0, rn.x * rn.x + rn.y * rn.y);
    acc.step();
  }
  acc.template write<1>(partials);
}

// p = conj(m) + beta p  (beta real; with first = 1: p = conj(m))
template <typename T>
__global__ void k_cg_p(int64_t n, const cplx_t<T>* __restrict__ m, cplx_t<T>* __restrict__ p,
                       const KState* __restrict__ ks, const int* __restrict__ active,
                       int first) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].beta}, sc);
  const T beta = first ? (T)0 : sc[0].x;
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const int64_t g = off + i;
    const C mv = m[g];
    if (first) {
      p[g] = conjc(mv);
    } else {
      const C pv = p[g];
      p[g] = mk<C>(mv.x + beta * pv.x, -mv.y + beta * pv.y);
    }
  }
}

// Scalar steps of the normal-equation CG, one block per RHS; partials hold one
// sum per block.
//  phase 0: gamma = ||A^H r||^2 (set-up)
//  phase 1: alpha = gamma / ||A p||^2
//  phase 2: ||r||^2: convergence, iterations += 1
//  phase 3: beta = ||A^H r||^2 / gamma, gamma = ||A^H r||^2
__global__ void k_cg_scalar(int phase, int nblk, const double* partials, KState* ks,
                            int* active) {
  const int r = blockIdx.x;
  if (!active[r]) return;
  double tot[1];
  sum_partials<1>(partials, nblk, r, tot);
  if (threadIdx.x != 0) return;
  KState& k = ks[r];
  const double v = tot[0];
  auto breakdown = [&]() { k.status = KS_BREAKDOWN; active[r] = 0; };
  if (!isfinite(v)) { breakdown(); return; }
  if (phase == 0) {
    if (!(v > 0.0)) { breakdown(); return; }
    k.rho = make_double2(v, 0.0);
    k.beta = make_double2(0.0, 0.0);
  } else if (phase == 1) {
    if (!(v > 0.0)) { breakdown(); return; }
    k.alpha = make_double2(k.rho.x / v, 0.0);
  } else if (phase == 2) {
    k.rnorm2 = v;
    k.iters += 1;
    if (k.rnorm2 <= k.tol2 * k.bnorm2) { k.status = KS_CONV; active[r] = 0; return; }
    if (k.iters >= k.max_iter) { k.status = KS_NOCONV; active[r] = 0; return; }
  } else {
    if (!(v > 0.0)) { breakdown(); return; }
    k.beta = make_double2(v / k.rho.x, 0.0);
    k.rho = make_double2(v, 0.0);
  }
}

// ---- launchers -------------------------------------------------------------------
template <typename T>
cudaError_t launch_gp_vec(int which, int64_t n, int R, const GpVecs<T>& v, double* partials,
                          const KState* ks, const int* active, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  switch (which) {
    case 0: k_gp_p<T><<<g, kThreads, 0, st>>>(n, v.r, v.p, v.u, v.at, v.q, v.w, ks, active); break;
    case 1: k_gp_t<T><<<g, kThreads, 0, st>>>(n, v.r, v.q, v.t, v.w, v.u, v.y, ks, active); break;
    case 2: k_gp_dots<T><<<g, kThreads, 0, st>>>(n, v.at, v.t, v.y, partials, active); break;
    default:
      k_gp_x<T><<<g, kThreads, 0, st>>>(n, v.x, v.r, v.p, v.q, v.u, v.z, v.t, v.y, v.at, v.rt,
                                         partials, ks, active);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gp_zeta(int R, int nblk, const double* partials, KState* ks, int* active,
                           cudaStream_t st) {
  k_gp_zeta<<<R, kThreads, 0, st>>>(nblk, partials, ks, active);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_vec(int which, int64_t n, int R, cplx_t<T>* x, cplx_t<T>* r,
                          cplx_t<T>* p, const cplx_t<T>* w, cplx_t<T>* c, const cplx_t<T>* m,
                          double* partials, const KState* ks, const int* active,
                          cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  switch (which) {
    case 0: k_cg_conj<T><<<g, kThreads, 0, st>>>(n, r, c, active); break;
    case 1: k_cg_norm<T><<<g, kThreads, 0, st>>>(n, w, partials, active); break;
    case 2: k_cg_xr<T><<<g, kThreads, 0, st>>>(n, x, r, p, w, c, partials, ks, active); break;
    case 3: k_cg_norm<T><<<g, kThreads, 0, st>>>(n, m, partials, active); break;
    case 4: k_cg_p<T><<<g, kThreads, 0, st>>>(n, m, p, ks, active, 1); break;
    default: k_cg_p<T><<<g, kThreads, 0, st>>>(n, m, p, ks, active, 0);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cg_scalar(int phase, int R, int nblk, const double* partials, KState* ks,
                             int* active, cudaStream_t st) {
  k_cg_scalar<<<R, kThreads, 0, st>>>(phase, nblk, partials, ks, active);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_gp_vec<float>(int, int64_t, int, const GpVecs<float>&, double*,
                                          const KState*, const int*, cudaStream_t);
template cudaError_t launch_gp_vec<double>(int, int64_t, int, const GpVecs<double>&, double*,
                                           const KState*, const int*, cudaStream_t);
template cudaError_t launch_cg_vec<float>(int, int64_t, int, float2*, float2*, float2*,
                                          const float2*, float2*, const float2*, double*,
                                          const KState*, const int*, cudaStream_t);
template cudaError_t launch_cg_vec<double>(int, int64_t, int, double2*, double2*, double2*,
                                           const double2*, double2*, const double2*, double*,
                                           const KState*, const int*, cudaStream_t);

}  // namespace dda
