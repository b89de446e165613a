// The Krylov scalar steps (internal), shared by the one-block scalar kernels
// and by the vector passes that finish them in their last block.  BiCGSTAB:
//   alpha = rho / <rhat, v>            (sums: <rhat, v>)
//   omega = <t, s> / <t, t>            (sums: <t, s>, <t, t>)
//   rho' = <rhat, r>, ||r||^2: convergence test, then
//   beta = (rho' / rho) (alpha / omega) (sums: <rhat, r>, ||r||^2)
// QMR (complex symmetric): see krylov.cu.  All in FP64 on the per-RHS state.
#pragma once

#include "dda_ops.h"
#include "reduce.cuh"

namespace dda {

__device__ __forceinline__ bool ks_finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }
// a / b with one FP64 reciprocal (divisions are long dependency chains on
// this part's FP64 pipe, and these steps sit on the solve's critical path)
__device__ __forceinline__ double2 ks_cdiv(double2 a, double2 b) {
  const double inv = 1.0 / (b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ double2 ks_cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// tot[0..1] = <rhat, v>
__device__ inline void step_alpha(const double* tot, KState& k, int* active_r) {
  const double2 rv = make_double2(tot[0], tot[1]);
  if (!(rv.x != 0.0 || rv.y != 0.0) || !ks_finite2(rv)) {
    k.status = KS_BREAKDOWN;
    *active_r = 0;
    return;
  }
  k.alpha = ks_cdiv(k.rho, rv);
}

// tot[0..1] = <t, s>, tot[2] = <t, t>
__device__ inline void step_omega(const double* tot, KState& k) {
  const double tt = tot[2];
  if (tt > 0.0 && isfinite(tt)) {
    const double inv = 1.0 / tt;
    k.omega = make_double2(tot[0] * inv, tot[1] * inv);
  }
  else {
    k.omega = make_double2(0.0, 0.0);
  }
}

// tot[0..1] = <rhat, r>, tot[2] = ||r||^2
__device__ inline void step_rho(const double* tot, KState& k, int* active_r) {
  const double2 rho_new = make_double2(tot[0], tot[1]);
  k.rnorm2 = tot[2];
  k.iters += 1;
  if (k.rnorm2 <= k.tol2 * k.bnorm2) {
    k.status = KS_CONV; *active_r = 0; return;
  }
  if (!isfinite(k.rnorm2) || !ks_finite2(rho_new) || (rho_new.x == 0.0 && rho_new.y == 0.0) ||
      (k.omega.x == 0.0 && k.omega.y == 0.0)) {
    k.status = KS_BREAKDOWN; *active_r = 0; return;
  }
  if (k.iters >= k.max_iter) {
    k.status = KS_NOCONV; *active_r = 0; return;
  }
  // beta = (rho' / rho)(alpha / omega) as one quotient
  k.beta = ks_cdiv(ks_cmul(rho_new, k.alpha), ks_cmul(k.rho, k.omega));
  k.rho_old = k.rho;
  k.rho = rho_new;
}

// QMR: tot[0..1] = sigma = q^T A q;  alpha = rho / sigma
__device__ inline void step_qmr_sigma(const double* tot, KState& k, int* active_r) {
  const double2 sigma = make_double2(tot[0], tot[1]);
  if (!(sigma.x != 0.0 || sigma.y != 0.0) || !ks_finite2(sigma)) {
    // this iteration's first pass already applied the pending update
    k.qa1 = make_double2(0.0, 0.0);
    k.qa2 = make_double2(0.0, 0.0);
    k.status = KS_BREAKDOWN;
    *active_r = 0;
    return;
  }
  k.alpha = ks_cdiv(k.rho, sigma);
}

// QMR: tot[0] = ||r||^2, tot[1..2] = r^T r.  Quasi-residual rotation, the
// pending d/x coefficients, the convergence bound tau^2 (k + 1) and beta.
__device__ inline void step_qmr(const double* tot, KState& k, int* active_r) {
  const double rn2 = tot[0];
  const double2 rho_new = make_double2(tot[1], tot[2]);
  const double th = sqrt(rn2) / k.tau;
  const double c2 = 1.0 / (1.0 + th * th);
  const double tau = k.tau * th * sqrt(c2);
  k.qa1 = make_double2(c2 * k.theta * k.theta, 0.0);
  k.qa2 = make_double2(c2 * k.alpha.x, c2 * k.alpha.y);
  k.theta = th;
  k.tau = tau;
  k.rnorm2 = rn2;
  k.iters += 1;
  if (!isfinite(rn2) || !isfinite(tau)) {
    k.qa1 = make_double2(0.0, 0.0);
    k.qa2 = make_double2(0.0, 0.0);
    k.status = KS_BREAKDOWN; *active_r = 0; return;
  }
  if (tau * tau * (k.iters + 1) <= k.tol2 * k.bnorm2) {
    k.status = KS_CONV; *active_r = 0; return;
  }
  if (!ks_finite2(rho_new) || hypot(rho_new.x, rho_new.y) <= k.rho_floor * rn2) {
    k.status = KS_BREAKDOWN; *active_r = 0; return;
  }
  if (k.iters >= k.max_iter) {
    k.status = KS_NOCONV; *active_r = 0; return;
  }
  k.beta = ks_cdiv(rho_new, k.rho);
  k.rho_old = k.rho;
  k.rho = rho_new;
}

// Called by every thread of every block of a row after the block's NV partials
// are written (by thread 0).  Two levels of tickets (see FoldArgs): the last
// block of each group sums the group's partials in block order, the last group
// sums the group sums in group order (FP64) and runs the scalar step; each
// finisher re-arms its counter.  The result does not depend on which blocks
// finish last.
template <int NV>
__device__ void fold_scalar_step(const double* partials, const FoldArgs& f) {
  __shared__ int last;
  const int r = blockIdx.y;
  const int nb = gridDim.x;
  // one group (the plain last-block scheme) while the last block's sum over all
  // partials stays short; groups of >= 64 blocks beyond that
  const int G = nb <= kFoldSingle ? nb : max(64, (nb + kFoldGroups - 1) / kFoldGroups);
  const int ng = (nb + G - 1) / G;
  const int g = blockIdx.x / G;
  const int gsz = min(G, nb - g * G);
  unsigned* cnt = f.counter + (int64_t)r * (1 + kFoldGroups);
  double* gs = f.gsum + (int64_t)r * kFoldGroups * 4;
  if (threadIdx.x == 0) {
    // thread 0 wrote the block's partials: make them visible before its ticket
    // (the other threads wrote nothing the finisher reads, and a fence in
    // every thread would hold each block until all of its stores drained)
    __threadfence();
    const unsigned ticket = atomicAdd(&cnt[1 + g], 1u);
    last = ticket == (unsigned)gsz - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[NV], tot[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  const double* p = partials + ((int64_t)r * nb + (int64_t)g * G) * NV;
  for (int b = threadIdx.x; b < gsz; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += __ldcg(p + (int64_t)b * NV + i);
  }
  block_sum<NV>(acc, tot);
  if (ng > 1) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) gs[4 * g + i] = tot[i];
      cnt[1 + g] = 0;
      __threadfence();
      const unsigned ticket = atomicAdd(&cnt[0], 1u);
      last = ticket == (unsigned)ng - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int q = threadIdx.x; q < ng; q += blockDim.x) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += __ldcg(gs + 4 * q + i);
    }
    block_sum<NV>(acc, tot);
  }
  if (threadIdx.x == 0) {
    if (ng == 1) cnt[1] = 0;
    KState& k = f.ks[r];
    int* act = f.active + r;
    if (f.step == FOLD_ALPHA) step_alpha(tot, k, act);
    else if (f.step == FOLD_OMEGA) step_omega(tot, k);
    else if (f.step == FOLD_RHO) step_rho(tot, k, act);
    else if (f.step == FOLD_QSIGMA) step_qmr_sigma(tot, k, act);
    else if (f.step == FOLD_QMR) step_qmr(tot, k, act);
    if (ng > 1) cnt[0] = 0;
  }
}

}  // namespace dda
