// BiCGSTAB (van der Vorst 1992; the PIM method the guide's PBCGST option runs,
// Sec. "Choice of Iterative Algorithm") for R right-hand sides at once, plus
// the vector kernels of the FP64-refined FP32 solve.
//
// Every kernel covers all R right-hand sides (grid.y = rhs) and skips the ones
// whose `active` flag is 0, so a converged RHS is frozen while the others go
// on.  Inner products and norms are accumulated in FP64 whatever the vector
// precision, with a deterministic two-stage reduction: each block writes one
// partial per value, and a single block per RHS adds the partials in a fixed
// tree order inside the scalar kernels, so repeated runs are bit-identical.
#include "dda_ops.h"
#include "krylov_scalar.cuh"
#include "reduce.cuh"

namespace dda {

int reduce_blocks(int64_t n) {
  int64_t b = (n + 4 * kThreads - 1) / (4 * kThreads);
  if (b > 1216) b = 1216;  // 8 per SM on 152 SMs
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

template <typename C> __device__ __forceinline__ C from_d2(double2 a) {
  return mk<C>(a.x, a.y);
}


// ---- incident field ------------------------------------------------------------
template <typename T>
__global__ void k_einc(int nx, int ny, int nz, const uint8_t* __restrict__ comp,
                       RhsTables tb, cplx_t<T>* __restrict__ b) {
  using C = cplx_t<T>;
  const int r = blockIdx.y;
  const int64_t nbox = (int64_t)nx * ny * nz;
  GRID_LOOP(i, nbox) {
    const int ix = (int)(i % nx);
    const int64_t q = i / nx;
    const int iy = (int)(q % ny), iz = (int)(q / ny);
    double2 ph = make_double2(0.0, 0.0);
    if (comp[i]) ph = cmul(cmul(tb.phx[(int64_t)r * nx + ix], tb.phy[(int64_t)r * ny + iy]),
                           tb.phz[(int64_t)r * nz + iz]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 e = tb.pol[r * 3 + c];
      b[((int64_t)r * 3 + c) * nbox + i] = from_d2<C>(cmul(e, ph));
    }
  }
}

template <typename T>
cudaError_t launch_einc(int nx, int ny, int nz, const uint8_t* comp, RhsTables tb, int R,
                        cplx_t<T>* b, cudaStream_t st) {
  const int64_t nbox = (int64_t)nx * ny * nz;
  dim3 g(reduce_blocks(nbox), R);
  k_einc<T><<<g, kThreads, 0, st>>>(nx, ny, nz, comp, tb, b);
  note_launch();
  return cudaGetLastError();
}

// ---- BiCGSTAB -------------------------------------------------------------------
template <typename T>
__global__ void k_bicg_init(int64_t n, const cplx_t<T>* __restrict__ b,
                            const cplx_t<T>* __restrict__ ax, cplx_t<T>* __restrict__ r,
                            cplx_t<T>* __restrict__ rhat, cplx_t<T>* __restrict__ p,
                            cplx_t<T>* __restrict__ v, double* partials) {
  using C = cplx_t<T>;
  const int64_t off = (int64_t)blockIdx.y * n;
  ChunkAcc<T, 2> acc;
  GRID_LOOP(i, n) {
    const C bi = b[off + i];
    C ri = bi;
    if (ax) ri = csub(bi, ax[off + i]);
    r[off + i] = ri;
    rhat[off + i] = ri;
    p[off + i] = mk<C>(0, 0);
    v[off + i] = mk<C>(0, 0);
    acc.add(0, ri.x * ri.x + ri.y * ri.y);
    acc.add(1, bi.x * bi.x + bi.y * bi.y);
    acc.step();
  }
  acc.template write<2>(partials);
}

template <typename T>
cudaError_t launch_bicg_init(int64_t n, int R, const cplx_t<T>* b, const cplx_t<T>* ax,
                             cplx_t<T>* r, cplx_t<T>* rhat, cplx_t<T>* p, cplx_t<T>* v,
                             double* partials, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_bicg_init<T><<<g, kThreads, 0, st>>>(n, b, ax, r, rhat, p, v, partials);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_state_init(int nblk, const double* partials, KState* ks, int* active,
                             double tol, int max_iter) {
  const int r = blockIdx.x;
  double tot[2];
  sum_partials<2>(partials, nblk, r, tot);
  if (threadIdx.x == 0) {
    KState k;
    k.rnorm2 = tot[0];
    k.bnorm2 = tot[1];
    k.rho = make_double2(tot[0], 0.0);
    k.rho_old = make_double2(1.0, 0.0);
    k.alpha = make_double2(1.0, 0.0);
    k.omega = make_double2(1.0, 0.0);
    k.beta = make_double2(0.0, 0.0);
    k.tol2 = tol * tol;
    k.iters = 0;
    k.max_iter = max_iter;
    k.active_unused = 0;
    const bool done = !(k.rnorm2 > k.tol2 * k.bnorm2);
    k.status = done ? KS_CONV : KS_RUN;
    if (!isfinite(k.rnorm2)) k.status = KS_BREAKDOWN;
    ks[r] = k;
    active[r] = k.status == KS_RUN ? 1 : 0;
  }
}

cudaError_t launch_state_init(int R, int nblk, const double* partials, KState* ks,
                              int* active, double tol, int max_iter, cudaStream_t st) {
  k_state_init<<<R, kThreads, 0, st>>>(nblk, partials, ks, active, tol, max_iter);
  note_launch();
  return cudaGetLastError();
}

// The last node of a device-side iteration loop (the body of a CUDA-graph
// while-node): counts the block of iterations just run in ctl[0] and keeps the
// loop going while some right-hand side is still active and fewer than ctl[1]
// blocks have run -- so the loop ends after at most ctl[1] blocks whatever the
// flags say.
__global__ void k_loop_continue(cudaGraphConditionalHandle h, const int* __restrict__ active,
                                int R, int* ctl) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int a = 0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) a |= active[r];
  if (a) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int done = ctl[0] + 1;
    ctl[0] = done;
    cudaGraphSetConditional(h, (any && done < ctl[1]) ? 1u : 0u);
  }
}

cudaError_t launch_loop_continue(cudaGraphConditionalHandle h, const int* active, int R,
                                 int* ctl, cudaStream_t st) {
  k_loop_continue<<<1, kThreads, 0, st>>>(h, active, R, ctl);
  note_launch();
  return cudaGetLastError();
}



__global__ void k_scalar_alpha(int nblk, const double* partials, KState* ks, int* active) {
  const int r = blockIdx.x;
  if (!active[r]) return;
  double tot[2];
  sum_partials<2>(partials, nblk, r, tot);
  if (threadIdx.x == 0) step_alpha(tot, ks[r], active + r);
}

cudaError_t launch_scalar_alpha(int R, int nblk, const double* partials, KState* ks,
                                int* active, cudaStream_t st) {
  k_scalar_alpha<<<R, kThreads, 0, st>>>(nblk, partials, ks, active);
  note_launch();
  return cudaGetLastError();
}




template <typename T>
__global__ void k_update_xr(int64_t n, cplx_t<T>* __restrict__ x, cplx_t<T>* __restrict__ r,
                            const cplx_t<T>* __restrict__ p, const cplx_t<T>* __restrict__ s,
                            const cplx_t<T>* __restrict__ t, const cplx_t<T>* __restrict__ rhat,
                            double* partials, const KState* __restrict__ ks,
                            const int* __restrict__ active, FoldArgs fold) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[2];
  block_scalars<C, 2>({ks[rr].alpha, ks[rr].omega}, sc);
  const C alpha = sc[0], omega = sc[1];
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 4> acc;
  // batches of U elements per thread, every load of a batch issued before its
  // stores, so that 5 U loads per thread are in flight at once
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
    C xv[U], pv[U], sv[U], tv[U], hv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < n) {
        xv[u] = x[off + i]; pv[u] = p[off + i]; sv[u] = s[off + i];
        tv[u] = t[off + i]; hv[u] = rhat[off + i];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= n) break;
      x[off + i] = cadd(xv[u], cadd(cmul(alpha, pv[u]), cmul(omega, sv[u])));
      const C ri = csub(sv[u], cmul(omega, tv[u]));
      r[off + i] = ri;
      const C h = hv[u];
      acc.add(0, h.x * ri.x + h.y * ri.y);
      acc.add(1, h.x * ri.y - h.y * ri.x);
      acc.add(2, ri.x * ri.x + ri.y * ri.y);
      acc.step();
    }
  }
  acc.template write<4>(partials);
  if (fold.counter) fold_scalar_step<4>(partials, fold);
}

template <typename T>
cudaError_t launch_update_xr(int64_t n, int R, cplx_t<T>* x, cplx_t<T>* r,
                             const cplx_t<T>* p, const cplx_t<T>* s, const cplx_t<T>* t,
                             const cplx_t<T>* rhat, double* partials, const KState* ks,
                             const int* active, cudaStream_t st, FoldArgs fold) {
  dim3 g(reduce_blocks(n), R);
  k_update_xr<T><<<g, kThreads, 0, st>>>(n, x, r, p, s, t, rhat, partials, ks, active, fold);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_scalar_rho(int nblk, const double* partials, KState* ks, int* active) {
  const int r = blockIdx.x;
  if (!active[r]) return;
  double tot[4];
  sum_partials<4>(partials, nblk, r, tot);
  if (threadIdx.x == 0) step_rho(tot, ks[r], active + r);
}

cudaError_t launch_scalar_rho(int R, int nblk, const double* partials, KState* ks,
                              int* active, cudaStream_t st) {
  k_scalar_rho<<<R, kThreads, 0, st>>>(nblk, partials, ks, active);
  note_launch();
  return cudaGetLastError();
}

// ---- QMR for complex-symmetric A ------------------------------------------------
// The DDA matrix is complex symmetric (A = A^T), so the Lanczos process can
// run on the bilinear form x^T y with a single sequence of vectors and one
// matvec per iteration; the iterate minimises the quasi-residual (Freund 1992,
// coupled two-term recurrences of Freund & Nachtigal 1994; the guide's
// QMRCCG option, Sec. "Choice of Iterative Algorithm").  Per iteration k:
//   t = A q, sigma = q^T t, alpha = rho / sigma, r <- r - alpha t,
//   theta' = ||r|| / tau, c^2 = 1 / (1 + theta'^2), tau <- tau theta' c,
//   d <- c^2 theta^2 d + c^2 alpha q, x <- x + d, rho' = r^T r,
//   beta = rho' / rho, q <- r + beta q,
// and ||b - A x_k|| <= tau_k sqrt(k + 1) bounds the true residual.  The
// d/x/q updates of one iteration run in the next iteration's first FFT pass;
// the last one is applied by k_qmr_flush.

template <typename T>
__global__ void k_qmr_init(int64_t n, const cplx_t<T>* __restrict__ b,
                           const cplx_t<T>* __restrict__ ax, cplx_t<T>* __restrict__ r,
                           cplx_t<T>* __restrict__ q, cplx_t<T>* __restrict__ d,
                           double* partials) {
  using C = cplx_t<T>;
  const int64_t off = (int64_t)blockIdx.y * n;
  ChunkAcc<T, 4> acc;
  GRID_LOOP(i, n) {
    const C bi = b[off + i];
    C ri = bi;
    if (ax) ri = csub(bi, ax[off + i]);
    r[off + i] = ri;
    q[off + i] = mk<C>(0, 0);
    d[off + i] = mk<C>(0, 0);
    acc.add(0, ri.x * ri.x + ri.y * ri.y);
    acc.add(1, bi.x * bi.x + bi.y * bi.y);
    acc.add(2, ri.x * ri.x - ri.y * ri.y);
    acc.add(3, (T)2 * ri.x * ri.y);
    acc.step();
  }
  acc.template write<4>(partials);
}

template <typename T>
cudaError_t launch_qmr_init(int64_t n, int R, const cplx_t<T>* b, const cplx_t<T>* ax,
                            cplx_t<T>* r, cplx_t<T>* q, cplx_t<T>* d, double* partials,
                            cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_qmr_init<T><<<g, kThreads, 0, st>>>(n, b, ax, r, q, d, partials);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_qmr_state(int nblk, const double* partials, KState* ks, int* active,
                            double tol, int max_iter, double rho_floor) {
  const int r = blockIdx.x;
  double tot[4];
  sum_partials<4>(partials, nblk, r, tot);
  if (threadIdx.x == 0) {
    KState k;
    k.rnorm2 = tot[0];
    k.bnorm2 = tot[1];
    k.rho = make_double2(tot[2], tot[3]);
    k.rho_old = make_double2(1.0, 0.0);
    k.alpha = make_double2(0.0, 0.0);
    k.omega = make_double2(0.0, 0.0);
    k.beta = make_double2(0.0, 0.0);  // first pass: q = r + 0 q = r
    k.tau = sqrt(tot[0]);
    k.theta = 0.0;
    k.qa1 = make_double2(0.0, 0.0);   // no pending update yet
    k.qa2 = make_double2(0.0, 0.0);
    k.tol2 = tol * tol;
    k.iters = 0;
    k.max_iter = max_iter;
    k.active_unused = 0;
    k.rho_floor = rho_floor;
    const bool done = !(k.rnorm2 > k.tol2 * k.bnorm2);
    k.status = done ? KS_CONV : KS_RUN;
    // r^T r can vanish for r != 0 (e.g. circularly polarized E_inc has
    // E_j . E_j = 0 at every site): the bilinear Lanczos process cannot start
    if (!isfinite(k.rnorm2) || !finite2(k.rho)) k.status = KS_BREAKDOWN;
    else if (!done && hypot(k.rho.x, k.rho.y) <= k.rho_floor * k.rnorm2) k.status = KS_BREAKDOWN;
    ks[r] = k;
    active[r] = k.status == KS_RUN ? 1 : 0;
  }
}

cudaError_t launch_qmr_state(int R, int nblk, const double* partials, KState* ks,
                             int* active, double tol, int max_iter, double rho_floor,
                             cudaStream_t st) {
  k_qmr_state<<<R, kThreads, 0, st>>>(nblk, partials, ks, active, tol, max_iter, rho_floor);
  note_launch();
  return cudaGetLastError();
}


template <typename T>
__global__ void k_qmr_update_r(int64_t n, cplx_t<T>* __restrict__ r,
                               const cplx_t<T>* __restrict__ t, double* partials,
                               const KState* __restrict__ ks, const int* __restrict__ active,
                               FoldArgs fold) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  if (!active[rr]) return;
  C sc[1];
  block_scalars<C, 1>({ks[rr].alpha}, sc);
  const C alpha = sc[0];
  const int64_t off = (int64_t)rr * n;
  ChunkAcc<T, 4> acc;
  // batches of U elements per thread, loads before stores (as k_update_xr)
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
    C rv[U], tv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < n) { rv[u] = r[off + i]; tv[u] = t[off + i]; }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= n) break;
      const C ri = csub(rv[u], cmul(alpha, tv[u]));
      r[off + i] = ri;
      acc.add(0, ri.x * ri.x + ri.y * ri.y);
      acc.add(1, ri.x * ri.x - ri.y * ri.y);
      acc.add(2, (T)2 * ri.x * ri.y);
      acc.step();
    }
  }
  acc.template write<4>(partials);
  if (fold.counter) fold_scalar_step<4>(partials, fold);
}

template <typename T>
cudaError_t launch_qmr_update_r(int64_t n, int R, cplx_t<T>* r, const cplx_t<T>* t,
                                double* partials, const KState* ks, const int* active,
                                cudaStream_t st, FoldArgs fold) {
  dim3 g(reduce_blocks(n), R);
  k_qmr_update_r<T><<<g, kThreads, 0, st>>>(n, r, t, partials, ks, active, fold);
  note_launch();
  return cudaGetLastError();
}


template <typename T>
__global__ void k_qmr_flush(int64_t n, cplx_t<T>* __restrict__ x, cplx_t<T>* __restrict__ d,
                            const cplx_t<T>* __restrict__ q, const KState* __restrict__ ks) {
  using C = cplx_t<T>;
  const int rr = blockIdx.y;
  const double2 a1d = ks[rr].qa1, a2d = ks[rr].qa2;
  if (a1d.x == 0.0 && a1d.y == 0.0 && a2d.x == 0.0 && a2d.y == 0.0) return;
  const C a1 = from_d2<C>(a1d), a2 = from_d2<C>(a2d);
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const C dn = cadd(cmul(a1, d[off + i]), cmul(a2, q[off + i]));
    d[off + i] = dn;
    x[off + i] = cadd(x[off + i], dn);
  }
}

template <typename T>
cudaError_t launch_qmr_flush(int64_t n, int R, cplx_t<T>* x, cplx_t<T>* d,
                             const cplx_t<T>* q, const KState* ks, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_qmr_flush<T><<<g, kThreads, 0, st>>>(n, x, d, q, ks);
  note_launch();
  return cudaGetLastError();
}

// ---- refinement helpers -------------------------------------------------------------
__global__ void k_norm2(int64_t n, const double2* __restrict__ v, double* partials) {
  const int64_t off = (int64_t)blockIdx.y * n;
  double acc[1] = {0.0};
  GRID_LOOP(i, n) {
    const double2 a = v[off + i];
    acc[0] += a.x * a.x + a.y * a.y;
  }
  write_partials<1>(acc, partials);
}

cudaError_t launch_norm2(int64_t n, int R, const double2* v, double* partials,
                         cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_norm2<<<g, kThreads, 0, st>>>(n, v, partials);
  note_launch();
  return cudaGetLastError();
}

template <int NV>
__global__ void k_finalize(int nblk, const double* partials, double* out) {
  const int r = blockIdx.x;
  double tot[NV];
  sum_partials<NV>(partials, nblk, r, tot);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) out[r * NV + i] = tot[i];
  }
}

cudaError_t launch_finalize_sums(int R, int nblk, int nval, const double* partials,
                                 double* out, cudaStream_t st) {
  switch (nval) {
    case 1: k_finalize<1><<<R, kThreads, 0, st>>>(nblk, partials, out); break;
    case 2: k_finalize<2><<<R, kThreads, 0, st>>>(nblk, partials, out); break;
    case 4: k_finalize<4><<<R, kThreads, 0, st>>>(nblk, partials, out); break;
    case 6: k_finalize<6><<<R, kThreads, 0, st>>>(nblk, partials, out); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

// r may alias ax (each element is read before it is written by the same thread)
__global__ void k_residual(int64_t n, const double2* __restrict__ b, const double2* ax,
                           double2* r) {
  const int64_t off = (int64_t)blockIdx.y * n;
  GRID_LOOP(i, n) r[off + i] = csub(b[off + i], ax[off + i]);
}

cudaError_t launch_residual(int64_t n, int R, const double2* b, const double2* ax,
                            double2* r, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_residual<<<g, kThreads, 0, st>>>(n, b, ax, r);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_scale_to_f32(int64_t n, const double2* __restrict__ r64,
                               const double* __restrict__ norms, float2* __restrict__ r32,
                               const int* __restrict__ active) {
  const int rr = blockIdx.y;
  const double nr = norms[rr];
  // inactive RHS get a zero right-hand side, so the inner solve skips them
  const double sc = (nr > 0.0 && (!active || active[rr])) ? 1.0 / sqrt(nr) : 0.0;
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const double2 a = r64[off + i];
    r32[off + i] = make_float2((float)(a.x * sc), (float)(a.y * sc));
  }
}

cudaError_t launch_scale_to_f32(int64_t n, int R, const double2* r64, const double* norms,
                                float2* r32, const int* active, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_scale_to_f32<<<g, kThreads, 0, st>>>(n, r64, norms, r32, active);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_accumulate(int64_t n, double2* __restrict__ x64, const float2* __restrict__ d32,
                             const double* __restrict__ norms, const int* __restrict__ active) {
  const int rr = blockIdx.y;
  if (active && !active[rr]) return;
  const double sc = sqrt(norms[rr]);
  const int64_t off = (int64_t)rr * n;
  GRID_LOOP(i, n) {
    const float2 d = d32[off + i];
    double2 a = x64[off + i];
    a.x += sc * (double)d.x;
    a.y += sc * (double)d.y;
    x64[off + i] = a;
  }
}

cudaError_t launch_accumulate(int64_t n, int R, double2* x64, const float2* d32,
                              const double* norms, const int* active, cudaStream_t st) {
  dim3 g(reduce_blocks(n), R);
  k_accumulate<<<g, kThreads, 0, st>>>(n, x64, d32, norms, active);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_split_df(int64_t n, const double2* __restrict__ a, df64c* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = from_io<df64c>(a[i]);
}

cudaError_t launch_split_df(int64_t n, const double2* in, df64c* out, cudaStream_t st) {
  k_split_df<<<reduce_blocks(n), kThreads, 0, st>>>(n, in, out);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_f64_to_f32(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  GRID_LOOP(i, n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_f32_to_f64(int64_t n, const float2* __restrict__ a, double2* __restrict__ b) {
  GRID_LOOP(i, n) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

cudaError_t launch_f64_to_f32(int64_t n, const double2* a, float2* b, cudaStream_t st) {
  k_f64_to_f32<<<reduce_blocks(n), kThreads, 0, st>>>(n, a, b);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_f32_to_f64(int64_t n, const float2* a, double2* b, cudaStream_t st) {
  k_f32_to_f64<<<reduce_blocks(n), kThreads, 0, st>>>(n, a, b);
  note_launch();
  return cudaGetLastError();
}

// ---- gather / scatter between the site list and the box ------------------------------
__global__ void k_sites_to_box(int64_t N, int64_t nbox, const int64_t* __restrict__ site,
                               const double2* __restrict__ v, double2* __restrict__ box) {
  const int r = blockIdx.y;
  GRID_LOOP(j, N) {
    const int64_t s = site[j];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      box[((int64_t)r * 3 + c) * nbox + s] = v[((int64_t)r * N + j) * 3 + c];
  }
}

__global__ void k_box_to_sites(int64_t N, int64_t nbox, const int64_t* __restrict__ site,
                               const double2* __restrict__ box, double2* __restrict__ v) {
  const int r = blockIdx.y;
  GRID_LOOP(j, N) {
    const int64_t s = site[j];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      v[((int64_t)r * N + j) * 3 + c] = box[((int64_t)r * 3 + c) * nbox + s];
  }
}

cudaError_t launch_sites_to_box(int64_t N, int64_t nbox, int R, const int64_t* site,
                                const double2* v, double2* box, cudaStream_t st) {
  dim3 g(reduce_blocks(N), R);
  k_sites_to_box<<<g, kThreads, 0, st>>>(N, nbox, site, v, box);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_box_to_sites(int64_t N, int64_t nbox, int R, const int64_t* site,
                                const double2* box, double2* v, cudaStream_t st) {
  dim3 g(reduce_blocks(N), R);
  k_box_to_sites<<<g, kThreads, 0, st>>>(N, nbox, site, box, v);
  note_launch();
  return cudaGetLastError();
}

// ---- explicit instantiations ---------------------------------------------------------
#define INST(T)                                                                              \
  template cudaError_t launch_einc<T>(int, int, int, const uint8_t*, RhsTables, int,         \
                                      cplx_t<T>*, cudaStream_t);                             \
  template cudaError_t launch_bicg_init<T>(int64_t, int, const cplx_t<T>*, const cplx_t<T>*, \
                                           cplx_t<T>*, cplx_t<T>*, cplx_t<T>*, cplx_t<T>*,   \
                                           double*, cudaStream_t);                           \
  template cudaError_t launch_update_xr<T>(int64_t, int, cplx_t<T>*, cplx_t<T>*,             \
                                           const cplx_t<T>*, const cplx_t<T>*,               \
                                           const cplx_t<T>*, const cplx_t<T>*, double*,      \
                                           const KState*, const int*, cudaStream_t,    \
                                           FoldArgs);                                  \
  template cudaError_t launch_qmr_init<T>(int64_t, int, const cplx_t<T>*, const cplx_t<T>*,  \
                                          cplx_t<T>*, cplx_t<T>*, cplx_t<T>*, double*,       \
                                          cudaStream_t);                                     \
  template cudaError_t launch_qmr_update_r<T>(int64_t, int, cplx_t<T>*, const cplx_t<T>*,    \
                                              double*, const KState*, const int*,            \
                                              cudaStream_t, FoldArgs);                                 \
  template cudaError_t launch_qmr_flush<T>(int64_t, int, cplx_t<T>*, cplx_t<T>*,             \
                                           const cplx_t<T>*, const KState*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dda
