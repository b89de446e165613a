// The A.P product (the guide's eq. AP=E) as a zero-padded FFT convolution.
//
// (A P)_j = alpha_j^{-1} P_j - sum_{l != j} G(r_j - r_l) P_l.  The sum is a
// discrete convolution over lattice offsets; embedding it in a periodic grid of
// at least (2nx-1)(2ny-1)(2nz-1) points makes it circular, so it equals
// IFFT( Ghat . FFT(P) ) restricted to the box (Sec. "Choice of FFT Algorithm";
// Goodman, Draine & Flatau 1990).  The 3-D transforms are done axis by axis:
//   x pass  : per (rhs, comp, z, y<ny) row, nx inputs -> Lx outputs
//   y pass  : per (rhs, comp, z) plane and column tile, ny -> Ly (in place)
//   z pass  : per (rhs, ky) and column tile: forward along z (nz inputs),
//             3x3 complex-symmetric multiply by Ghat, inverse along z, keep nz
//   y pass  : inverse, Ly -> ny
//   x pass  : inverse, Lx -> nx, then y = ainv * P - conv on occupied sites.
// Inputs that are known to be zero (beyond the box) are never read and outputs
// outside the box are never written (pruned transforms).
#include "dda_ops.h"
#include "fft_core.cuh"
#include "reduce.cuh"

namespace dda {

// --------------------------------------------------------------------------
// x pass, forward: box rows -> scratch rows (y < ny)
// grid: (row tiles, R); block: rows [row0, row0+nlines) of RHS blockIdx.y
// --------------------------------------------------------------------------
// Prologue of the first pass, fused with a BiCGSTAB vector update:
//   XIN_PLAIN : transform x as given;
//   XIN_P     : p <- r + beta (p - omega v), stored back, then transformed;
//   XIN_S     : s <- r - alpha v, stored, then transformed.
enum { XIN_PLAIN = 0, XIN_P = 1, XIN_S = 2 };

template <typename T> struct XinArgs {
  const cplx_t<T>* r;
  cplx_t<T>* pv;          // p (XIN_P, read and written) or s (XIN_S, written)
  const cplx_t<T>* v;
  const KState* ks;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_x_fwd(OpView<T> op, const cplx_t<T>* __restrict__ in,
                            cplx_t<T>* __restrict__ buf, int nlines,
                            const int* __restrict__ active, XinArgs<T> xa) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int nx = op.nx, Lx = op.Lx;
  const int rows = 3 * op.nz * op.ny;
  const int row0 = blockIdx.x * nlines;
  const int ps = nlines + 1;
  const int64_t off = (int64_t)r * rows * nx;
  C c1 = mk<C>(0, 0), c2 = mk<C>(0, 0);
  if (MODE == XIN_P) {
    c1 = mk<C>(xa.ks[r].beta.x, xa.ks[r].beta.y);
    c2 = mk<C>(xa.ks[r].omega.x, xa.ks[r].omega.y);
  } else if (MODE == XIN_S) {
    c1 = mk<C>(xa.ks[r].alpha.x, xa.ks[r].alpha.y);
  }
  for (int e = threadIdx.x; e < nlines * nx; e += blockDim.x) {
    const int line = e / nx, p = e - line * nx;
    const int row = row0 + line;
    C val = mk<C>(0, 0);
    if (row < rows) {
      const int64_t g = off + (int64_t)row * nx + p;
      if (MODE == XIN_PLAIN) {
        val = in[g];
      } else if (MODE == XIN_P) {
        val = cadd(xa.r[g], cmul(c1, csub(xa.pv[g], cmul(c2, xa.v[g]))));
        xa.pv[g] = val;
      } else {
        val = csub(xa.r[g], cmul(c1, xa.v[g]));
        xa.pv[g] = val;
      }
    }
    s[p * ps + line] = val;
  }
  for (int e = threadIdx.x; e < nlines * (Lx - nx); e += blockDim.x) {
    const int line = e % nlines, p = nx + e / nlines;
    s[p * ps + line] = mk<C>(0, 0);
  }
  __syncthreads();
  fft_smem<C, false>(s, nlines, ps, op.px, op.twx);
  const int64_t plane_sz = (int64_t)op.Ly * Lx;
  C* dst = buf + (int64_t)r * 3 * op.nz * plane_sz;
  for (int e = threadIdx.x; e < nlines * Lx; e += blockDim.x) {
    const int line = e / Lx, p = e - line * Lx;
    const int row = row0 + line;
    if (row < rows) {
      const int plane = row / op.ny, y = row - plane * op.ny;
      dst[plane * plane_sz + (int64_t)y * Lx + p] = s[p * ps + line];
    }
  }
}

// --------------------------------------------------------------------------
// y pass (forward: ny -> Ly rows; inverse: Ly -> ny rows), in place.
// grid: (column tiles, 3*nz planes, R).  The first stage reads straight from
// global memory and the last stage writes straight back (coalesced across the
// tile's columns); only the inner stages go through shared memory.
// --------------------------------------------------------------------------
template <typename C> struct ColIO {
  C* base;        // first column of the tile, row 0
  int64_t rs;     // row stride (elements)
  int ncol;       // valid columns in the tile
  int nrow;       // rows that exist on this side (input rows for loads, output rows for stores)
  __device__ __forceinline__ C operator()(int t, int p) const {
    return (t < ncol && p < nrow) ? base[p * rs + t] : mk<C>(0, 0);
  }
  __device__ __forceinline__ void operator()(int t, int p, C v) const {
    if (t < ncol && p < nrow) base[p * rs + t] = v;
  }
};

template <typename T, bool INV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_y(OpView<T> op, cplx_t<T>* __restrict__ buf,
                                               int tile, const int* __restrict__ active) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, Ly = op.Ly;
  const int col0 = blockIdx.x * tile;
  const int ncol = min(tile, Lx - col0);
  C* base = buf + ((int64_t)r * 3 * op.nz + blockIdx.y) * (int64_t)Ly * Lx + col0;
  ColIO<C> in{base, Lx, ncol, INV ? Ly : op.ny};
  ColIO<C> out{base, Lx, ncol, INV ? op.ny : Ly};
  if (op.py.nstage >= 2) {
    if (INV) fft_global_inv<C>(s, tile, tile, op.py, op.twy, in, out);
    else fft_global_fwd<C>(s, tile, tile, op.py, op.twy, in, out);
    return;
  }
  // one stage (Ly <= 16) or none: through shared memory
  for (int e = threadIdx.x; e < Ly * tile; e += blockDim.x) {
    const int p = e / tile, t = e - p * tile;
    s[p * tile + t] = in(t, p);
  }
  __syncthreads();
  fft_smem<C, INV>(s, tile, tile, op.py, op.twy);
  for (int e = threadIdx.x; e < Ly * tile; e += blockDim.x) {
    const int p = e / tile, t = e - p * tile;
    out(t, p, s[p * tile + t]);
  }
}

// --------------------------------------------------------------------------
// z pass: forward FFT along z, multiply by Ghat (3x3 complex symmetric),
// inverse FFT along z; the three components of a column tile in one CTA.
// grid: (column tiles, Ly, R).  Lines in shared memory: c*tile + t, row pitch ps.
// The last forward stage, the multiply and the first inverse stage run in
// registers for all three components of one butterfly.
// --------------------------------------------------------------------------
// Octant index of frequency (kx, ky, kz) and the reflections applied per axis.
template <typename T>
__device__ __forceinline__ void ghat_index(const OpView<T>& op, int kx, int ky, int kz,
                                           int64_t& idx, bool& fx, bool& fy, bool& fz) {
  fx = kx > (op.Lx >> 1); fy = ky > (op.Ly >> 1); fz = kz > (op.Lz >> 1);
  const int hx = fx ? op.Lx - kx : kx;
  const int hy = fy ? op.Ly - ky : ky;
  const int hz = fz ? op.Lz - kz : kz;
  idx = ((int64_t)hz * op.Hy + hy) * op.Hx + hx;
}

template <typename T>
__device__ __forceinline__ void ghat_apply(const OpView<T>& op, int kx, int ky, int kz,
                                           cplx_t<T>& x0, cplx_t<T>& x1, cplx_t<T>& x2) {
  using C = cplx_t<T>;
  int64_t gi; bool fx, fy, fz;
  ghat_index(op, kx, ky, kz, gi, fx, fy, fz);
  const int64_t gs = (int64_t)op.Hz * op.Hy * op.Hx;
  const C gxx = __ldg(&op.ghat[gi]);
  C gxy = __ldg(&op.ghat[gi + gs]);
  C gxz = __ldg(&op.ghat[gi + 2 * gs]);
  const C gyy = __ldg(&op.ghat[gi + 3 * gs]);
  C gyz = __ldg(&op.ghat[gi + 4 * gs]);
  const C gzz = __ldg(&op.ghat[gi + 5 * gs]);
  // odd components change sign under the reflection of an odd axis
  if (fx != fy) { gxy.x = -gxy.x; gxy.y = -gxy.y; }
  if (fx != fz) { gxz.x = -gxz.x; gxz.y = -gxz.y; }
  if (fy != fz) { gyz.x = -gyz.x; gyz.y = -gyz.y; }
  const C a = x0, b = x1, c = x2;
  x0 = cadd(cadd(cmul(gxx, a), cmul(gxy, b)), cmul(gxz, c));
  x1 = cadd(cadd(cmul(gxy, a), cmul(gyy, b)), cmul(gyz, c));
  x2 = cadd(cadd(cmul(gxz, a), cmul(gyz, b)), cmul(gzz, c));
}

template <typename C> struct ZIO {
  C* base;          // component 0, row 0, first column of the tile
  int64_t comp_sz;  // elements between components
  int64_t plane;    // elements between z rows
  int tile, ncol, nz;
  __device__ __forceinline__ C operator()(int l, int p) const {
    const int c = l / tile, t = l - c * tile;
    return (t < ncol && p < nz) ? base[c * comp_sz + p * plane + t] : mk<C>(0, 0);
  }
  __device__ __forceinline__ void operator()(int l, int p, C v) const {
    const int c = l / tile, t = l - c * tile;
    if (t < ncol && p < nz) base[c * comp_sz + p * plane + t] = v;
  }
};

// last forward stage + multiply + first inverse stage (block = R, span 1).  A
// thread owns R consecutive positions of one column for all three components;
// it transforms each component in registers and leaves it in place, multiplies
// position by position, and transforms back -- no barrier is needed between
// these steps because no other thread touches those positions.
template <typename T, int R>
__device__ __forceinline__ void z_mid(cplx_t<T>* s, int tile, int ps, int ncol, int col0,
                                      int ky, const OpView<T>& op) {
  using C = cplx_t<T>;
  const int nb = tile * (op.Lz / R);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int t = b % tile, blk = b / tile;
    C* q = s + (blk * R) * ps + t;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C v[R];
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = q[i * ps + c * tile];
      dft<R, false>(v);
#pragma unroll
      for (int i = 0; i < R; ++i) q[i * ps + c * tile] = v[i];
    }
    if (t < ncol) {
      const int kx = op.kx_at[col0 + t];
#pragma unroll 1
      for (int i = 0; i < R; ++i) {
        C* w = q + i * ps;
        C a = w[0], bb = w[tile], c = w[2 * tile];
        ghat_apply<T>(op, kx, ky, op.kz_at[blk * R + i], a, bb, c);
        w[0] = a; w[tile] = bb; w[2 * tile] = c;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C v[R];
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = q[i * ps + c * tile];
      dft<R, true>(v);
#pragma unroll
      for (int i = 0; i < R; ++i) q[i * ps + c * tile] = v[i];
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_z_mul(OpView<T> op, cplx_t<T>* __restrict__ buf,
                                                   int tile, int ps,
                                                   const int* __restrict__ active) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, Ly = op.Ly, Lz = op.Lz, nz = op.nz;
  const int pyy = blockIdx.y;
  const int ky = op.ky_at[pyy];
  const int col0 = blockIdx.x * tile;
  const int ncol = min(tile, Lx - col0);
  const int nl = 3 * tile;
  const int64_t plane_sz = (int64_t)Ly * Lx;
  const int64_t comp_sz = (int64_t)nz * plane_sz;
  C* base = buf + (int64_t)r * 3 * comp_sz + (int64_t)pyy * Lx + col0;
  ZIO<C> io{base, comp_sz, plane_sz, tile, ncol, nz};
  const AxisPlan& P = op.pz;
  const int last = P.nstage - 1;
  if (P.nstage >= 2) {
    DDA_RADIX_DISPATCH(P.radix[0], (stage_first_fwd<C, RR>(s, nl, ps, Lz, op.twz, io)));
    fft_inner_stages<C, false>(s, nl, ps, P, op.twz);
  } else {
    for (int e = threadIdx.x; e < Lz * nl; e += blockDim.x) {
      const int p = e / nl, l = e - p * nl;
      s[p * ps + l] = io(l, p);
    }
    __syncthreads();
  }
  if (P.nstage >= 1) {
    // the plan puts a radix <= 8 last
    DDA_RADIX_DISPATCH_SMALL(P.radix[last], (z_mid<T, RR>(s, tile, ps, ncol, col0, ky, op)));
  } else {  // Lz = 1
    for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
      C* q = s + t;
      C a = q[0], b = q[tile], c = q[2 * tile];
      ghat_apply<T>(op, op.kx_at[col0 + t], ky, 0, a, b, c);
      q[0] = a; q[tile] = b; q[2 * tile] = c;
    }
    __syncthreads();
  }
  if (P.nstage >= 2) {
    fft_inner_stages<C, true>(s, nl, ps, P, op.twz);
    DDA_RADIX_DISPATCH(P.radix[0], (stage_last_inv<C, RR>(s, nl, ps, Lz, op.twz, io)));
  } else {
    for (int e = threadIdx.x; e < Lz * nl; e += blockDim.x) {
      const int p = e / nl, l = e - p * nl;
      io(l, p, s[p * ps + l]);
    }
  }
}

// --------------------------------------------------------------------------
// x pass, inverse + diagonal term: y = ainv * x - conv on occupied sites
// grid: (row tiles, R)
// --------------------------------------------------------------------------
// Epilogue of the last pass, fused with BiCGSTAB inner products (FP64-accumulated,
// per-block partials [R][gridDim.x][NV]):
//   XOUT_PLAIN : none;
//   XOUT_RV    : <rhat, y>              (y = v = A p)
//   XOUT_TS    : <y, x>, <y, y>         (y = t = A s, x = s)
enum { XOUT_PLAIN = 0, XOUT_RV = 1, XOUT_TS = 2 };

template <typename T, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_x_inv(OpView<T> op, const cplx_t<T>* __restrict__ buf,
                            const cplx_t<T>* __restrict__ xin, cplx_t<T>* __restrict__ yout,
                            int nlines, const int* __restrict__ active,
                            const cplx_t<T>* __restrict__ rhat, double* __restrict__ partials) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int nx = op.nx, Lx = op.Lx;
  const int rows = 3 * op.nz * op.ny;
  const int row0 = blockIdx.x * nlines;
  const int ps = nlines + 1;
  const int64_t plane_sz = (int64_t)op.Ly * Lx;
  const C* src = buf + (int64_t)r * 3 * op.nz * plane_sz;
  for (int e = threadIdx.x; e < nlines * Lx; e += blockDim.x) {
    const int line = e / Lx, p = e - line * Lx;
    const int row = row0 + line;
    C v = mk<C>(0, 0);
    if (row < rows) {
      const int plane = row / op.ny, y = row - plane * op.ny;
      v = src[plane * plane_sz + (int64_t)y * Lx + p];
    }
    s[p * ps + line] = v;
  }
  __syncthreads();
  fft_smem<C, true>(s, nlines, ps, op.px, op.twx);
  const C* ai = op.ainv + (int64_t)r * op.ncomp1;
  const C* xr = xin + (int64_t)r * rows * nx;
  C* yr = yout + (int64_t)r * rows * nx;
  const int nyz = op.ny * op.nz;
  ChunkAcc<T, 4> acc;
  for (int e = threadIdx.x; e < nlines * nx; e += blockDim.x) {
    const int line = e / nx, p = e - line * nx;
    const int row = row0 + line;
    if (row < rows) {
      const int64_t site = (int64_t)(row % nyz) * nx + p;
      const int cm = op.comp[site];
      const int64_t g = (int64_t)row * nx + p;
      C out = mk<C>(0, 0);
      const C xv = xr[g];
      if (cm) out = csub(cmul(ai[cm], xv), s[p * ps + line]);
      yr[g] = out;
      if (MODE == XOUT_RV) {
        const C h = rhat[(int64_t)r * rows * nx + g];
        acc.add(0, h.x * out.x + h.y * out.y);
        acc.add(1, h.x * out.y - h.y * out.x);
        acc.step();
      } else if (MODE == XOUT_TS) {
        acc.add(0, out.x * xv.x + out.y * xv.y);
        acc.add(1, out.x * xv.y - out.y * xv.x);
        acc.add(2, out.x * out.x + out.y * out.y);
        acc.step();
      }
    }
  }
  if (MODE != XOUT_PLAIN) {
    acc.flush();
    if (MODE == XOUT_RV) {
      double v2[2] = {acc.tot[0], acc.tot[1]};
      write_partials<2>(v2, partials);
    } else {
      write_partials<4>(acc.tot, partials);
    }
  }
}

// --------------------------------------------------------------------------
// launch configuration
// --------------------------------------------------------------------------
template <typename T>
MatvecLaunch plan_matvec(const OpView<T>& op) {
  using C = cplx_t<T>;
  MatvecLaunch L{};
  // x passes: 256 threads, lines of Lx points, <= 32 KB of shared memory per CTA
  int nl = 16;
  while (nl > 1 && (size_t)nl * (op.Lx + 1) * sizeof(C) > 32 * 1024) nl >>= 1;
  while (nl < 64 && (size_t)(2 * nl) * (op.Lx + 1) * sizeof(C) <= 16 * 1024) nl <<= 1;
  L.x_lines = nl;
  L.x_threads = 256;
  L.x_smem = (size_t)op.Lx * (nl + 1) * sizeof(C);
  // y pass: a tile of 128 B of columns (16 FP32 / 8 FP64 complex), 256 threads
  int ty = 128 / (int)sizeof(C);
  while (ty > 2 && (size_t)ty * op.Ly * sizeof(C) > 64 * 1024) ty >>= 1;
  L.y_tile = ty;
  L.y_threads = 256;
  L.y_smem = (size_t)op.Ly * ty * sizeof(C);
  // z pass: three components of a tile of columns; the row pitch is made odd
  // when the tile is narrower than a half-warp's 128 B so that the butterflies
  // of neighbouring blocks fall on different banks
  int tz = 128 / (int)sizeof(C);
  while (tz > 2 && (size_t)3 * tz * op.Lz * sizeof(C) > 64 * 1024) tz >>= 1;
  L.z_tile = tz;
  L.z_ps = 3 * tz + (tz * (int)sizeof(C) < 128 ? 1 : 0);
  L.z_threads = 256;
  L.z_smem = (size_t)op.Lz * L.z_ps * sizeof(C);
  return L;
}

template <typename T>
cudaError_t configure_matvec_kernels(const MatvecLaunch& L) {
  (void)L;
  cudaError_t e;
  const void* xk[] = {(const void*)k_fft_x_fwd<T, XIN_PLAIN>, (const void*)k_fft_x_fwd<T, XIN_P>,
                      (const void*)k_fft_x_fwd<T, XIN_S>, (const void*)k_fft_x_inv<T, XOUT_PLAIN>,
                      (const void*)k_fft_x_inv<T, XOUT_RV>, (const void*)k_fft_x_inv<T, XOUT_TS>};
  for (const void* k : xk) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_fft_y<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fft_y<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fft_z_mul<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
  return e;
}

template <typename T, int XIN, int XOUT>
static cudaError_t matvec_passes(const OpView<T>& op, const MatvecLaunch& L, int R,
                                 const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch,
                                 const int* active, cudaStream_t st, const cudaEvent_t* ev,
                                 XinArgs<T> xa, const cplx_t<T>* rhat, double* partials) {
  const int rows = 3 * op.nz * op.ny;
  if (ev) cudaEventRecord(ev[0], st);
  dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
  k_fft_x_fwd<T, XIN><<<gx, L.x_threads, L.x_smem, st>>>(op, x, scratch, L.x_lines, active, xa);
  note_launch();
  if (ev) cudaEventRecord(ev[1], st);
  dim3 gy((op.Lx + L.y_tile - 1) / L.y_tile, 3 * op.nz, R);
  k_fft_y<T, false><<<gy, L.y_threads, L.y_smem, st>>>(op, scratch, L.y_tile, active);
  note_launch();
  if (ev) cudaEventRecord(ev[2], st);
  dim3 gz((op.Lx + L.z_tile - 1) / L.z_tile, op.Ly, R);
  k_fft_z_mul<T><<<gz, L.z_threads, L.z_smem, st>>>(op, scratch, L.z_tile, L.z_ps, active);
  note_launch();
  if (ev) cudaEventRecord(ev[3], st);
  k_fft_y<T, true><<<gy, L.y_threads, L.y_smem, st>>>(op, scratch, L.y_tile, active);
  note_launch();
  if (ev) cudaEventRecord(ev[4], st);
  k_fft_x_inv<T, XOUT><<<gx, L.x_threads, L.x_smem, st>>>(op, scratch, x, y, L.x_lines, active,
                                                          rhat, partials);
  note_launch();
  if (ev) cudaEventRecord(ev[5], st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_matvec(const OpView<T>& op, const MatvecLaunch& L, int R,
                          const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch,
                          const int* active, cudaStream_t st, const cudaEvent_t* ev) {
  return matvec_passes<T, XIN_PLAIN, XOUT_PLAIN>(op, L, R, x, y, scratch, active, st, ev,
                                                 XinArgs<T>{}, nullptr, nullptr);
}

template <typename T>
int matvec_partial_blocks(const OpView<T>& op, const MatvecLaunch& L) {
  const int rows = 3 * op.nz * op.ny;
  return (rows + L.x_lines - 1) / L.x_lines;
}

template <typename T>
cudaError_t launch_matvec_p(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, cplx_t<T>* p, cplx_t<T>* v,
                            const cplx_t<T>* rhat, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev) {
  XinArgs<T> xa{r, p, v, ks};
  return matvec_passes<T, XIN_P, XOUT_RV>(op, L, R, p, v, scratch, active, st, ev, xa, rhat,
                                          partials);
}

template <typename T>
cudaError_t launch_matvec_s(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, const cplx_t<T>* v, cplx_t<T>* s_vec,
                            cplx_t<T>* t_vec, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev) {
  XinArgs<T> xa{r, s_vec, v, ks};
  return matvec_passes<T, XIN_S, XOUT_TS>(op, L, R, s_vec, t_vec, scratch, active, st, ev, xa,
                                          nullptr, partials);
}

template <typename T>
cudaError_t launch_x_fwd(const OpView<T>& op, const MatvecLaunch& L, int R,
                         const cplx_t<T>* x, cplx_t<T>* out, cudaStream_t st) {
  const int rows = 3 * op.nz * op.ny;
  dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
  k_fft_x_fwd<T, XIN_PLAIN><<<gx, L.x_threads, L.x_smem, st>>>(op, x, out, L.x_lines, nullptr,
                                                               XinArgs<T>{});
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_x_fwd<double>(const OpView<double>&, const MatvecLaunch&, int,
                                          const double2*, double2*, cudaStream_t);

template MatvecLaunch plan_matvec<float>(const OpView<float>&);
template MatvecLaunch plan_matvec<double>(const OpView<double>&);
template cudaError_t configure_matvec_kernels<float>(const MatvecLaunch&);
template cudaError_t configure_matvec_kernels<double>(const MatvecLaunch&);
#define INST_KRY(T)                                                                        \
  template int matvec_partial_blocks<T>(const OpView<T>&, const MatvecLaunch&);            \
  template cudaError_t launch_matvec_p<T>(const OpView<T>&, const MatvecLaunch&, int,       \
                                          const cplx_t<T>*, cplx_t<T>*, cplx_t<T>*,         \
                                          const cplx_t<T>*, cplx_t<T>*, const KState*,      \
                                          double*, const int*, cudaStream_t,                \
                                          const cudaEvent_t*);                              \
  template cudaError_t launch_matvec_s<T>(const OpView<T>&, const MatvecLaunch&, int,       \
                                          const cplx_t<T>*, const cplx_t<T>*, cplx_t<T>*,   \
                                          cplx_t<T>*, cplx_t<T>*, const KState*, double*,   \
                                          const int*, cudaStream_t, const cudaEvent_t*);
INST_KRY(float)
INST_KRY(double)
#undef INST_KRY

template cudaError_t launch_matvec<float>(const OpView<float>&, const MatvecLaunch&, int,
                                          const float2*, float2*, float2*, const int*,
                                          cudaStream_t, const cudaEvent_t*);
template cudaError_t launch_matvec<double>(const OpView<double>&, const MatvecLaunch&, int,
                                           const double2*, double2*, double2*, const int*,
                                           cudaStream_t, const cudaEvent_t*);

}  // namespace dda
