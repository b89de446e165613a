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

namespace dda {

// --------------------------------------------------------------------------
// x pass, forward: box rows -> scratch rows (y < ny)
// grid: (row tiles, R); block: rows [row0, row0+nlines) of RHS blockIdx.y
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_fft_x_fwd(OpView<T> op, const cplx_t<T>* __restrict__ in,
                            cplx_t<T>* __restrict__ buf, int nlines,
                            const int* __restrict__ active) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int nx = op.nx, Lx = op.Lx;
  const int rows = 3 * op.nz * op.ny;
  const int row0 = blockIdx.x * nlines;
  const int ps = nlines + 1;
  const C* src = in + ((int64_t)r * rows) * nx;
  for (int e = threadIdx.x; e < nlines * nx; e += blockDim.x) {
    const int line = e / nx, p = e - line * nx;
    const int row = row0 + line;
    s[p * ps + line] = row < rows ? src[(int64_t)row * nx + p] : mk<C>(0, 0);
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
// y pass (forward: ny -> Ly rows; inverse: Ly -> ny rows), in place
// grid: (column tiles, 3*nz planes, R)
// --------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void k_fft_y(OpView<T> op, cplx_t<T>* __restrict__ buf, int tile,
                        const int* __restrict__ active) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, Ly = op.Ly;
  const int col0 = blockIdx.x * tile;
  const int ncol = min(tile, Lx - col0);
  const int ps = tile;
  const int n_in = INV ? Ly : op.ny;
  const int n_out = INV ? op.ny : Ly;
  C* base = buf + ((int64_t)r * 3 * op.nz + blockIdx.y) * (int64_t)Ly * Lx + col0;
  for (int e = threadIdx.x; e < n_in * tile; e += blockDim.x) {
    const int p = e / tile, t = e - p * tile;
    s[p * ps + t] = t < ncol ? base[(int64_t)p * Lx + t] : mk<C>(0, 0);
  }
  for (int e = threadIdx.x; e < (Ly - n_in) * tile; e += blockDim.x) {
    const int p = n_in + e / tile, t = e % tile;
    s[p * ps + t] = mk<C>(0, 0);
  }
  __syncthreads();
  fft_smem<C, INV>(s, tile, ps, op.py, op.twy);
  for (int e = threadIdx.x; e < n_out * tile; e += blockDim.x) {
    const int p = e / tile, t = e - p * tile;
    if (t < ncol) base[(int64_t)p * Lx + t] = s[p * ps + t];
  }
}

// --------------------------------------------------------------------------
// z pass: forward FFT along z, multiply by Ghat (3x3 complex symmetric),
// inverse FFT along z; all three components of a column tile in one CTA.
// grid: (column tiles, Ly, R); shared memory holds 3*tile lines.
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
__global__ void k_fft_z_mul(OpView<T> op, cplx_t<T>* __restrict__ buf, int tile,
                            const int* __restrict__ active) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, Ly = op.Ly, Lz = op.Lz, nz = op.nz;
  const int ky = blockIdx.y;
  const int col0 = blockIdx.x * tile;
  const int ncol = min(tile, Lx - col0);
  const int nl = 3 * tile;
  const int ps = nl;
  const int64_t plane_sz = (int64_t)Ly * Lx;
  const int64_t comp_sz = (int64_t)nz * plane_sz;
  C* base = buf + (int64_t)r * 3 * comp_sz + (int64_t)ky * Lx + col0;
  for (int e = threadIdx.x; e < nz * nl; e += blockDim.x) {
    const int p = e / nl, l = e - p * nl;
    const int c = l / tile, t = l - c * tile;
    s[p * ps + l] = t < ncol ? base[c * comp_sz + p * plane_sz + t] : mk<C>(0, 0);
  }
  for (int e = threadIdx.x; e < (Lz - nz) * nl; e += blockDim.x) {
    const int p = nz + e / nl, l = e % nl;
    s[p * ps + l] = mk<C>(0, 0);
  }
  __syncthreads();
  fft_smem<C, false>(s, nl, ps, op.pz, op.twz);
  // pointwise multiply; positions along x, y, z are digit-reversed frequencies
  const int64_t gstride = (int64_t)op.Hz * op.Hy * op.Hx;
  const int kyf = op.ky_at[ky];
  for (int e = threadIdx.x; e < Lz * tile; e += blockDim.x) {
    const int pz = e / tile, t = e - pz * tile;
    if (t < ncol) {
      int64_t gi; bool fx, fy, fz;
      ghat_index(op, op.kx_at[col0 + t], kyf, op.kz_at[pz], gi, fx, fy, fz);
      const C gxx = op.ghat[gi];
      C gxy = op.ghat[gi + gstride];
      C gxz = op.ghat[gi + 2 * gstride];
      const C gyy = op.ghat[gi + 3 * gstride];
      C gyz = op.ghat[gi + 4 * gstride];
      const C gzz = op.ghat[gi + 5 * gstride];
      // odd components change sign under reflection of an odd axis
      if (fx != fy) { gxy.x = -gxy.x; gxy.y = -gxy.y; }
      if (fx != fz) { gxz.x = -gxz.x; gxz.y = -gxz.y; }
      if (fy != fz) { gyz.x = -gyz.x; gyz.y = -gyz.y; }
      C* q = s + pz * ps + t;
      const C x0 = q[0], x1 = q[tile], x2 = q[2 * tile];
      q[0] = cadd(cadd(cmul(gxx, x0), cmul(gxy, x1)), cmul(gxz, x2));
      q[tile] = cadd(cadd(cmul(gxy, x0), cmul(gyy, x1)), cmul(gyz, x2));
      q[2 * tile] = cadd(cadd(cmul(gxz, x0), cmul(gyz, x1)), cmul(gzz, x2));
    }
  }
  __syncthreads();
  fft_smem<C, true>(s, nl, ps, op.pz, op.twz);
  for (int e = threadIdx.x; e < nz * nl; e += blockDim.x) {
    const int p = e / nl, l = e - p * nl;
    const int c = l / tile, t = l - c * tile;
    if (t < ncol) base[c * comp_sz + p * plane_sz + t] = s[p * ps + l];
  }
}

// --------------------------------------------------------------------------
// x pass, inverse + diagonal term: y = ainv * x - conv on occupied sites
// grid: (row tiles, R)
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_fft_x_inv(OpView<T> op, const cplx_t<T>* __restrict__ buf,
                            const cplx_t<T>* __restrict__ xin, cplx_t<T>* __restrict__ yout,
                            int nlines, const int* __restrict__ active) {
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
  for (int e = threadIdx.x; e < nlines * nx; e += blockDim.x) {
    const int line = e / nx, p = e - line * nx;
    const int row = row0 + line;
    if (row < rows) {
      const int64_t site = (int64_t)(row % nyz) * nx + p;
      const int cm = op.comp[site];
      const int64_t g = (int64_t)row * nx + p;
      C out = mk<C>(0, 0);
      if (cm) out = csub(cmul(ai[cm], xr[g]), s[p * ps + line]);
      yr[g] = out;
    }
  }
}

// --------------------------------------------------------------------------
// launch configuration
// --------------------------------------------------------------------------
static int threads_for(int nlines, int L) {
  // enough threads for the butterflies of a radix-4 stage, 64..512
  int th = nlines * L / 4;
  th = ((th + 31) / 32) * 32;
  return th < 64 ? 64 : (th > 512 ? 512 : th);
}

template <typename T>
MatvecLaunch plan_matvec(const OpView<T>& op) {
  using C = cplx_t<T>;
  MatvecLaunch L{};
  // x passes: lines of Lx points, ~16-32 KB of shared memory per CTA
  int nl = 16;
  while (nl > 1 && (size_t)nl * (op.Lx + 1) * sizeof(C) > 32 * 1024) nl >>= 1;
  while (nl < 64 && (size_t)(2 * nl) * (op.Lx + 1) * sizeof(C) <= 16 * 1024) nl <<= 1;
  L.x_lines = nl;
  L.x_threads = threads_for(nl, op.Lx);
  L.x_smem = (size_t)op.Lx * (nl + 1) * sizeof(C);
  // y pass: column tile (tile * element >= 64 B keeps rows coalesced)
  int ty = sizeof(T) == 4 ? 16 : 8;
  while (ty > 1 && (size_t)ty * op.Ly * sizeof(C) > 64 * 1024) ty >>= 1;
  L.y_tile = ty;
  L.y_threads = threads_for(ty, op.Ly);
  L.y_smem = (size_t)op.Ly * ty * sizeof(C);
  // z pass: 3 components per tile
  int tz = sizeof(T) == 4 ? 8 : 4;
  while (tz > 1 && (size_t)3 * tz * op.Lz * sizeof(C) > 100 * 1024) tz >>= 1;
  L.z_tile = tz;
  L.z_threads = threads_for(3 * tz, op.Lz);
  L.z_smem = (size_t)op.Lz * 3 * tz * sizeof(C);
  return L;
}

template <typename T>
cudaError_t configure_matvec_kernels(const MatvecLaunch& L) {
  (void)L;
  cudaError_t e;
  e = cudaFuncSetAttribute(k_fft_x_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fft_x_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
  if (e != cudaSuccess) return e;
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

template <typename T>
cudaError_t launch_matvec(const OpView<T>& op, const MatvecLaunch& L, int R,
                          const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch,
                          const int* active, cudaStream_t st, const cudaEvent_t* ev) {
  const int rows = 3 * op.nz * op.ny;
  if (ev) cudaEventRecord(ev[0], st);
  dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
  k_fft_x_fwd<T><<<gx, L.x_threads, L.x_smem, st>>>(op, x, scratch, L.x_lines, active);
  note_launch();
  if (ev) cudaEventRecord(ev[1], st);
  dim3 gy((op.Lx + L.y_tile - 1) / L.y_tile, 3 * op.nz, R);
  k_fft_y<T, false><<<gy, L.y_threads, L.y_smem, st>>>(op, scratch, L.y_tile, active);
  note_launch();
  if (ev) cudaEventRecord(ev[2], st);
  dim3 gz((op.Lx + L.z_tile - 1) / L.z_tile, op.Ly, R);
  k_fft_z_mul<T><<<gz, L.z_threads, L.z_smem, st>>>(op, scratch, L.z_tile, active);
  note_launch();
  if (ev) cudaEventRecord(ev[3], st);
  k_fft_y<T, true><<<gy, L.y_threads, L.y_smem, st>>>(op, scratch, L.y_tile, active);
  note_launch();
  if (ev) cudaEventRecord(ev[4], st);
  k_fft_x_inv<T><<<gx, L.x_threads, L.x_smem, st>>>(op, scratch, x, y, L.x_lines, active);
  note_launch();
  if (ev) cudaEventRecord(ev[5], st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_fwd(const OpView<T>& op, const MatvecLaunch& L, int R,
                         const cplx_t<T>* x, cplx_t<T>* out, cudaStream_t st) {
  const int rows = 3 * op.nz * op.ny;
  dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
  k_fft_x_fwd<T><<<gx, L.x_threads, L.x_smem, st>>>(op, x, out, L.x_lines, nullptr);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_x_fwd<double>(const OpView<double>&, const MatvecLaunch&, int,
                                          const double2*, double2*, cudaStream_t);

template MatvecLaunch plan_matvec<float>(const OpView<float>&);
template MatvecLaunch plan_matvec<double>(const OpView<double>&);
template cudaError_t configure_matvec_kernels<float>(const MatvecLaunch&);
template cudaError_t configure_matvec_kernels<double>(const MatvecLaunch&);
template cudaError_t launch_matvec<float>(const OpView<float>&, const MatvecLaunch&, int,
                                          const float2*, float2*, float2*, const int*,
                                          cudaStream_t, const cudaEvent_t*);
template cudaError_t launch_matvec<double>(const OpView<double>&, const MatvecLaunch&, int,
                                           const double2*, double2*, double2*, const int*,
                                           cudaStream_t, const cudaEvent_t*);

}  // namespace dda
