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
//
// This header holds the kernel and launcher templates; matvec_f32.cu,
// matvec_f64.cu and matvec_df.cu instantiate them for one arithmetic each, so
// the three compile in parallel.
#pragma once

#include <type_traits>

#include "dda_ops.h"
#include "fft_core.cuh"
#include "fft_plan.cuh"
#include "krylov_scalar.cuh"
#include "reduce.cuh"

namespace dda {

// --------------------------------------------------------------------------
// x pass, forward: box rows -> scratch rows (y < ny)
// grid: (row tiles, R); block: rows [row0, row0+nlines) of RHS blockIdx.y
// --------------------------------------------------------------------------
// Prologue of the first pass, fused with a BiCGSTAB vector update:
//   XIN_PLAIN : transform x as given;
//   XIN_P     : p <- r + beta (p - omega v), stored back, then transformed;
//   XIN_S     : s <- r - alpha v, stored, then transformed;
//   XIN_Q     : the QMR step left pending by the previous iteration,
//               d <- a1 d + a2 q, x <- x + d, then q <- r + beta q, stored
//               and transformed (all with the old q).
enum { XIN_PLAIN = 0, XIN_P = 1, XIN_S = 2, XIN_Q = 3 };

template <typename T> struct XinArgs {
  const cplx_t<T>* r;
  cplx_t<T>* pv;          // p (XIN_P), s (XIN_S) or q (XIN_Q)
  const cplx_t<T>* v;
  const KState* ks;
  cplx_t<T>* d;           // XIN_Q: QMR direction and iterate
  cplx_t<T>* x;
};

// P: void -- the radix plan is read at run time; a FixedPlan -- Lx and the
// stages are compile-time constants (FP32, see fft_plan.cuh).
template <class P> constexpr int plan_len() {
  if constexpr (std::is_void<P>::value) return 0;
  else return P::L;
}

template <typename T, int MODE, class P = void>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_x_fwd(OpView<T> op, const io_t<T>* __restrict__ in,
                            cplx_t<T>* __restrict__ buf, int nlines, unsigned long long div_nl,
                            const int* __restrict__ active, XinArgs<T> xa) {
  using C = cplx_t<T>;
  constexpr int LP = plan_len<P>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int nx = op.nx, Lx = LP ? LP : op.Lx;
  const int rows = 3 * op.nz * op.ny;
  const int row0 = blockIdx.x * nlines;
  const int ps = nlines + 1;
  const int64_t off = (int64_t)r * rows * nx;
  C c1 = mk<C>(0, 0), c2 = mk<C>(0, 0), c3 = mk<C>(0, 0);
  if constexpr (MODE == XIN_P) {
    C sc[2];
    block_scalars<C, 2>({xa.ks[r].beta, xa.ks[r].omega}, sc);
    c1 = sc[0]; c2 = sc[1];
  } else if constexpr (MODE == XIN_S) {
    C sc[1];
    block_scalars<C, 1>({xa.ks[r].alpha}, sc);
    c1 = sc[0];
  } else if constexpr (MODE == XIN_Q) {
    C sc[3];
    block_scalars<C, 3>({xa.ks[r].beta, xa.ks[r].qa1, xa.ks[r].qa2}, sc);
    c1 = sc[0]; c2 = sc[1]; c3 = sc[2];
  }
  // the CTA's rows are one contiguous chunk of the box vector.  Elements go in
  // batches of U per thread with every load of a batch issued before any
  // store (the prologue writes vectors the next elements read from, so
  // without this split each thread would wait on one element at a time).
  const int nin = min(nlines, rows - row0) * nx;
  const int64_t g0 = off + (int64_t)row0 * nx;
  constexpr int U = 4;
  const int total = nlines * nx;
  for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
    C va[U], vb[U], vc[U], vd[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < nin) {
        const int64_t g = g0 + e;
        if (MODE == XIN_PLAIN) {
          va[u] = from_io<C>(in[g]);
        } else if (MODE == XIN_P) {
          va[u] = xa.r[g]; vb[u] = xa.pv[g]; vc[u] = xa.v[g];
        } else if (MODE == XIN_Q) {
          va[u] = xa.r[g]; vb[u] = xa.pv[g]; vc[u] = xa.d[g]; vd[u] = xa.x[g];
        } else {
          va[u] = xa.r[g]; vc[u] = xa.v[g];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= total) break;
      const int line = fast_div(e, op.div_nx), p = e - line * nx;
      C val = mk<C>(0, 0);
      if (e < nin) {
        const int64_t g = g0 + e;
        if (MODE == XIN_PLAIN) {
          val = va[u];
        } else if (MODE == XIN_P) {
          val = cadd(va[u], cmul(c1, csub(vb[u], cmul(c2, vc[u]))));
          xa.pv[g] = val;
        } else if (MODE == XIN_Q) {
          const C q = vb[u];
          const C dn = cadd(cmul(c2, vc[u]), cmul(c3, q));
          xa.d[g] = dn;
          xa.x[g] = cadd(vd[u], dn);
          val = cadd(va[u], cmul(c1, q));
          xa.pv[g] = val;
        } else {
          val = csub(va[u], cmul(c1, vc[u]));
          xa.pv[g] = val;
        }
      }
      s[p * ps + line] = val;
    }
  }
  // padding: with at most Lx/2 values per row (and an even first radix) the
  // first stage never reads positions >= Lx/2, so only nx .. Lx/2 - 1 are zeroed
  const bool half = 2 * nx <= Lx && op.px.radix[0] % 2 == 0;
  const int zend = half ? Lx / 2 : Lx;
  for (int e = threadIdx.x; e < nlines * (zend - nx); e += blockDim.x) {
    const int q = fast_div(e, div_nl), line = e - q * nlines, p = nx + q;
    s[p * ps + line] = mk<C>(0, 0);
  }
  __syncthreads();
  if constexpr (std::is_void<P>::value) fft_smem<C, false>(s, nlines, ps, op.px, op.twx, half);
  else fft_smem_p<C, false, P>(s, nlines, div_nl, ps, op.twx, half);
  const int64_t plane_sz = (int64_t)op.Ly * Lx;
  C* dst = buf + (int64_t)r * 3 * op.nz * plane_sz;
  // one line at a time: the row's plane and y are worked out once per line
  const int nrow = min(nlines, rows - row0);
  for (int line = 0; line < nrow; ++line) {
    const int row = row0 + line;
    const int plane = fast_div(row, op.div_ny), y = row - plane * op.ny;
    C* drow = dst + plane * plane_sz + (int64_t)y * Lx;
#pragma unroll 4
    for (int p = threadIdx.x; p < Lx; p += blockDim.x) drow[p] = s[p * ps + line];
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
    // ny of the Ly rows carry data (forward input, inverse output)
    const bool half = 2 * op.ny <= Ly;
    if (INV) fft_global_inv<C>(s, tile, tile, op.py, op.twy, in, out, half);
    else fft_global_fwd<C>(s, tile, tile, op.py, op.twy, in, out, half);
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

// y pass with a radix plan P fixed at compile time (FP32, a tile of TILE
// columns): the same stages and operations as k_fft_y (bit-identical output).
template <int TILE, bool INV, class P>
__global__ void __launch_bounds__(256, 3)
k_fft_y_p(OpView<float> op, float2* __restrict__ buf, const int* __restrict__ active) {
  using C = float2;
  constexpr int L = P::L, NS = P::NS, R0 = P::radix(0), S0 = P::span(0);
  constexpr int RL = P::radix(NS - 1);
  constexpr unsigned long long DV = div_magic_c(TILE);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, ny = op.ny;
  const int col0 = blockIdx.x * TILE;
  const int ncol = min(TILE, Lx - col0);
  C* base = buf + ((int64_t)r * 3 * op.nz + blockIdx.y) * (int64_t)L * Lx + col0;
  const C* __restrict__ tw = op.twy;
  const bool half = 2 * ny <= L;
  const int64_t sstride = (int64_t)S0 * Lx;
  if (!INV) {
    // first stage (radix R0, span S0) from global memory: ny input rows
    for (int b = threadIdx.x; b < TILE * S0; b += blockDim.x) {
      const int t = b % TILE, j = b / TILE;
      const C* src = base + (int64_t)j * Lx + t;
      const bool ok = t < ncol;
      C v[R0];
      if (R0 % 2 == 0 && half) {
#pragma unroll
        for (int i = 0; i < R0 / 2; ++i)
          v[i] = (ok && j + i * S0 < ny) ? src[i * sstride] : make_float2(0.f, 0.f);
        if constexpr (R0 % 2 == 0) dft_half<R0, false, true, false>(v);
      } else {
#pragma unroll
        for (int i = 0; i < R0; ++i)
          v[i] = (ok && j + i * S0 < ny) ? src[i * sstride] : make_float2(0.f, 0.f);
        dft<R0, false>(v);
      }
      if (j > 0) {
#pragma unroll
        for (int m = 1; m < R0; ++m) v[m] = cmul(v[m], ldc(&tw[j * (R0 - 1) + (m - 1)]));
      }
#pragma unroll
      for (int m = 0; m < R0; ++m) s[(j + m * S0) * TILE + t] = v[m];
    }
    __syncthreads();
    stages_p<C, false, P, 1, NS - 2>(s, TILE, DV, TILE, tw);
    // last stage (radix RL, span 1) to global memory: all L rows
    for (int b = threadIdx.x; b < TILE * (L / RL); b += blockDim.x) {
      const int t = b % TILE, blk = b / TILE;
      C v[RL];
#pragma unroll
      for (int i = 0; i < RL; ++i) v[i] = s[(blk * RL + i) * TILE + t];
      dft<RL, false>(v);
      if (t < ncol) {
        C* dst = base + (int64_t)blk * RL * Lx + t;
#pragma unroll
        for (int m = 0; m < RL; ++m) dst[(int64_t)m * Lx] = v[m];
      }
    }
  } else {
    // first inverse stage (radix RL, span 1) from global memory: all L rows
    for (int b = threadIdx.x; b < TILE * (L / RL); b += blockDim.x) {
      const int t = b % TILE, blk = b / TILE;
      const C* src = base + (int64_t)blk * RL * Lx + t;
      const bool ok = t < ncol;
      C v[RL];
#pragma unroll
      for (int m = 0; m < RL; ++m) v[m] = ok ? src[(int64_t)m * Lx] : make_float2(0.f, 0.f);
      dft<RL, true>(v);
#pragma unroll
      for (int i = 0; i < RL; ++i) s[(blk * RL + i) * TILE + t] = v[i];
    }
    __syncthreads();
    stages_p<C, true, P, 1, NS - 2>(s, TILE, DV, TILE, tw);
    // last inverse stage (radix R0) to global memory: ny output rows
    for (int b = threadIdx.x; b < TILE * S0; b += blockDim.x) {
      const int t = b % TILE, j = b / TILE;
      C* dst = base + (int64_t)j * Lx + t;
      const bool ok = t < ncol;
      C v[R0];
#pragma unroll
      for (int m = 0; m < R0; ++m) v[m] = s[(j + m * S0) * TILE + t];
      if (j > 0) {
#pragma unroll
        for (int m = 1; m < R0; ++m) v[m] = cmulc(ldc(&tw[j * (R0 - 1) + (m - 1)]), v[m]);
      }
      if (R0 % 2 == 0 && half) {
        if constexpr (R0 % 2 == 0) dft_half<R0, true, false, true>(v);
#pragma unroll
        for (int i = 0; i < R0 / 2; ++i)
          if (ok && j + i * S0 < ny) dst[i * sstride] = v[i];
      } else {
        dft<R0, true>(v);
#pragma unroll
        for (int i = 0; i < R0; ++i)
          if (ok && j + i * S0 < ny) dst[i * sstride] = v[i];
      }
    }
  }
}

// --------------------------------------------------------------------------
// z pass: forward FFT along z, multiply by Ghat (3x3 complex symmetric),
// inverse FFT along z; the three components of a column tile in one CTA.
// grid: (column tiles, Ly, R).  Lines in shared memory: c*tile + t, row pitch ps.
// The last forward stage, the multiply and the first inverse stage run in
// registers for all three components of one butterfly.
// --------------------------------------------------------------------------
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

// The six components of Ghat at octant point o are stored together,
// ghat[6 o .. 6 o + 5] = xx, xy, xz, yy, yz, zz (48 B in FP32, 96 B in FP64).
template <typename T> struct G6;
template <> struct G6<float> {
  static __device__ __forceinline__ void load_smem(const float2* g, float2 (&v)[6]) {
    const float4* q = reinterpret_cast<const float4*>(g);
    const float4 a = q[0], b = q[1], c = q[2];
    v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
    v[4] = make_float2(c.x, c.y); v[5] = make_float2(c.z, c.w);
  }
  static __device__ __forceinline__ void load(const float2* g, float2 (&v)[6]) {
    const float4* q = reinterpret_cast<const float4*>(g);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
    v[4] = make_float2(c.x, c.y); v[5] = make_float2(c.z, c.w);
  }
};
template <> struct G6<df64> {
  static __device__ __forceinline__ void load_smem(const df64c* g, df64c (&v)[6]) {
    const float4* q = reinterpret_cast<const float4*>(g);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 a = q[i];
      v[i].x = df64(a.x, a.y);
      v[i].y = df64(a.z, a.w);
    }
  }
  static __device__ __forceinline__ void load(const df64c* g, df64c (&v)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = ldc(g + i);
  }
};
template <> struct G6<double> {
  static __device__ __forceinline__ void load_smem(const double2* g, double2 (&v)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = g[i];
  }
  static __device__ __forceinline__ void load(const double2* g, double2 (&v)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = __ldg(g + i);
  }
};

// last forward stage + multiply + first inverse stage (block = R, span 1).  A
// thread owns R consecutive positions of one column for all three components;
// it transforms each component in registers and leaves it in place, multiplies
// position by position, and transforms back -- no barrier is needed between
// these steps because no other thread touches those positions.
// w = Ghat(k) v (symmetric, components xx..zz), or w = hhat(k) x v (CROSS:
// components 0..2 hold hhat, each odd in its own axis)
template <typename T, bool CROSS>
__device__ __forceinline__ void spectral_mul(cplx_t<T> (&g)[6], bool fx, bool fy, bool fz,
                                             cplx_t<T>* w, int stride) {
  using C = cplx_t<T>;
  const C a = w[0], bb = w[stride], c = w[2 * stride];
  if (CROSS) {
    if (fx) { g[0].x = -g[0].x; g[0].y = -g[0].y; }
    if (fy) { g[1].x = -g[1].x; g[1].y = -g[1].y; }
    if (fz) { g[2].x = -g[2].x; g[2].y = -g[2].y; }
    w[0] = csub(cmul(g[1], c), cmul(g[2], bb));
    w[stride] = csub(cmul(g[2], a), cmul(g[0], c));
    w[2 * stride] = csub(cmul(g[0], bb), cmul(g[1], a));
    return;
  }
  // odd components change sign under the reflection of an odd axis
  if (fx != fy) { g[1].x = -g[1].x; g[1].y = -g[1].y; }
  if (fx != fz) { g[2].x = -g[2].x; g[2].y = -g[2].y; }
  if (fy != fz) { g[4].x = -g[4].x; g[4].y = -g[4].y; }
  w[0] = cadd(cadd(cmul(g[0], a), cmul(g[1], bb)), cmul(g[2], c));
  w[stride] = cadd(cadd(cmul(g[1], a), cmul(g[3], bb)), cmul(g[4], c));
  w[2 * stride] = cadd(cadd(cmul(g[2], a), cmul(g[4], bb)), cmul(g[5], c));
}

template <typename T, int R, int TILE, bool GS, bool CROSS>
__device__ __forceinline__ void z_mid(cplx_t<T>* s, int ps, int ncol, int col0, bool fy,
                                      int hy, const cplx_t<T>* gs, const OpView<T>& op) {
  using C = cplx_t<T>;
  const int nb = TILE * (op.Lz / R);
  const int hz_half = op.Lz >> 1;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int t = b % TILE, blk = b / TILE;
    C* q = s + (blk * R) * ps + t;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C v[R];
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = q[i * ps + c * TILE];
      dft<R, false>(v);
#pragma unroll
      for (int i = 0; i < R; ++i) q[i * ps + c * TILE] = v[i];
    }
    if (t < ncol) {
      const int kx = op.kx_at[col0 + t];
      const bool fx = kx > (op.Lx >> 1);
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int kz = op.kz_at[blk * R + i];
        const bool fz = kz > hz_half;
        const int hz = fz ? op.Lz - kz : kz;
        C g[6];
        if (GS) {
          G6<T>::load_smem(gs + 6 * (hz * TILE + t), g);
        } else {
          const int hx = fx ? op.Lx - kx : kx;
          G6<T>::load(op.ghat + 6 * (((int64_t)hz * op.Hy + hy) * op.Hx + hx), g);
        }
        spectral_mul<T, CROSS>(g, fx, fy, fz, q + i * ps, TILE);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C v[R];
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = q[i * ps + c * TILE];
      dft<R, true>(v);
#pragma unroll
      for (int i = 0; i < R; ++i) q[i * ps + c * TILE] = v[i];
    }
  }
  __syncthreads();
}

// Start copying the CTA's Ghat tile -- rows hz = 0..Lz/2 of the octant for its
// fixed ky and its TILE columns, gs[6 (hz TILE + t) + c] -- into shared memory
// with cp.async; it lands while the forward z transform runs.
template <typename T, int TILE>
__device__ __forceinline__ void ghat_tile_async(const OpView<T>& op, cplx_t<T>* gs, int col0,
                                                int ncol, int hy) {
  constexpr int CH = 6 * (int)sizeof(cplx_t<T>) / 16;  // 16-byte chunks per point
  const int n = op.Hz * TILE * CH;
  const int64_t plane = (int64_t)op.Hy * op.Hx;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int ch = e % CH, pt = e / CH;
    const int t = pt % TILE, hz = pt / TILE;
    if (t < ncol) {
      const int kx = op.kx_at[col0 + t];
      const int hx = kx > (op.Lx >> 1) ? op.Lx - kx : kx;
      const char* src = reinterpret_cast<const char*>(
          op.ghat + 6 * (hz * plane + (int64_t)hy * op.Hx + hx)) + 16 * ch;
      char* dst = reinterpret_cast<char*>(gs + 6 * (hz * TILE + t)) + 16 * ch;
      cp_async<16>(dst, src);
    }
  }
  cp_async_commit();
}

// grid: (column tiles, Ly, R).  Shared memory: Lz x ps, lines c * TILE + t,
// then (GS) the Ghat tile (16-byte aligned); without GS the multiply reads
// Ghat from global memory (long z lines, where the tile would not fit).
template <typename T, int TILE, bool GS, bool CROSS = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_fft_z_mul(OpView<T> op, cplx_t<T>* __restrict__ buf, int ps, const int* __restrict__ active) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, Ly = op.Ly, Lz = op.Lz, nz = op.nz;
  const int pyy = blockIdx.y;
  const int ky = op.ky_at[pyy];
  const bool fy = ky > (Ly >> 1);
  const int hy = fy ? Ly - ky : ky;
  const int col0 = blockIdx.x * TILE;
  const int ncol = min(TILE, Lx - col0);
  constexpr int NL = 3 * TILE;
  const int64_t plane_sz = (int64_t)Ly * Lx;
  const int64_t comp_sz = (int64_t)nz * plane_sz;
  C* base = buf + (int64_t)r * 3 * comp_sz + (int64_t)pyy * Lx + col0;
  ZIO<C> io{base, comp_sz, plane_sz, TILE, ncol, nz};
  C* gs = reinterpret_cast<C*>(smem_raw + (((size_t)Lz * ps * sizeof(C) + 15) & ~(size_t)15));
  if (GS) ghat_tile_async<T, TILE>(op, gs, col0, ncol, hy);
  const AxisPlan& P = op.pz;
  const int last = P.nstage - 1;
  if (P.nstage >= 2) {
    DDA_RADIX_DISPATCH(P.radix[0], (stage_first_fwd<C, RR>(s, NL, ps, Lz, op.twz, io,
                                                          2 * nz <= Lz)));
    fft_inner_stages<C, false>(s, NL, ps, P, op.twz);
  } else {
    for (int e = threadIdx.x; e < Lz * NL; e += blockDim.x) {
      const int p = e / NL, l = e - p * NL;
      s[p * ps + l] = io(l, p);
    }
  }
  if (GS) cp_async_wait_all();
  __syncthreads();
  if (P.nstage >= 1) {
    // the plan puts a radix <= 8 last
    DDA_RADIX_DISPATCH_SMALL(P.radix[last],
                             (z_mid<T, RR, TILE, GS, CROSS>(s, ps, ncol, col0, fy, hy, gs, op)));
  } else {  // Lz = 1: multiply only
    for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
      const int kx = op.kx_at[col0 + t];
      const bool fx = kx > (Lx >> 1);
      C g[6];
      if (GS) G6<T>::load_smem(gs + 6 * t, g);
      else G6<T>::load(op.ghat + 6 * ((int64_t)hy * op.Hx + (fx ? Lx - kx : kx)), g);
      spectral_mul<T, CROSS>(g, fx, fy, false, s + t, TILE);
    }
    __syncthreads();
  }
  if (P.nstage >= 2) {
    fft_inner_stages<C, true>(s, NL, ps, P, op.twz);
    DDA_RADIX_DISPATCH(P.radix[0], (stage_last_inv<C, RR>(s, NL, ps, Lz, op.twz, io,
                                                         2 * nz <= Lz)));
  } else {
    for (int e = threadIdx.x; e < Lz * NL; e += blockDim.x) {
      const int p = e / NL, l = e - p * NL;
      io(l, p, s[p * ps + l]);
    }
  }
}

// --------------------------------------------------------------------------
// z pass with a radix plan P fixed at compile time (FP32).  It runs the same
// stages, twiddles, multiply and operations in the same order as k_fft_z_mul
// (the product is bit-identical); the shared-memory pitch, strides, loop
// bounds and the frequency at each digit-reversed position (P::k_at) become
// constants, which takes the index arithmetic out of the issue-bound loop and
// leaves a smaller kernel (one plan, no radix dispatch) for the instruction
// cache.
// --------------------------------------------------------------------------
template <int TILE> constexpr int zc_pitch() { return 3 * TILE + (TILE * 8 < 128 ? 1 : 0); }

// Up to 384 threads (the same 85-register budget as 3 x 256): long lines
// (three or more stages) stage a Ghat tile big enough to leave only two CTAs
// per SM, and more threads per CTA keep the stages' butterfly counts busy.
template <int TILE, bool GS, class P>
__global__ void __launch_bounds__(384, 2)
k_fft_z_mul_p(OpView<float> op, float2* __restrict__ buf, const int* __restrict__ active) {
  using C = float2;
  constexpr int L = P::L, NS = P::NS, R0 = P::radix(0), S0 = P::span(0);
  constexpr int RL = P::radix(NS - 1), NL = 3 * TILE, PS = zc_pitch<TILE>();
  constexpr unsigned long long DV = div_magic_c(NL);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int Lx = op.Lx, Ly = op.Ly, nz = op.nz;
  const int pyy = blockIdx.y;
  const int ky = op.ky_at[pyy];
  const bool fy = ky > (Ly >> 1);
  const int hy = fy ? Ly - ky : ky;
  const int col0 = blockIdx.x * TILE;
  const int ncol = min(TILE, Lx - col0);
  const int64_t plane_sz = (int64_t)Ly * Lx;
  const int64_t comp_sz = (int64_t)nz * plane_sz;
  C* base = buf + (int64_t)r * 3 * comp_sz + (int64_t)pyy * Lx + col0;
  C* gs = reinterpret_cast<C*>(smem_raw + (((size_t)L * PS * sizeof(C) + 15) & ~(size_t)15));
  if (GS) ghat_tile_async<float, TILE>(op, gs, col0, ncol, hy);
  const C* __restrict__ tw = op.twz;
  const bool half = 2 * nz <= L;
  const int64_t sstride = (int64_t)S0 * plane_sz;  // global distance of one butterfly input
  // first forward stage (radix R0, span S0), read straight from global memory
  for (int b = threadIdx.x; b < NL * S0; b += blockDim.x) {
    const int line = b % NL, j = b / NL;
    const int c = line / TILE, t = line - c * TILE;
    const C* src = base + c * comp_sz + (int64_t)j * plane_sz + t;
    const bool ok = t < ncol;
    C v[R0];
    if (R0 % 2 == 0 && half) {
#pragma unroll
      for (int i = 0; i < R0 / 2; ++i)
        v[i] = (ok && j + i * S0 < nz) ? src[i * sstride] : make_float2(0.f, 0.f);
      if constexpr (R0 % 2 == 0) dft_half<R0, false, true, false>(v);
    } else {
#pragma unroll
      for (int i = 0; i < R0; ++i)
        v[i] = (ok && j + i * S0 < nz) ? src[i * sstride] : make_float2(0.f, 0.f);
      dft<R0, false>(v);
    }
    if (j > 0) {
#pragma unroll
      for (int m = 1; m < R0; ++m) v[m] = cmul(v[m], ldc(&tw[j * (R0 - 1) + (m - 1)]));
    }
#pragma unroll
    for (int m = 0; m < R0; ++m) s[(j + m * S0) * PS + line] = v[m];
  }
  if constexpr (NS > 2) {
    __syncthreads();
    stages_p<C, false, P, 1, NS - 2>(s, NL, DV, PS, tw);
  }
  if (GS) cp_async_wait_all();
  __syncthreads();
  // last forward stage + multiply + first inverse stage (radix RL, span 1):
  // a thread owns RL consecutive positions of one column, all three components
  {
    const int kxh = Lx >> 1;
    for (int b = threadIdx.x; b < TILE * (L / RL); b += blockDim.x) {
      const int t = b % TILE, blk = b / TILE;
      C* q = s + blk * RL * PS + t;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C v[RL];
#pragma unroll
        for (int i = 0; i < RL; ++i) v[i] = q[i * PS + c * TILE];
        dft<RL, false>(v);
#pragma unroll
        for (int i = 0; i < RL; ++i) q[i * PS + c * TILE] = v[i];
      }
      if (t < ncol) {
        const int kx = op.kx_at[col0 + t];
        const bool fx = kx > kxh;
#pragma unroll
        for (int i = 0; i < RL; ++i) {
          const int kz = P::k_at(blk * RL + i);
          const bool fz = kz > L / 2;
          const int hz = fz ? L - kz : kz;
          C g[6];
          if (GS) {
            G6<float>::load_smem(gs + 6 * (hz * TILE + t), g);
          } else {
            const int hx = fx ? Lx - kx : kx;
            G6<float>::load(op.ghat + 6 * (((int64_t)hz * op.Hy + hy) * op.Hx + hx), g);
          }
          spectral_mul<float, false>(g, fx, fy, fz, q + i * PS, TILE);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C v[RL];
#pragma unroll
        for (int i = 0; i < RL; ++i) v[i] = q[i * PS + c * TILE];
        dft<RL, true>(v);
#pragma unroll
        for (int i = 0; i < RL; ++i) q[i * PS + c * TILE] = v[i];
      }
    }
  }
  __syncthreads();
  if constexpr (NS > 2) stages_p<C, true, P, 1, NS - 2>(s, NL, DV, PS, tw);
  // last inverse stage (radix R0), written straight to global memory
  for (int b = threadIdx.x; b < NL * S0; b += blockDim.x) {
    const int line = b % NL, j = b / NL;
    const int c = line / TILE, t = line - c * TILE;
    C* dst = base + c * comp_sz + (int64_t)j * plane_sz + t;
    const bool ok = t < ncol;
    C v[R0];
#pragma unroll
    for (int m = 0; m < R0; ++m) v[m] = s[(j + m * S0) * PS + line];
    if (j > 0) {
#pragma unroll
      for (int m = 1; m < R0; ++m) v[m] = cmulc(ldc(&tw[j * (R0 - 1) + (m - 1)]), v[m]);
    }
    if (R0 % 2 == 0 && half) {
      if constexpr (R0 % 2 == 0) dft_half<R0, true, false, true>(v);
#pragma unroll
      for (int i = 0; i < R0 / 2; ++i)
        if (ok && j + i * S0 < nz) dst[i * sstride] = v[i];
    } else {
      dft<R0, true>(v);
#pragma unroll
      for (int i = 0; i < R0; ++i)
        if (ok && j + i * S0 < nz) dst[i * sstride] = v[i];
    }
  }
}

template <int TILE, bool GS>
static size_t zp_smem(const OpView<float>& op) {
  const size_t d = ((size_t)op.Lz * zc_pitch<TILE>() * sizeof(float2) + 15) & ~(size_t)15;
  return d + (GS ? (size_t)6 * op.Hz * TILE * sizeof(float2) : 0);
}

// FP32 passes with a compiled radix plan (matvec_fixed.cu).  Each returns
// false, launching nothing, when no compiled variant matches the axis plan
// and the schedule's tile.
bool launch_y_fixed(bool inv, const OpView<float>& op, const MatvecLaunch& L, int R,
                    float2* scratch, const int* active, cudaStream_t st);
bool launch_z_fixed(const OpView<float>& op, const MatvecLaunch& L, int R, float2* scratch,
                    const int* active, cudaStream_t st);
bool z_fixed_plan(const AxisPlan& P);
template <int XIN>
bool launch_x_fwd_fixed(const OpView<float>& op, const MatvecLaunch& L, int R, const float2* x,
                        float2* scratch, const int* active, XinArgs<float> xa, cudaStream_t st);
template <int XOUT>
bool launch_x_inv_fixed(const OpView<float>& op, const MatvecLaunch& L, int R,
                        const float2* scratch, const float2* x, float2* y, const int* active,
                        const float2* rhat, double* partials, cudaStream_t st, FoldArgs fold);
cudaError_t configure_fixed_kernels();

// One y pass (forward: ny -> Ly rows, inverse: Ly -> ny rows) with the
// schedule's tile (a compiled radix plan where one matches).
template <typename T, bool INV>
static void launch_y_pass(const OpView<T>& op, const MatvecLaunch& L, int R,
                          cplx_t<T>* scratch, const int* active, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (launch_y_fixed(INV, op, L, R, scratch, active, st)) return;
  }
  dim3 gy((op.Lx + L.y_tile - 1) / L.y_tile, 3 * op.nz, R);
  k_fft_y<T, INV><<<gy, L.y_threads, L.y_smem, st>>>(op, scratch, L.y_tile, active);
}

// One z pass (forward z, multiply, inverse z) with the schedule's tile.
template <typename T, bool CROSS>
static void launch_z_pass(const OpView<T>& op, const MatvecLaunch& L, int R,
                          cplx_t<T>* scratch, const int* active, cudaStream_t st) {
  if constexpr (std::is_same<T, df64>::value) {
    // double-float passes use one z variant (4 columns, Ghat from global
    // memory): the arithmetic is ~10x the FP32 code, so fewer instantiations
    // keep the build short
    dim3 gz((op.Lx + 3) / 4, op.Ly, R);
    k_fft_z_mul<T, 4, false, CROSS><<<gz, L.z_threads, L.z_smem, st>>>(op, scratch, L.z_ps,
                                                                      active);
  } else {
    dim3 gz((op.Lx + L.z_tile - 1) / L.z_tile, op.Ly, R);
    if constexpr (std::is_same<T, float>::value && !CROSS) {
      if (launch_z_fixed(op, L, R, scratch, active, st)) return;
    }
#define DDA_ZL(TT, GG) \
  k_fft_z_mul<T, TT, GG, CROSS><<<gz, L.z_threads, L.z_smem, st>>>(op, scratch, L.z_ps, active)
    if (L.z_gs) {
      switch (L.z_tile) {
        case 16: DDA_ZL(16, true); break;
        case 8: DDA_ZL(8, true); break;
        case 4: DDA_ZL(4, true); break;
        default: DDA_ZL(2, true); break;
      }
    } else {
      switch (L.z_tile) {
        case 16: DDA_ZL(16, false); break;
        case 8: DDA_ZL(8, false); break;
        case 4: DDA_ZL(4, false); break;
        default: DDA_ZL(2, false); break;
      }
    }
#undef DDA_ZL
  }
}

// --------------------------------------------------------------------------
// x pass, inverse + diagonal term: y = ainv * x - conv on occupied sites
// grid: (row tiles, R)
// --------------------------------------------------------------------------
// Epilogue of the last pass, fused with the Krylov inner products (block sums
// as in ChunkAcc, FP64 per-block partials [R][gridDim.x][NV]; with a FoldArgs
// the last block of each RHS row also runs the scalar step those sums feed):
//   XOUT_PLAIN : none;
//   XOUT_RV    : <rhat, y>              (y = v = A p)
//   XOUT_TS    : <y, x>, <y, y>         (y = t = A s, x = s)
//   XOUT_QT    : x^T y, unconjugated    (y = t = A q, x = q; QMR)
//   XOUT_FIELD : y = sum_{l != j} G_jl x_l on EVERY box site, occupied or
//                not (the field the dipoles radiate; near-field output)
enum { XOUT_PLAIN = 0, XOUT_RV = 1, XOUT_TS = 2, XOUT_QT = 3, XOUT_FIELD = 4 };

template <typename T, int MODE, class P = void>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_fft_x_inv(OpView<T> op, const cplx_t<T>* __restrict__ buf,
                            const io_t<T>* __restrict__ xin, io_t<T>* __restrict__ yout,
                            int nlines, unsigned long long div_nl, const int* __restrict__ active,
                            const io_t<T>* __restrict__ rhat, double* __restrict__ partials,
                            FoldArgs fold) {
  using C = cplx_t<T>;
  constexpr int LP = plan_len<P>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int nx = op.nx, Lx = LP ? LP : op.Lx;
  const int rows = 3 * op.nz * op.ny;
  const int row0 = blockIdx.x * nlines;
  const int ps = nlines + 1;
  const int64_t plane_sz = (int64_t)op.Ly * Lx;
  const C* src = buf + (int64_t)r * 3 * op.nz * plane_sz;
  // the epilogue's inputs (x, and rhat for XOUT_RV) are contiguous chunks of the
  // box vectors: start copying them now, behind the spectral rows
  // (box-vector elements: FP64 for df64 passes, same size as C)
  using IO = io_t<T>;
  static_assert(sizeof(IO) == sizeof(C), "box and FFT elements must have one size");
  IO* sx = reinterpret_cast<IO*>(s + (size_t)Lx * ps);
  IO* sh = sx + (size_t)nlines * nx;
  // the composition bytes of the CTA's sites (lines of nx bytes)
  unsigned char* scm = reinterpret_cast<unsigned char*>(sh + (size_t)nlines * nx);
  const int nin = min(nlines, rows - row0) * nx;
  const int64_t g0 = ((int64_t)r * rows + row0) * nx;
  for (int e = threadIdx.x; e < nin; e += blockDim.x) {
    cp_async<(int)sizeof(IO)>(&sx[e], &xin[g0 + e]);
    if (MODE == XOUT_RV) cp_async<(int)sizeof(IO)>(&sh[e], &rhat[g0 + e]);
  }
  // the epilogue's alpha^{-1} entries (3 per composition), when few
  constexpr int kAiSmem = 24;
  __shared__ C sai[kAiSmem];
  const bool ai_smem = op.ncomp1 * 3 <= kAiSmem;
  const C* ai = op.ainv + (int64_t)r * op.ncomp1 * 3;
  if (MODE != XOUT_FIELD && ai_smem)
    for (int i = threadIdx.x; i < op.ncomp1 * 3; i += blockDim.x) sai[i] = ai[i];
  // all of the tile's loads in flight at once (asynchronous copies, the
  // composition bytes in 4-byte pieces when lines are whole words); the row's
  // plane and y are worked out once per line.  Each line's site information
  // for the epilogue (composition row, polarization component) goes to a
  // small table (at most 64 lines per CTA).
  __shared__ int line_site[64], line_comp[64];
  const bool cm_words = (nx & 3) == 0;
  for (int line = 0; line < nlines; ++line) {
    const int row = row0 + line;
    if (row < rows) {
      const int plane = fast_div(row, op.div_ny), y = row - plane * op.ny;
      const C* srow = src + plane * plane_sz + (int64_t)y * Lx;
      for (int p = threadIdx.x; p < Lx; p += blockDim.x)
        cp_async<(int)sizeof(C)>(&s[p * ps + line], &srow[p]);
      // row = (c nz + z) ny + y  ->  sites (z ny + y) nx + p
      const int c = fast_div(plane, op.div_nz);
      const int site = ((plane - c * op.nz) * op.ny + y) * nx;
      if (MODE != XOUT_FIELD) {
        if (cm_words) {
          for (int p = 4 * threadIdx.x; p < nx; p += 4 * blockDim.x)
            cp_async<4>(&scm[line * nx + p], &op.comp[site + p]);
        } else {
          for (int p = threadIdx.x; p < nx; p += blockDim.x) scm[line * nx + p] = op.comp[site + p];
        }
      }
      if (threadIdx.x == 0) {
        line_site[line] = site;
        line_comp[line] = c;
      }
    } else {
      for (int p = threadIdx.x; p < Lx; p += blockDim.x) s[p * ps + line] = mk<C>(0, 0);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  // only positions < nx <= Lx/2 are used below
  if constexpr (std::is_void<P>::value) fft_smem<C, true>(s, nlines, ps, op.px, op.twx, 2 * nx <= Lx);
  else fft_smem_p<C, true, P>(s, nlines, div_nl, ps, op.twx, 2 * nx <= Lx);
  const C* aiv = ai_smem ? sai : ai;
  IO* yr = yout + g0;
  // (df64 passes only run the plain epilogue; their accumulator type is unused)
  ChunkAcc<std::conditional_t<std::is_same<T, df64>::value, double, T>, 4> acc;
  // batches of U elements per thread: the composition bytes of a batch are
  // read before any output is stored (a byte pointer may alias the output,
  // which would otherwise serialise every element's load behind the previous
  // element's store)
  constexpr int U = 4;
  for (int e0 = threadIdx.x; e0 < nin; e0 += U * blockDim.x) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int e = e0 + u * blockDim.x;
    if (e >= nin) break;
    const int line = fast_div(e, op.div_nx), p = e - line * nx;
    // the alpha^{-1} entry of composition cm on axis c is 3 cm + c (0: vacant)
    int cm = 0;
    if (MODE != XOUT_FIELD) {
      cm = scm[e];
      cm = cm ? 3 * cm + line_comp[line] : 0;
    }
    C out = mk<C>(0, 0);
    const C xv = from_io<C>(sx[e]);
    if (MODE == XOUT_FIELD) out = s[p * ps + line];
    else if (cm) out = csub(cmul(aiv[cm], xv), s[p * ps + line]);
    yr[e] = to_io<IO>(out);
    {
      if constexpr (MODE == XOUT_RV) {
        const C h = from_io<C>(sh[e]);
        acc.add(0, h.x * out.x + h.y * out.y);
        acc.add(1, h.x * out.y - h.y * out.x);
        acc.step();
      } else if constexpr (MODE == XOUT_TS) {
        acc.add(0, out.x * xv.x + out.y * xv.y);
        acc.add(1, out.x * xv.y - out.y * xv.x);
        acc.add(2, out.x * out.x + out.y * out.y);
        acc.step();
      } else if constexpr (MODE == XOUT_QT) {
        acc.add(0, xv.x * out.x - xv.y * out.y);
        acc.add(1, xv.x * out.y + xv.y * out.x);
        acc.step();
      }
    }
  }
  }
  if constexpr (MODE != XOUT_PLAIN && MODE != XOUT_FIELD) {
    if constexpr (MODE == XOUT_RV || MODE == XOUT_QT) {
      acc.template write<2>(partials);
      if (fold.counter) fold_scalar_step<2>(partials, fold);
    } else {
      acc.template write<4>(partials);
      if (fold.counter) fold_scalar_step<4>(partials, fold);
    }
  }
}

static inline unsigned long long div_magic(int d) {
  return ((1ull << 36) + (unsigned long long)d - 1) / (unsigned long long)d;
}

// One forward x pass (prologue mode XIN) with the schedule's line count (a
// compiled radix plan where one matches).
template <typename T, int XIN>
static void launch_x_fwd_pass(const OpView<T>& op, const MatvecLaunch& L, int R,
                              const io_t<T>* x, cplx_t<T>* scratch, const int* active,
                              XinArgs<T> xa, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (launch_x_fwd_fixed<XIN>(op, L, R, x, scratch, active, xa, st)) return;
  }
  const int rows = 3 * op.nz * op.ny;
  dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
  k_fft_x_fwd<T, XIN><<<gx, L.x_threads, L.x_smem, st>>>(op, x, scratch, L.x_lines,
                                                         div_magic(L.x_lines), active, xa);
}

// One inverse x pass (epilogue mode XOUT) with the schedule's line count.
template <typename T, int XOUT>
static void launch_x_inv_pass(const OpView<T>& op, const MatvecLaunch& L, int R,
                              const cplx_t<T>* scratch, const io_t<T>* x, io_t<T>* y,
                              const int* active, const io_t<T>* rhat, double* partials,
                              cudaStream_t st, FoldArgs fold = FoldArgs()) {
  if constexpr (std::is_same<T, float>::value && XOUT != XOUT_FIELD) {
    if (launch_x_inv_fixed<XOUT>(op, L, R, scratch, x, y, active, rhat, partials, st, fold))
      return;
  }
  const int rows = 3 * op.nz * op.ny;
  dim3 gx((rows + L.x_lines - 1) / L.x_lines, R);
  k_fft_x_inv<T, XOUT><<<gx, L.x_threads, L.xinv_smem, st>>>(op, scratch, x, y, L.x_lines,
                                                             div_magic(L.x_lines), active, rhat,
                                                             partials, fold);
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
  while (nl > 1 && (size_t)nl * (op.Lx + 1) * sizeof(C) > 36 * 1024) nl >>= 1;
  while (nl < 64 && (size_t)(2 * nl) * (op.Lx + 1) * sizeof(C) <= 36 * 1024) nl <<= 1;
  L.x_lines = nl;
  L.x_threads = 256;
  L.x_smem = (size_t)op.Lx * (nl + 1) * sizeof(C);
  L.xinv_smem = x_inv_smem_bytes(op.Lx, nl, op.nx, sizeof(C));  // + x, rhat, composition
  // y pass: a tile of 128 B of columns (16 FP32 / 8 FP64 complex), 256 threads
  int ty = 128 / (int)sizeof(C);
  while (ty > 2 && (size_t)ty * op.Ly * sizeof(C) > 64 * 1024) ty >>= 1;
  L.y_tile = ty;
  L.y_threads = 256;
  L.y_smem = (size_t)op.Ly * ty * sizeof(C);
  // z pass: three components of a tile of 64 B of columns plus the tile's Ghat
  // rows (octant, 6 components) staged in shared memory, halved while the CTA
  // would need more than 64 KB -- but not below 64 B rows: long z lines keep
  // 64 B rows and read Ghat from global memory instead.  The row pitch is made
  // odd when the tile is narrower than a half-warp's 128 B so that the
  // butterflies of neighbouring blocks fall on different banks.
  const int tz_min = 64 / (int)sizeof(C);
  auto pitch = [&](int tt) { return 3 * tt + (tt * (int)sizeof(C) < 128 ? 1 : 0); };
  auto zbytes = [&](int tt, bool gsm) {
    const size_t d = ((size_t)op.Lz * pitch(tt) * sizeof(C) + 15) & ~(size_t)15;
    return d + (gsm ? (size_t)6 * op.Hz * tt * sizeof(C) : 0);
  };
  int tz = tz_min;
  L.z_gs = zbytes(tz, true) <= 64 * 1024;
  if (!L.z_gs)
    while (tz > 2 && zbytes(tz, false) > 104 * 1024) tz >>= 1;
  L.z_tile = tz;
  L.z_ps = pitch(tz);
  L.z_smem = zbytes(tz, L.z_gs);
  L.z_threads = 256;
  return L;
}

template <typename T>
cudaError_t configure_matvec_kernels(const MatvecLaunch& L) {
  (void)L;
  cudaError_t e;
  const void* xk[] = {(const void*)k_fft_x_fwd<T, XIN_PLAIN>, (const void*)k_fft_x_fwd<T, XIN_P>,
                      (const void*)k_fft_x_fwd<T, XIN_S>, (const void*)k_fft_x_fwd<T, XIN_Q>,
                      (const void*)k_fft_x_inv<T, XOUT_PLAIN>, (const void*)k_fft_x_inv<T, XOUT_RV>,
                      (const void*)k_fft_x_inv<T, XOUT_TS>, (const void*)k_fft_x_inv<T, XOUT_QT>,
                      (const void*)k_fft_x_inv<T, XOUT_FIELD>};
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
  const void* zk[] = {(const void*)k_fft_z_mul<T, 16, true>, (const void*)k_fft_z_mul<T, 8, true>,
                      (const void*)k_fft_z_mul<T, 4, true>, (const void*)k_fft_z_mul<T, 2, true>,
                      (const void*)k_fft_z_mul<T, 16, false>, (const void*)k_fft_z_mul<T, 8, false>,
                      (const void*)k_fft_z_mul<T, 4, false>, (const void*)k_fft_z_mul<T, 2, false>};
  for (const void* k : zk) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  if constexpr (std::is_same<T, float>::value) {
    e = configure_fixed_kernels();
    if (e != cudaSuccess) return e;
  }
  if constexpr (sizeof(T) == 8) {  // magnetic near field (FP64 only)
    const void* zc[] = {(const void*)k_fft_z_mul<T, 16, true, true>,
                        (const void*)k_fft_z_mul<T, 8, true, true>,
                        (const void*)k_fft_z_mul<T, 4, true, true>,
                        (const void*)k_fft_z_mul<T, 2, true, true>,
                        (const void*)k_fft_z_mul<T, 16, false, true>,
                        (const void*)k_fft_z_mul<T, 8, false, true>,
                        (const void*)k_fft_z_mul<T, 4, false, true>,
                        (const void*)k_fft_z_mul<T, 2, false, true>};
    for (const void* k : zc) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return e;
    }
  }
  return e;
}

template <typename T, int XIN, int XOUT, bool CROSS = false>
static cudaError_t matvec_passes(const OpView<T>& op, const MatvecLaunch& L, int R,
                                 const io_t<T>* x, io_t<T>* y, cplx_t<T>* scratch,
                                 const int* active, cudaStream_t st, const cudaEvent_t* ev,
                                 XinArgs<T> xa, const io_t<T>* rhat, double* partials,
                                 FoldArgs fold = FoldArgs()) {
  // inside a stream capture the events must be external nodes to be recorded
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (ev) cudaStreamIsCapturing(st, &cap);
  auto record = [&](cudaEvent_t e) {
    if (cap == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  };
  if (ev) record(ev[0]);
  launch_x_fwd_pass<T, XIN>(op, L, R, x, scratch, active, xa, st);
  note_launch();
  if (ev) record(ev[1]);
  launch_y_pass<T, false>(op, L, R, scratch, active, st);
  note_launch();
  if (ev) record(ev[2]);
  launch_z_pass<T, CROSS>(op, L, R, scratch, active, st);
  note_launch();
  if (ev) record(ev[3]);
  launch_y_pass<T, true>(op, L, R, scratch, active, st);
  note_launch();
  if (ev) record(ev[4]);
  launch_x_inv_pass<T, XOUT>(op, L, R, scratch, x, y, active, rhat, partials, st, fold);
  note_launch();
  if (ev) record(ev[5]);
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
cudaError_t launch_field(const OpView<T>& op, const MatvecLaunch& L, int R,
                         const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch,
                         cudaStream_t st, bool magnetic) {
  if (magnetic)
    return matvec_passes<T, XIN_PLAIN, XOUT_FIELD, true>(op, L, R, x, y, scratch, nullptr, st,
                                                         nullptr, XinArgs<T>{}, nullptr,
                                                         nullptr);
  return matvec_passes<T, XIN_PLAIN, XOUT_FIELD>(op, L, R, x, y, scratch, nullptr, st,
                                                 nullptr, XinArgs<T>{}, nullptr, nullptr);
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
                            const cudaEvent_t* ev, FoldArgs fold) {
  XinArgs<T> xa{r, p, v, ks};
  return matvec_passes<T, XIN_P, XOUT_RV>(op, L, R, p, v, scratch, active, st, ev, xa, rhat,
                                          partials, fold);
}

template <typename T>
cudaError_t launch_matvec_s(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, const cplx_t<T>* v, cplx_t<T>* s_vec,
                            cplx_t<T>* t_vec, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev, FoldArgs fold) {
  XinArgs<T> xa{r, s_vec, v, ks};
  return matvec_passes<T, XIN_S, XOUT_TS>(op, L, R, s_vec, t_vec, scratch, active, st, ev, xa,
                                          nullptr, partials, fold);
}

template <typename T>
cudaError_t launch_matvec_rv(const OpView<T>& op, const MatvecLaunch& L, int R,
                             const cplx_t<T>* x, cplx_t<T>* y, const cplx_t<T>* rhat,
                             cplx_t<T>* scratch, double* partials, const int* active,
                             cudaStream_t st, const cudaEvent_t* ev) {
  return matvec_passes<T, XIN_PLAIN, XOUT_RV>(op, L, R, x, y, scratch, active, st, ev,
                                              XinArgs<T>{}, rhat, partials);
}

template <typename T>
cudaError_t launch_matvec_q(const OpView<T>& op, const MatvecLaunch& L, int R,
                            const cplx_t<T>* r, cplx_t<T>* q, cplx_t<T>* d, cplx_t<T>* x,
                            cplx_t<T>* t_vec, cplx_t<T>* scratch, const KState* ks,
                            double* partials, const int* active, cudaStream_t st,
                            const cudaEvent_t* ev, FoldArgs fold) {
  XinArgs<T> xa{r, q, nullptr, ks, d, x};
  return matvec_passes<T, XIN_Q, XOUT_QT>(op, L, R, q, t_vec, scratch, active, st, ev, xa,
                                          nullptr, partials, fold);
}

template <typename T>
cudaError_t launch_x_fwd(const OpView<T>& op, const MatvecLaunch& L, int R,
                         const cplx_t<T>* x, cplx_t<T>* out, cudaStream_t st) {
  launch_x_fwd_pass<T, XIN_PLAIN>(op, L, R, x, out, nullptr, XinArgs<T>{}, st);
  note_launch();
  return cudaGetLastError();
}

}  // namespace dda
