// z pass on column pairs (FP32, the kernel's own radix plan P of the z length,
// radices of at most 8, fixed at compile time, and NT threads per CTA).
//
// The same arithmetic as k_fft_z_mul_p -- forward FFT along z, the 3x3
// complex-symmetric multiply by Ghat, inverse FFT along z, for the three
// polarization components of each column -- with the work laid out for fewer
// instructions per point and for reuse of Ghat:
//   * a thread always works on two neighbouring columns at once: shared memory
//     holds a pair as one float4 (16-byte loads and stores, every twiddle
//     loaded once for both columns, half the index arithmetic), and rows are
//     stored without padding so that consecutive threads touch consecutive
//     16-byte words;
//   * a CTA owns TILE columns at one octant row hy and runs both rows that
//     share it (ky = hy and ky = Ly - hy) for every right-hand side, so every
//     pass of the CTA reads the same Ghat rows: from L2 after the first (GS =
//     false), or staged once in shared memory with cp.async while the first
//     forward transform runs (GS = true);
//   * the last forward stage, the multiply and the first inverse stage are
//     separate sweeps over shared memory (each conflict-free for this layout).
// The plan P (e.g. 512 = 8 x 8 x 8) need not be the target's z plan: the z
// transform starts and ends inside this kernel, so only the frequency held at
// each position (P::k_at, for the multiply) and P's twiddle table (op.twz_pair)
// matter.  Small radices keep the registers low enough for two CTAs of NT
// threads per SM, and NT is a multiple of the pair-lines per row so every
// thread keeps one pair-line for the whole kernel (no index division in the
// loops).  The arithmetic is the same transform with another factorization,
// so results agree with the other z kernels to rounding, not bit for bit.
//
// grid: (ceil(Lx / TILE), Ly / 2 + 1), any block size.  Needs Lx even (pairs
// of columns are 16-byte aligned).  Shared memory: Lz * 3 * TILE/2 float4,
// plus (GS) the Ghat tile, (Lz/2 + 1) * TILE * 6 float2.
#pragma once

#include "matvec_impl.cuh"

namespace dda {

__device__ __forceinline__ void split4(const float4 q, float2& a, float2& b) {
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}

// One in-place stage ST of plan P on NU pair-lines of shared memory, both
// columns of each pair (forward: DFT then twiddles; inverse: the adjoint).
template <bool INV, class P, int ST, int NU, int NT>
__device__ __forceinline__ void stage_pair(float4* sd, const float2* __restrict__ tw) {
  constexpr int R = P::radix(ST), B = P::block(ST), S = P::span(ST), NB = P::L / R;
  static_assert(NT % NU == 0, "a thread keeps one pair-line");
  const float2* __restrict__ tws = tw + P::tw_off(ST);
  const int u = threadIdx.x % NU;
  for (int q = threadIdx.x / NU; q < NB; q += NT / NU) {
    const int blk = q / S, j = q - blk * S;
    float4* base = sd + (blk * B + j) * NU + u;
    float2 va[R], vb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) split4(base[i * S * NU], va[i], vb[i]);
    if constexpr (!INV) {
      dft<R, false>(va);
      dft<R, false>(vb);
      if (S > 1 && j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          const float2 w = ldc(&tws[j * (R - 1) + (m - 1)]);
          va[m] = cmul(va[m], w);
          vb[m] = cmul(vb[m], w);
        }
      }
    } else {
      if (S > 1 && j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          const float2 w = ldc(&tws[j * (R - 1) + (m - 1)]);
          va[m] = cmulc(w, va[m]);
          vb[m] = cmulc(w, vb[m]);
        }
      }
      dft<R, true>(va);
      dft<R, true>(vb);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) base[i * S * NU] = make_float4(va[i].x, va[i].y, vb[i].x, vb[i].y);
  }
  __syncthreads();
}

// Stages LO..HI forward (ascending) or inverse (descending).
template <bool INV, class P, int LO, int HI, int NU, int NT>
__device__ __forceinline__ void stages_pair(float4* sd, const float2* __restrict__ tw) {
  if constexpr (LO <= HI) {
    if constexpr (!INV) {
      stage_pair<false, P, LO, NU, NT>(sd, tw);
      stages_pair<false, P, LO + 1, HI, NU, NT>(sd, tw);
    } else {
      stage_pair<true, P, HI, NU, NT>(sd, tw);
      stages_pair<true, P, LO, HI - 1, NU, NT>(sd, tw);
    }
  }
}

template <int TILE, class P, bool GS, int NT>
__global__ void __launch_bounds__(NT, 2)
k_fft_z_pairs(OpView<float> op, float2* __restrict__ buf, int R, const int* __restrict__ active) {
  static_assert(TILE % 2 == 0, "column pairs");
  constexpr int L = P::L, NS = P::NS, R0 = P::radix(0), S0 = P::span(0);
  constexpr int NP = TILE / 2, NU = 3 * NP;
  static_assert(NT % NU == 0 && NT % NP == 0, "a thread keeps one pair-line");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sd = reinterpret_cast<float4*>(smem_raw);
  float2* gs = reinterpret_cast<float2*>(sd + L * NU);
  const int Lx = op.Lx, Ly = op.Ly, nz = op.nz;
  const int hy = blockIdx.y;
  const int col0 = blockIdx.x * TILE;
  const int npv = min(TILE, Lx - col0) >> 1;  // pairs inside the grid (Lx even)
  if (GS) ghat_tile_async<float, TILE>(op, gs, col0, 2 * npv, hy);
  const int64_t plane_sz = (int64_t)Ly * Lx;
  const int64_t comp_sz = (int64_t)nz * plane_sz;
  const bool half = 2 * nz <= L;
  const float2* __restrict__ tw = op.twz_pair;
  const int kxh = Lx >> 1;
  const int u = threadIdx.x % NU;           // this thread's pair-line ...
  const int c = u / NP, tp = u - c * NP;    // ... = component c, column pair tp
  const int tpm = threadIdx.x % NP;         // its column pair in the multiply
  // the rows sharing octant row hy: ky = hy, and ky = Ly - hy unless that is hy
  const int nrow = (hy == 0 || 2 * hy == Ly) ? 1 : 2;
  for (int rr = 0; rr < nrow; ++rr) {
    const int ky = rr ? Ly - hy : hy;
    const bool fy = rr != 0;  // ky > Ly / 2
    const int pyy = op.ypos_at[ky];
    for (int r = 0; r < R; ++r) {
      if (active && !active[r]) continue;
      float2* base = buf + (int64_t)r * 3 * comp_sz + (int64_t)pyy * Lx + col0;
      // ---- first forward stage (radix R0, span S0), read from global memory
      for (int j = threadIdx.x / NU; j < S0; j += NT / NU) {
        const bool ok = tp < npv;
        const float2* src = base + c * comp_sz + (int64_t)j * plane_sz + 2 * tp;
        float2 va[R0], vb[R0];
        if (R0 % 2 == 0 && half) {
#pragma unroll
          for (int i = 0; i < R0 / 2; ++i) {
            const float4 q = (ok && j + i * S0 < nz)
                                 ? *reinterpret_cast<const float4*>(src + (int64_t)i * S0 * plane_sz)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            split4(q, va[i], vb[i]);
          }
          if constexpr (R0 % 2 == 0) {
            dft_half<R0, false, true, false>(va);
            dft_half<R0, false, true, false>(vb);
          }
        } else {
#pragma unroll
          for (int i = 0; i < R0; ++i) {
            const float4 q = (ok && j + i * S0 < nz)
                                 ? *reinterpret_cast<const float4*>(src + (int64_t)i * S0 * plane_sz)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            split4(q, va[i], vb[i]);
          }
          dft<R0, false>(va);
          dft<R0, false>(vb);
        }
        if (j > 0) {
#pragma unroll
          for (int m = 1; m < R0; ++m) {
            const float2 w = ldc(&tw[j * (R0 - 1) + (m - 1)]);
            va[m] = cmul(va[m], w);
            vb[m] = cmul(vb[m], w);
          }
        }
#pragma unroll
        for (int m = 0; m < R0; ++m)
          sd[(j + m * S0) * NU + u] = make_float4(va[m].x, va[m].y, vb[m].x, vb[m].y);
      }
      __syncthreads();
      stages_pair<false, P, 1, NS - 1, NU, NT>(sd, tw);
      if (GS) {  // the Ghat tile has landed (a no-op after the first pass)
        cp_async_wait_all();
        __syncthreads();
      }
      // ---- multiply by Ghat at each frequency (all three components)
      for (int p = threadIdx.x / NP; p < L && tpm < npv; p += NT / NP) {
        const int tp = tpm;
        const int kz = P::k_at(p);
        const bool fz = kz > L / 2;
        const int hz = fz ? L - kz : kz;
        float4* row = sd + p * NU + tp;
        float2 a[3], bb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) split4(row[c * NP], a[c], bb[c]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int kx = op.kx_at[col0 + 2 * tp + e];
          const bool fx = kx > kxh;
          float2 g[6];
          if (GS) {
            G6<float>::load_smem(gs + 6 * (hz * TILE + 2 * tp + e), g);
          } else {
            const int hx = fx ? Lx - kx : kx;
            G6<float>::load(op.ghat + 6 * (((int64_t)hz * op.Hy + hy) * op.Hx + hx), g);
          }
          spectral_mul<float, false>(g, fx, fy, fz, e ? bb : a, 1);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) row[c * NP] = make_float4(a[c].x, a[c].y, bb[c].x, bb[c].y);
      }
      __syncthreads();
      stages_pair<true, P, 1, NS - 1, NU, NT>(sd, tw);
      // ---- last inverse stage (radix R0), written to global memory (z < nz)
      for (int j = threadIdx.x / NU; j < S0; j += NT / NU) {
        const bool ok = tp < npv;
        float2* dst = base + c * comp_sz + (int64_t)j * plane_sz + 2 * tp;
        float2 va[R0], vb[R0];
#pragma unroll
        for (int m = 0; m < R0; ++m) split4(sd[(j + m * S0) * NU + u], va[m], vb[m]);
        if (j > 0) {
#pragma unroll
          for (int m = 1; m < R0; ++m) {
            const float2 w = ldc(&tw[j * (R0 - 1) + (m - 1)]);
            va[m] = cmulc(w, va[m]);
            vb[m] = cmulc(w, vb[m]);
          }
        }
        if (R0 % 2 == 0 && half) {
          if constexpr (R0 % 2 == 0) {
            dft_half<R0, true, false, true>(va);
            dft_half<R0, true, false, true>(vb);
          }
#pragma unroll
          for (int i = 0; i < R0 / 2; ++i)
            if (ok && j + i * S0 < nz)
              *reinterpret_cast<float4*>(dst + (int64_t)i * S0 * plane_sz) =
                  make_float4(va[i].x, va[i].y, vb[i].x, vb[i].y);
        } else {
          dft<R0, true>(va);
          dft<R0, true>(vb);
#pragma unroll
          for (int i = 0; i < R0; ++i)
            if (ok && j + i * S0 < nz)
              *reinterpret_cast<float4*>(dst + (int64_t)i * S0 * plane_sz) =
                  make_float4(va[i].x, va[i].y, vb[i].x, vb[i].y);
        }
      }
      __syncthreads();  // the next pass overwrites sd
    }
  }
  if (GS) cp_async_wait_all();  // no copy outlives the CTA (every RHS may be frozen)
}

template <int TILE, class P, bool GS> constexpr size_t zpair_smem() {
  return (size_t)P::L * 3 * (TILE / 2) * sizeof(float4) +
         (GS ? (size_t)(P::L / 2 + 1) * TILE * 6 * sizeof(float2) : 0);
}

}  // namespace dda
