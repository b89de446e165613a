// z pass on column pairs (FP32, the kernel's own radix plan P of the z length,
// radices of at most 8, fixed at compile time, and NT threads per CTA).
//
// The same arithmetic as k_fft_z_mul_p -- forward FFT along z, the 3x3
// complex-symmetric multiply by Ghat, inverse FFT along z, for the three
// polarization components of each column -- with the work laid out for fewer
// instructions per point and for reuse of Ghat:
//   * a thread always works on two neighbouring columns at once: shared memory
//     holds a pair as one float4 (16-byte loads and stores, every twiddle
//     loaded once for both columns, half the index arithmetic);
//   * a CTA owns TILE columns at one octant row hy and runs both rows that
//     share it (ky = hy and ky = Ly - hy) for every right-hand side, so every
//     pass of the CTA reads the same Ghat rows: from L2 after the first (GS =
//     false), or staged once in shared memory with cp.async while the first
//     forward transform runs (GS = true);
//   * the last forward stage, the multiply and the first inverse stage are
//     separate sweeps over shared memory.  The layout keeps every 16-byte
//     access free of bank conflicts (for the 512-point plan; nearly so for
//     the others): transform rows padded per plan and tile (zpair_row), the
//     first and last stages' thread map (zpair_first_map), the multiply's
//     skewed position order (skew_item) and the Ghat tile's column stride
//     (zpair_gstride);
//   * optionally (TMA) each pass's column tile is loaded and stored by the
//     tensor-memory accelerator: one cp.async.bulk.tensor box per pass, landing
//     in (and leaving from) the upper half of the transform's shared memory,
//     with an mbarrier wait bounded in time (a kernel whose copy never arrives
//     sets op.zerr and returns).
// The plan P (e.g. 512 = 8 x 8 x 8) need not be the target's z plan: the z
// transform starts and ends inside this kernel, so only the frequency held at
// each position (P::k_at, for the multiply) and P's twiddle table (op.twz_pair)
// matter.  Small radices keep the registers low enough for two CTAs of NT
// threads per SM, and NT is a multiple of the pair-lines per row so every
// thread keeps one pair-line for the whole kernel (no index division in the
// loops).  The arithmetic is the same transform with another factorization,
// so results agree with the other z kernels to rounding, not bit for bit.
//
// grid: (ceil(Lx / TILE), Ly / 2 + 1), NT threads.  Needs Lx even (pairs of
// columns are 16-byte aligned) and, for TMA, nz <= 256.  Shared memory: the
// padded rows, zpair_row(Lz) float4, plus (GS) the Ghat tile,
// TILE * zpair_gstride(Lz/2 + 1, TILE) float2.
#pragma once

#include <cuda.h>  // CUtensorMap

#include "matvec_impl.cuh"

namespace dda {

// ---- tensor-memory-access (TMA) copies and mbarriers, inline PTX ----------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// global -> shared copy of one box of a 4-D tensor map, completing on bar
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_addr(bar))
      : "memory");
}
// shared -> global copy of one box (elements outside the tensor are dropped)
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0,
                                             int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::
          "l"(reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// wait until the committed bulk stores have read their shared memory
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// wait until the committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Bounded wait on an mbarrier phase: false after 2^22 polls (each poll may
// suspend the thread for a while in hardware), i.e. well over a second.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void split4(const float4 q, float2& a, float2& b) {
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}

// Rows of the transform in shared memory: position pos of the NU = 3 TILE/2
// pair-lines starts at float4 index pos * NU + (pos / D) * K, i.e. K float4
// are skipped after every D positions (none where D = 0).  D and K are chosen
// per plan and tile so that every stage's 16-byte accesses, the multiply's and
// the staged tile's fall in distinct bank slots per quarter-warp (a model of
// the bank mapping over all of the kernel's access patterns; the plans of
// lengths 64 and 288 keep unpadded rows, where no padding helped).
__host__ __device__ constexpr int zpair_pad_div(int L, int tile) {
  return L == 512 ? (tile == 4 ? 8 : 2) : L == 128 ? (tile == 4 ? 4 : 2) : 0;
}
__host__ __device__ constexpr int zpair_pad_k(int L, int tile) {
  return L == 512 ? (tile == 4 ? 6 : 1) : L == 128 ? (tile == 4 ? 6 : 2) : 0;
}
__host__ __device__ constexpr int zpair_row(int pos, int L, int tile) {
  return pos * (3 * tile / 2) +
         (zpair_pad_div(L, tile) ? pos / zpair_pad_div(L, tile) * zpair_pad_k(L, tile) : 0);
}

// Offset (float4) of element i of a butterfly of span S from its first
// element, in the padded rows of zpair_row: a multiple of the padding period D
// apart (D | S), or inside one period (S = 1, D | block), so it is a constant.
template <int L, int TILE, int S>
__device__ __forceinline__ constexpr int zpair_step(int i) {
  constexpr int D = zpair_pad_div(L, TILE), K = zpair_pad_k(L, TILE), NU = 3 * TILE / 2;
  return i * S * NU + (D == 0 ? 0 : S % D == 0 ? i * (S / D) * K : (i / D) * K);
}

// One in-place stage ST of plan P on NU pair-lines of shared memory, both
// columns of each pair (forward: DFT then twiddles; inverse: the adjoint).
template <bool INV, class P, int ST, int TILE, int NT>
__device__ __forceinline__ void stage_pair(float4* sd, const float2* __restrict__ tw) {
  constexpr int R = P::radix(ST), B = P::block(ST), S = P::span(ST), NB = P::L / R;
  constexpr int NU = 3 * TILE / 2, D = zpair_pad_div(P::L, TILE);
  static_assert(NT % NU == 0, "a thread keeps one pair-line");
  static_assert(D == 0 || S % D == 0 || (S == 1 && B % D == 0), "padding period");
  const float2* __restrict__ tws = tw + P::tw_off(ST);
  const int u = threadIdx.x % NU;
  for (int q = threadIdx.x / NU; q < NB; q += NT / NU) {
    const int blk = q / S, j = q - blk * S;
    float4* base = sd + zpair_row(blk * B + j, P::L, TILE) + u;
    float2 va[R], vb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) split4(base[zpair_step<P::L, TILE, S>(i)], va[i], vb[i]);
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
    for (int i = 0; i < R; ++i)
      base[zpair_step<P::L, TILE, S>(i)] = make_float4(va[i].x, va[i].y, vb[i].x, vb[i].y);
  }
  __syncthreads();
}

// The multiply visits the positions of a transform in a skewed order: item v
// (0 <= v < L) takes the last digit m_last = v mod R_last, the middle digits from
// the middle of v and the first digit m_0 = (m_last + top of v) mod R_0, so that
// neighbouring items differ both in the position's last digit (its shared-memory
// row, rows are consecutive) and in the frequency's first digit (its Ghat row);
// with either natural order the other would repeat across a quarter-warp and
// the 16-byte accesses would collide on the same banks.  Returns the position
// p and the frequency k held there.
template <class P>
__device__ __forceinline__ void skew_item(int v, int& p, int& k) {
  constexpr int NS = P::NS, R0 = P::radix(0), RL = P::radix(NS - 1);
  const int a = v % RL;
  int rest = v / RL;
  int pos = a * P::span(NS - 1), frq = a * P::nprod(NS - 1);
#pragma unroll
  for (int t = NS - 2; t >= 1; --t) {
    const int m = rest % P::radix(t);
    rest /= P::radix(t);
    pos += m * P::span(t);
    frq += m * P::nprod(t);
  }
  const int m0 = (a + rest) % R0;
  p = pos + m0 * P::span(0);
  k = frq + m0;
}

// Ghat tile of a pair-kernel CTA in shared memory: column t's rows hz at
// gs[t * stride + 6 hz] (float2), the column stride padded so that the columns
// one instruction reads (2 apart: 2 columns for TILE 4, 4 for TILE 8) start in
// different 16-byte slots of the 128-byte bank cycle (64 / 32 bytes apart).
__host__ __device__ constexpr int zpair_gstride(int Hz, int tile) {
  return (Hz * 6 + 7) / 8 * 8 + (tile == 4 ? 4 : 2);  // in float2
}


template <int TILE>
__device__ __forceinline__ void ghat_tile_pairs_async(const OpView<float>& op, float2* gs,
                                                      int col0, int ncol, int hy) {
  const int stride = zpair_gstride(op.Hz, TILE);
  const int n = op.Hz * TILE * 3;  // 16-byte chunks: 3 per point
  const int64_t plane = (int64_t)op.Hy * op.Hx;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int ch = e % 3, pt = e / 3;
    const int hz = pt % op.Hz, t = pt / op.Hz;
    if (t < ncol) {
      const int kx = op.kx_at[col0 + t];
      const int hx = kx > (op.Lx >> 1) ? op.Lx - kx : kx;
      const float2* src = op.ghat + 6 * (hz * plane + (int64_t)hy * op.Hx + hx) + 2 * ch;
      cp_async<16>(gs + t * stride + 6 * hz + 2 * ch, src);
    }
  }
  cp_async_commit();
}

// Stages LO..HI forward (ascending) or inverse (descending).
template <bool INV, class P, int LO, int HI, int TILE, int NT>
__device__ __forceinline__ void stages_pair(float4* sd, const float2* __restrict__ tw) {
  if constexpr (LO <= HI) {
    if constexpr (!INV) {
      stage_pair<false, P, LO, TILE, NT>(sd, tw);
      stages_pair<false, P, LO + 1, HI, TILE, NT>(sd, tw);
    } else {
      stage_pair<true, P, HI, TILE, NT>(sd, tw);
      stages_pair<true, P, LO, HI - 1, TILE, NT>(sd, tw);
    }
  }
}

// The first forward and the last inverse stage give each thread one
// (position j, component c, column pair tp): tp fastest, then 8 / NP
// consecutive positions, then the component, so that a quarter-warp's 16-byte
// accesses to the staged tile ([c][z][column]) and to the transform rows fall
// in distinct bank slots.
template <int TILE>
__device__ __forceinline__ void zpair_first_map(int tid, int& j, int& c, int& tp) {
  constexpr int NP = TILE / 2, JL = 8 / NP;
  tp = tid % NP;
  int r = tid / NP;
  const int jl = r % JL;
  r /= JL;
  c = r % 3;
  j = (r / 3) * JL + jl;
}

template <int TILE, class P, bool GS, int NT, bool TMA>
__global__ void __launch_bounds__(NT, 2)
k_fft_z_pairs(OpView<float> op, float2* __restrict__ buf, int R, const int* __restrict__ active,
              const __grid_constant__ CUtensorMap tmap) {
  static_assert(TILE % 2 == 0, "column pairs");
  constexpr int L = P::L, NS = P::NS, R0 = P::radix(0), S0 = P::span(0);
  constexpr int NP = TILE / 2, NU = 3 * NP;
  static_assert(NT % NU == 0 && NT % NP == 0, "a thread keeps one pair-line");
  constexpr int PD = zpair_pad_div(L, TILE);
  static_assert((zpair_row(L / 2, L, TILE) * 16) % 128 == 0, "TMA staging 128-byte aligned");
  static_assert(PD == 0 || S0 % PD == 0, "first-stage span a multiple of the padding period");
  extern __shared__ __align__(128) unsigned char zpair_smem_raw[];
  float4* sd = reinterpret_cast<float4*>(zpair_smem_raw);
  float2* gs = reinterpret_cast<float2*>(sd + zpair_row(L, L, TILE));
  const int Lx = op.Lx, Ly = op.Ly, nz = op.nz;
  const int hy = blockIdx.y;
  const int col0 = blockIdx.x * TILE;
  const int npv = min(TILE, Lx - col0) >> 1;  // pairs inside the grid (Lx even)
  if (GS) ghat_tile_pairs_async<TILE>(op, gs, col0, 2 * npv, hy);
  const int gstride = zpair_gstride(op.Hz, TILE);
  const int64_t plane_sz = (int64_t)Ly * Lx;
  const int64_t comp_sz = (int64_t)nz * plane_sz;
  const bool half = 2 * nz <= L;
  const float2* __restrict__ tw = op.twz_pair;
  int jf, c, tp;  // first/last stage: position, component, column pair
  zpair_first_map<TILE>(threadIdx.x, jf, c, tp);
  const int u = c * NP + tp;                // the pair-line
  const int tpm = threadIdx.x % NP;         // the column pair in the multiply
  // the multiply's two columns: frequency kx (octant column hx, flipped or not)
  int hxm[2] = {0, 0};
  bool fxm[2] = {false, false};
  if (tpm < npv) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int kx = op.kx_at[col0 + 2 * tpm + e];
      fxm[e] = kx > (Lx >> 1);
      hxm[e] = fxm[e] ? Lx - kx : kx;
    }
  }
  // TMA: each pass's input tile lands in the upper half of sd (rows >= L/2, free
  // until the first stage writes them: the inputs are the nz <= L/2 lower rows)
  // as [c][z][t]; the output tile leaves from there the same way.
  __shared__ __align__(8) uint64_t bar;
  float2* stg = reinterpret_cast<float2*>(sd + zpair_row(L / 2, L, TILE));
  unsigned phase = 0;
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  constexpr int NJ = (S0 + NT / NU - 1) / (NT / NU);  // first-stage items per thread
  // the rows sharing octant row hy: ky = hy, and ky = Ly - hy unless that is hy
  const int nrow = (hy == 0 || 2 * hy == Ly) ? 1 : 2;
  for (int rr = 0; rr < nrow; ++rr) {
    const int ky = rr ? Ly - hy : hy;
    const bool fy = rr != 0;  // ky > Ly / 2
    const int pyy = op.ypos_at[ky];
    for (int r = 0; r < R; ++r) {
      if (active && !active[r]) continue;
      float2* base = buf + (int64_t)r * 3 * comp_sz + (int64_t)pyy * Lx + col0;
      if (TMA) {
        if (threadIdx.x == 0) {
          fence_proxy_async();  // sd's earlier generic accesses before the async write
          mbar_arrive_expect_tx(&bar, (unsigned)(3 * nz * TILE * sizeof(float2)));
          tma_load_4d(stg, &tmap, &bar, col0, pyy, 0, 3 * r);
        }
        const bool ok = mbar_wait_bounded(&bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {  // the copy never completed: report and stop
          if (threadIdx.x == 0) {
            if (op.zerr) atomicExch(op.zerr, 1);
            bulk_wait_all();  // the stores already issued finish before the exit
          }
          if (GS) cp_async_wait_all();
          return;
        }
      }
      // ---- first forward stage (radix R0, span S0), read from global memory
      // (or, with TMA, from the staged tile; its outputs then wait for every
      // thread's reads before overwriting the staging rows)
      float4 keep[TMA ? NJ * R0 : 1];
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = jf + jj * (NT / NU);
        if (j >= S0) break;
        const bool ok = tp < npv;
        const float2* src = base + c * comp_sz + (int64_t)j * plane_sz + 2 * tp;
        float2 va[R0], vb[R0];
        const int nin = (R0 % 2 == 0 && half) ? R0 / 2 : R0;
#pragma unroll
        for (int i = 0; i < R0; ++i) {
          if (i >= nin) break;
          const int z = j + i * S0;
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (TMA) {
            if (z < nz) q = *reinterpret_cast<const float4*>(stg + (c * nz + z) * TILE + 2 * tp);
          } else if (ok && z < nz) {
            q = *reinterpret_cast<const float4*>(src + (int64_t)i * S0 * plane_sz);
          }
          split4(q, va[i], vb[i]);
        }
        if (R0 % 2 == 0 && half) {
          if constexpr (R0 % 2 == 0) {
            dft_half<R0, false, true, false>(va);
            dft_half<R0, false, true, false>(vb);
          }
        } else {
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
        for (int m = 0; m < R0; ++m) {
          const float4 o = make_float4(va[m].x, va[m].y, vb[m].x, vb[m].y);
          if (TMA) keep[jj * R0 + m] = o;
          else sd[zpair_row(j, L, TILE) + zpair_step<L, TILE, S0>(m) + u] = o;
        }
      }
      if (TMA) {
        __syncthreads();  // every staged input has been read
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          const int j = jf + jj * (NT / NU);
          if (j >= S0) break;
#pragma unroll
          for (int m = 0; m < R0; ++m)
            sd[zpair_row(j, L, TILE) + zpair_step<L, TILE, S0>(m) + u] = keep[jj * R0 + m];
        }
      }
      __syncthreads();
      stages_pair<false, P, 1, NS - 1, TILE, NT>(sd, tw);
      if (GS) {  // the Ghat tile has landed (a no-op after the first pass)
        cp_async_wait_all();
        __syncthreads();
      }
      // ---- multiply by Ghat at each frequency (all three components), the
      // positions in the skewed order of skew_item
      for (int v = threadIdx.x / NP; v < L && tpm < npv; v += NT / NP) {
        const int tp2 = tpm;
        int p, kz;
        skew_item<P>(v, p, kz);
        const bool fz = kz > L / 2;
        const int hz = fz ? L - kz : kz;
        float4* row = sd + zpair_row(p, L, TILE) + tp2;
        float2 a[3], bb[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) split4(row[cc * NP], a[cc], bb[cc]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float2 g[6];
          if (GS) {
            G6<float>::load_smem(gs + (2 * tp2 + e) * gstride + 6 * hz, g);
          } else {
            G6<float>::load(op.ghat + 6 * (((int64_t)hz * op.Hy + hy) * op.Hx + hxm[e]), g);
          }
          spectral_mul<float, false>(g, fxm[e], fy, fz, e ? bb : a, 1);
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          row[cc * NP] = make_float4(a[cc].x, a[cc].y, bb[cc].x, bb[cc].y);
      }
      __syncthreads();
      stages_pair<true, P, 1, NS - 1, TILE, NT>(sd, tw);
      // ---- last inverse stage (radix R0), written to global memory (z < nz);
      // with TMA the outputs go to the staging rows once every thread has
      // read its inputs, and one tensor store writes the tile
      float4 outk[TMA ? NJ * R0 : 1];
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = jf + jj * (NT / NU);
        if (j >= S0) break;
        const bool ok = tp < npv;
        float2* dst = base + c * comp_sz + (int64_t)j * plane_sz + 2 * tp;
        float2 va[R0], vb[R0];
#pragma unroll
        for (int m = 0; m < R0; ++m)
          split4(sd[zpair_row(j, L, TILE) + zpair_step<L, TILE, S0>(m) + u], va[m], vb[m]);
        if (j > 0) {
#pragma unroll
          for (int m = 1; m < R0; ++m) {
            const float2 w = ldc(&tw[j * (R0 - 1) + (m - 1)]);
            va[m] = cmulc(w, va[m]);
            vb[m] = cmulc(w, vb[m]);
          }
        }
        const bool hout = R0 % 2 == 0 && half;
        if (hout) {
          if constexpr (R0 % 2 == 0) {
            dft_half<R0, true, false, true>(va);
            dft_half<R0, true, false, true>(vb);
          }
        } else {
          dft<R0, true>(va);
          dft<R0, true>(vb);
        }
#pragma unroll
        for (int i = 0; i < R0; ++i) {
          if (hout && i >= R0 / 2) break;
          const float4 o = make_float4(va[i].x, va[i].y, vb[i].x, vb[i].y);
          if (TMA) outk[jj * R0 + i] = o;
          else if (ok && j + i * S0 < nz)
            *reinterpret_cast<float4*>(dst + (int64_t)i * S0 * plane_sz) = o;
        }
      }
      if (TMA) {
        __syncthreads();  // every input of the last stage has been read
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
          const int j = jf + jj * (NT / NU);
          if (j >= S0) break;
          // (with the pruned stage only i < R0/2 were formed; the others have
          // z >= R0/2 * S0 = L/2 >= nz)
#pragma unroll
          for (int i = 0; i < R0; ++i) {
            const int z = j + i * S0;
            if (z < nz)
              *reinterpret_cast<float4*>(stg + (c * nz + z) * TILE + 2 * tp) = outk[jj * R0 + i];
          }
        }
        fence_proxy_async();  // the generic writes, before the async store reads them
        __syncthreads();
        if (threadIdx.x == 0) {
          tma_store_4d(&tmap, stg, col0, pyy, 0, 3 * r);
          bulk_commit();
          bulk_wait_read();  // the staging rows may be overwritten from here on
        }
      }
      __syncthreads();  // the next pass overwrites sd
    }
  }
  if (GS) cp_async_wait_all();  // no copy outlives the CTA (every RHS may be frozen)
  if (TMA && threadIdx.x == 0) bulk_wait_all();
}

// 4-D tensor map of the spectral scratch [R][3][nz][Ly][Lx] (8-byte complex
// FP32 elements) with a box of TILE columns x 1 row x nz planes x 3 components,
// for the TMA variant; false when the driver call is unavailable or refuses
// (the caller then keeps the plain loads).
bool encode_zpair_map(CUtensorMap* map, const float2* scratch, int Lx, int Ly, int nz, int R,
                      int tile);

template <int TILE, class P, bool GS> constexpr size_t zpair_smem() {
  return (size_t)zpair_row(P::L, P::L, TILE) * sizeof(float4) +
         (GS ? (size_t)TILE * zpair_gstride(P::L / 2 + 1, TILE) * sizeof(float2) : 0);
}

}  // namespace dda
