// Radix plans known at compile time (internal).  The FFT passes read their
// plan (radices, blocks, spans, twiddle offsets, the frequency held at each
// digit-reversed position) from an AxisPlan at run time; for the plans of the
// common grid lengths the FP32 passes are also compiled with the plan fixed,
// so that every stride, loop bound and table index is a constant.  The stages
// below run exactly the operations of fft_stage / fft_smem in the same order.
#pragma once

#include "fft_core.cuh"

namespace dda {

// Stage t: radix radix(t), block B_t = L / (R_0 ... R_{t-1}), span
// S_t = B_t / R_t, twiddles w_{B_t}^{jm} at tw_off(t) + j (R_t - 1) + m - 1.
template <int R0, int R1, int R2 = 1, int R3 = 1> struct FixedPlan {
  static constexpr int NS = 1 + (R1 > 1) + (R2 > 1) + (R3 > 1);
  static constexpr int L = R0 * R1 * R2 * R3;
  static constexpr int radix(int t) { return t == 0 ? R0 : t == 1 ? R1 : t == 2 ? R2 : R3; }
  static constexpr int block(int t) {
    int b = L;
    for (int i = 0; i < t; ++i) b /= radix(i);
    return b;
  }
  static constexpr int span(int t) { return block(t) / radix(t); }
  static constexpr int tw_off(int t) {
    int o = 0;
    for (int i = 0; i < t; ++i) o += span(i) * (radix(i) - 1);
    return o;
  }
  static constexpr int nprod(int t) {
    int n = 1;
    for (int i = 0; i < t; ++i) n *= radix(i);
    return n;
  }
  // frequency at position pos after the forward (decimation in frequency)
  // transform: pos = sum_t m_t S_t holds sum_t m_t R_0 ... R_{t-1}
  static __device__ __forceinline__ int k_at(int pos) {
    int k = 0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int m = pos / span(t);
      pos -= m * span(t);
      k += m * nprod(t);
    }
    return k;
  }
};

// One in-place stage of `nlines` lines in shared memory (s[p ps + line]);
// HALF as in fft_stage.  div_nl is the fast_div magic of nlines.
template <typename C, bool INV, class P, int ST, bool HALF = false>
__device__ __forceinline__ void stage_p(C* s, int nlines, unsigned long long div_nl, int ps,
                                        const C* __restrict__ tw) {
  constexpr int R = P::radix(ST), B = P::block(ST), S = P::span(ST), NB = P::L / R;
  constexpr int RH = HALF ? R / 2 : R;
  const C* __restrict__ tws = tw + P::tw_off(ST);
  for (int b = threadIdx.x; b < nlines * NB; b += blockDim.x) {
    const int q = fast_div(b, div_nl), line = b - q * nlines;
    const int blk = q / S, j = q - blk * S;
    C* base = s + (blk * B + j) * ps + line;
    C v[R];
    if (!INV) {
#pragma unroll
      for (int i = 0; i < RH; ++i) v[i] = base[i * S * ps];
      if constexpr (HALF) dft_half<R, false, true, false>(v);
      else dft<R, false>(v);
      if (S > 1 && j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], ldc(&tws[j * (R - 1) + (m - 1)]));
      }
#pragma unroll
      for (int i = 0; i < R; ++i) base[i * S * ps] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = base[i * S * ps];
      if (S > 1 && j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc(ldc(&tws[j * (R - 1) + (m - 1)]), v[m]);
      }
      if constexpr (HALF) dft_half<R, true, false, true>(v);
      else dft<R, true>(v);
#pragma unroll
      for (int i = 0; i < RH; ++i) base[i * S * ps] = v[i];
    }
  }
  __syncthreads();
}

// Stage 0 with the zero-half pruning when `half` (even first radix only).
template <typename C, bool INV, class P>
__device__ __forceinline__ void stage0_p(C* s, int nlines, unsigned long long div_nl, int ps,
                                         const C* __restrict__ tw, bool half) {
  if constexpr (P::radix(0) % 2 == 0) {
    if (half) {
      stage_p<C, INV, P, 0, true>(s, nlines, div_nl, ps, tw);
      return;
    }
  }
  stage_p<C, INV, P, 0, false>(s, nlines, div_nl, ps, tw);
}

// Stages lo .. hi (forward: ascending; inverse: descending), lo >= 1.
template <typename C, bool INV, class P, int LO, int HI>
__device__ __forceinline__ void stages_p(C* s, int nlines, unsigned long long div_nl, int ps,
                                         const C* __restrict__ tw) {
  if constexpr (LO <= HI) {
    if constexpr (!INV) {
      stage_p<C, false, P, LO>(s, nlines, div_nl, ps, tw);
      stages_p<C, false, P, LO + 1, HI>(s, nlines, div_nl, ps, tw);
    } else {
      stage_p<C, true, P, HI>(s, nlines, div_nl, ps, tw);
      stages_p<C, true, P, LO, HI - 1>(s, nlines, div_nl, ps, tw);
    }
  }
}

// Full transform in shared memory (as fft_smem with a fixed plan).
template <typename C, bool INV, class P>
__device__ void fft_smem_p(C* s, int nlines, unsigned long long div_nl, int ps,
                           const C* __restrict__ tw, bool half) {
  if constexpr (!INV) {
    stage0_p<C, false, P>(s, nlines, div_nl, ps, tw, half);
    stages_p<C, false, P, 1, P::NS - 1>(s, nlines, div_nl, ps, tw);
  } else {
    stages_p<C, true, P, 1, P::NS - 1>(s, nlines, div_nl, ps, tw);
    stage0_p<C, true, P>(s, nlines, div_nl, ps, tw, half);
  }
}

constexpr unsigned long long div_magic_c(int d) {
  return ((1ull << 36) + (unsigned long long)d - 1) / (unsigned long long)d;
}

}  // namespace dda
