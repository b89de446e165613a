// Mixed radix-2/3/4/5/8 in-place FFT on lines held in shared memory.
//
// The guide's GPFA option factors each grid length as 2^a 3^b 5^c (Sec.
// "Choice of FFT Algorithm"); the same smooth lengths are transformed here.
// A CTA holds `nlines` lines of length L in shared memory as s[p*pstride +
// line] (line index fastest, so consecutive threads touch consecutive words
// and every stage is free of bank conflicts whatever its stride).
//
// Forward transforms are decimation in frequency: natural-order input,
// digit-reversed output.  Inverse transforms are decimation in time:
// digit-reversed input, natural-order output.  The spectra therefore never need
// a permutation: the pointwise multiply only has to know which frequency sits
// at each position (a small table), and every butterfly reads and writes the
// same R positions, so one butterfly at a time lives in registers and a stage
// needs a single barrier.
//
// Stage t (radix R, block B, span S = B/R) of the forward transform, for each
// block b and j < S:  y_m = sum_i x[bB + j + iS] w_R^{im},  x[bB + j + mS] =
// y_m w_B^{jm}, with w_n = exp(-2 pi i/n).  The inverse runs the adjoint
// stages in reverse order.  After all forward stages, position sum_t m_t S_t
// holds frequency sum_t m_t R_1...R_{t-1}.
#pragma once

#include "dda_common.cuh"

namespace dda {

// ---- radix-R DFTs in registers (forward: exp(-2 pi i nk/R); INV: conjugate) --
// HIN: the upper half of the inputs is known to be zero (zero padding: a
// transform of n <= L/2 values, first forward stage); HOUT: only the lower
// half of the outputs is wanted (pruned output, last inverse stage).  The
// skipped terms are exact zeros or unused results, so the kept outputs are
// bit-identical to the full transform's.
template <bool INV, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  if (HIN) { b = a; return; }
  if (HOUT) { a = cadd(a, b); return; }
  C t = csub(a, b); a = cadd(a, b); b = t;
}

template <bool INV, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  if (HIN) {  // a2 = a3 = 0
    const C d13 = cmul_i<INV>(a1);
    const C s = a0;
    if (!HOUT) { a2 = csub(s, a1); a3 = csub(s, d13); }
    a0 = cadd(s, a1);
    a1 = cadd(s, d13);
    return;
  }
  C s02 = cadd(a0, a2), d02 = csub(a0, a2);
  C s13 = cadd(a1, a3), d13 = cmul_i<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a1 = cadd(d02, d13);
  if (!HOUT) {
    a2 = csub(s02, s13);
    a3 = csub(d02, d13);
  }
}

template <bool INV, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft8(C (&a)[8]) {
  using T = decltype(a[0].x);
  const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV, HIN>(e0, e1, e2, e3);
  dft4<INV, HIN>(o0, o1, o2, o3);
  // W^1 = (1 -/+ i)/sqrt2, W^2 = -/+ i, W^3 = (-1 -/+ i)/sqrt2
  C w1, w3;
  if (INV) {
    w1.x = h * (o1.x - o1.y); w1.y = h * (o1.x + o1.y);
    w3.x = -h * (o3.x + o3.y); w3.y = h * (o3.x - o3.y);
  } else {
    w1.x = h * (o1.x + o1.y); w1.y = h * (o1.y - o1.x);
    w3.x = h * (o3.y - o3.x); w3.y = -h * (o3.x + o3.y);
  }
  C w2 = cmul_i<INV>(o2);
  if (!HOUT) {
    a[4] = csub(e0, o0); a[5] = csub(e1, w1);
    a[6] = csub(e2, w2); a[7] = csub(e3, w3);
  }
  a[0] = cadd(e0, o0);
  a[1] = cadd(e1, w1);
  a[2] = cadd(e2, w2);
  a[3] = cadd(e3, w3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
  using T = decltype(a0.x);
  const T s = (T)0.86602540378443864676;  // sqrt(3)/2
  C t1 = cadd(a1, a2);
  C t2; t2.x = a0.x - (T)0.5 * t1.x; t2.y = a0.y - (T)0.5 * t1.y;
  C d = csub(a1, a2);
  // forward: X1 = t2 - i s d, X2 = t2 + i s d
  C isd; isd.x = -s * d.y; isd.y = s * d.x;  // i*s*d
  a0 = cadd(a0, t1);
  if (INV) { a1 = cadd(t2, isd); a2 = csub(t2, isd); }
  else     { a1 = csub(t2, isd); a2 = cadd(t2, isd); }
}

template <bool INV, typename C> __device__ __forceinline__ void dft5(C (&a)[5]) {
  using T = decltype(a[0].x);
  const T c1 = (T)0.30901699437494742410;   // cos(2 pi/5) = (sqrt5 - 1)/4
  const T c2 = (T)-0.80901699437494742410;  // cos(4 pi/5) = -(sqrt5 + 1)/4
  const T s1 = (T)0.95105651629515357212;   // sin(2 pi/5)
  const T s2 = (T)0.58778525229247312917;   // sin(4 pi/5)
  C t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
  C t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
  C b1, b2;
  b1.x = a[0].x + c1 * t1.x + c2 * t2.x; b1.y = a[0].y + c1 * t1.y + c2 * t2.y;
  b2.x = a[0].x + c2 * t1.x + c1 * t2.x; b2.y = a[0].y + c2 * t1.y + c1 * t2.y;
  C u1, u2;  // i*(s1 t3 + s2 t4), i*(s2 t3 - s1 t4)
  u1.x = -(s1 * t3.y + s2 * t4.y); u1.y = s1 * t3.x + s2 * t4.x;
  u2.x = -(s2 * t3.y - s1 * t4.y); u2.y = s2 * t3.x - s1 * t4.x;
  a[0] = cadd(a[0], cadd(t1, t2));
  if (INV) {
    a[1] = cadd(b1, u1); a[4] = csub(b1, u1);
    a[2] = cadd(b2, u2); a[3] = csub(b2, u2);
  } else {
    a[1] = csub(b1, u1); a[4] = cadd(b1, u1);
    a[2] = csub(b2, u2); a[3] = cadd(b2, u2);
  }
}

// w * a with w = c - i s (forward) or c + i s (inverse)
template <bool INV, typename C, typename T>
__device__ __forceinline__ C rot(C a, T c, T s) {
  C r;
  if (INV) { r.x = c * a.x - s * a.y; r.y = c * a.y + s * a.x; }
  else     { r.x = c * a.x + s * a.y; r.y = c * a.y - s * a.x; }
  return r;
}

// 16 = 4 x 4: DFT4 over n1 for each n2, twiddle w16^(n2 k1), DFT4 over n2;
// X[k1 + 4 k2] ends in a[k1 + 4 k2].  With HIN the inputs n1 = 2, 3 are zero;
// with HOUT only k2 = 0, 1 are formed.
template <bool INV, bool HIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void dft16(C (&a)[16]) {
  using T = decltype(a[0].x);
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // pi/8
  const T h = (T)0.70710678118654752440;
  C y[4][4];  // y[n2][k1]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C b0 = a[n2], b1 = a[4 + n2], b2 = a[8 + n2], b3 = a[12 + n2];
    dft4<INV, HIN>(b0, b1, b2, b3);
    y[n2][0] = b0; y[n2][1] = b1; y[n2][2] = b2; y[n2][3] = b3;
  }
  // twiddles w16^(n2 k1): (1,1)=1, (1,2)=2, (1,3)=3, (2,1)=2, (2,2)=4, (2,3)=6,
  // (3,1)=3, (3,2)=6, (3,3)=9 in units of pi/8
  y[1][1] = rot<INV>(y[1][1], c1, s1);
  y[1][2] = rot<INV>(y[1][2], h, h);
  y[1][3] = rot<INV>(y[1][3], s1, c1);
  y[2][1] = rot<INV>(y[2][1], h, h);
  y[2][2] = cmul_i<INV>(y[2][2]);
  y[2][3] = rot<INV>(y[2][3], -h, h);
  y[3][1] = rot<INV>(y[3][1], s1, c1);
  y[3][2] = rot<INV>(y[3][2], -h, h);
  y[3][3] = rot<INV>(y[3][3], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C b0 = y[0][k1], b1 = y[1][k1], b2 = y[2][k1], b3 = y[3][k1];
    dft4<INV, false, HOUT>(b0, b1, b2, b3);
    a[k1] = b0; a[k1 + 4] = b1;
    if (!HOUT) { a[k1 + 8] = b2; a[k1 + 12] = b3; }
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C (&v)[R]) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 5) dft5<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else dft16<INV>(v);
}

// Even radices only: HIN -- v[R/2 ..] are zero; HOUT -- only v[0 .. R/2) wanted.
template <int R, bool INV, bool HIN, bool HOUT, typename C>
__device__ __forceinline__ void dft_half(C (&v)[R]) {
  static_assert(R % 2 == 0, "half transforms need an even radix");
  if constexpr (R == 2) dft2<INV, HIN, HOUT>(v[0], v[1]);
  else if constexpr (R == 4) dft4<INV, HIN, HOUT>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV, HIN, HOUT>(v);
  else dft16<INV, HIN, HOUT>(v);
}

// ---- one in-place stage ------------------------------------------------------
// HALF (even R, block B = L only, i.e. the first forward stage or the last
// inverse one): forward -- positions >= L/2 hold zeros and are not read;
// inverse -- only positions < L/2 are formed and written.
template <typename C, int R, bool INV, bool HALF = false>
__device__ __forceinline__ void fft_stage(C* s, int nlines, int pstride, int L, int B,
                                          unsigned long long sdiv, const C* __restrict__ tw) {
  const int S = B / R;
  const int nb = nlines * (L / R);
  constexpr int RH = HALF ? R / 2 : R;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = b % nlines, q = b / nlines;
    const int blk = fast_div(q, sdiv), j = q - blk * S;
    C* base = s + (blk * B + j) * pstride + line;
    C v[R];
    if (!INV) {
#pragma unroll
      for (int i = 0; i < RH; ++i) v[i] = base[i * S * pstride];
      if constexpr (HALF) dft_half<R, false, true, false>(v);
      else dft<R, false>(v);
      if (j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], ldc(&tw[j * (R - 1) + (m - 1)]));
      }
#pragma unroll
      for (int i = 0; i < R; ++i) base[i * S * pstride] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = base[i * S * pstride];
      if (j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc(ldc(&tw[j * (R - 1) + (m - 1)]), v[m]);
      }
      if constexpr (HALF) dft_half<R, true, false, true>(v);
      else dft<R, true>(v);
#pragma unroll
      for (int i = 0; i < RH; ++i) base[i * S * pstride] = v[i];
    }
  }
  __syncthreads();
}

#define DDA_RADIX_DISPATCH(radix, BODY)                 \
  switch (radix) {                                      \
    case 16: { constexpr int RR = 16; BODY; } break;    \
    case 8: { constexpr int RR = 8; BODY; } break;      \
    case 4: { constexpr int RR = 4; BODY; } break;      \
    case 2: { constexpr int RR = 2; BODY; } break;      \
    case 3: { constexpr int RR = 3; BODY; } break;      \
    default: { constexpr int RR = 5; BODY; } break;     \
  }

// the same without radix 16 (stages the plan never gives radix 16)
#define DDA_RADIX_DISPATCH_SMALL(radix, BODY)           \
  switch (radix) {                                      \
    case 8: { constexpr int RR = 8; BODY; } break;      \
    case 4: { constexpr int RR = 4; BODY; } break;      \
    case 2: { constexpr int RR = 2; BODY; } break;      \
    case 3: { constexpr int RR = 3; BODY; } break;      \
    default: { constexpr int RR = 5; BODY; } break;     \
  }

template <typename C, bool INV, int R, bool HALF = false>
__device__ __forceinline__ void run_stage(C* s, int nlines, int pstride, const AxisPlan& P,
                                          int st, const C* __restrict__ tw) {
  fft_stage<C, R, INV, HALF>(s, nlines, pstride, P.L, P.blk[st], P.sdiv[st],
                             tw + P.tw_off[st]);
}

template <typename C, bool INV, int R>
__device__ __forceinline__ void run_stage_half(C* s, int nlines, int pstride,
                                               const AxisPlan& P, int st,
                                               const C* __restrict__ tw, bool half) {
  if constexpr (R % 2 == 0) {
    if (half) {
      run_stage<C, INV, R, true>(s, nlines, pstride, P, st, tw);
      return;
    }
  }
  run_stage<C, INV, R, false>(s, nlines, pstride, P, st, tw);
}

// Full transform of `nlines` lines in shared memory, in place.  Forward: natural
// -> digit-reversed; inverse (unnormalized): digit-reversed -> natural.
// half: forward -- every line has zeros at positions >= L/2 (the caller need
// not write them); inverse -- only positions < L/2 are wanted (the others are
// left undefined).
template <typename C, bool INV>
__device__ void fft_smem(C* s, int nlines, int pstride, const AxisPlan& P,
                         const C* __restrict__ tw, bool half = false) {
  for (int k = 0; k < P.nstage; ++k) {
    const int st = INV ? P.nstage - 1 - k : k;
    if (st == 0) {  // block L: the stage the pruning applies to
      DDA_RADIX_DISPATCH(P.radix[0],
                         (run_stage_half<C, INV, RR>(s, nlines, pstride, P, 0, tw, half)));
    } else {
      DDA_RADIX_DISPATCH(P.radix[st], (run_stage<C, INV, RR>(s, nlines, pstride, P, st, tw)));
    }
  }
}

// ---- stages fused with global memory ---------------------------------------------
// The first forward stage (block = L) reads its R inputs straight from global
// memory through ld(line, p) (which returns 0 for positions beyond the input);
// the last inverse stage (its adjoint) writes straight to global memory through
// st(line, p, v) (which drops positions beyond the output).  The last forward
// stage (block = R, span 1) and its adjoint read/write R consecutive positions.
// Consecutive threads take consecutive lines, so with lines = consecutive
// columns of a row-major plane every global access is coalesced.

// With half (needs an even R): the caller guarantees that positions >= L/2 of
// every input line are zero, so only the lower half of each butterfly's inputs
// is read and the transform skips the zero terms.
template <typename C, int R, class LD>
__device__ __forceinline__ void stage_first_fwd(C* s, int nlines, int ps, int L,
                                                const C* __restrict__ tw, const LD& ld,
                                                bool half = false) {
  const int S = L / R;
  const int nb = nlines * S;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = b % nlines, j = b / nlines;
    C v[R];
    if constexpr (R % 2 == 0) {
      if (half) {
#pragma unroll
        for (int i = 0; i < R / 2; ++i) v[i] = ld(line, j + i * S);
        dft_half<R, false, true, false>(v);
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = ld(line, j + i * S);
        dft<R, false>(v);
      }
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = ld(line, j + i * S);
      dft<R, false>(v);
    }
    if (j > 0) {
#pragma unroll
      for (int m = 1; m < R; ++m) v[m] = cmul(v[m], ldc(&tw[j * (R - 1) + (m - 1)]));
    }
#pragma unroll
    for (int m = 0; m < R; ++m) s[(j + m * S) * ps + line] = v[m];
  }
  __syncthreads();
}

// With half (needs an even R): the caller keeps only positions < L/2 of every
// output line, so each butterfly forms and stores only its lower half.
template <typename C, int R, class ST>
__device__ __forceinline__ void stage_last_inv(const C* s, int nlines, int ps, int L,
                                               const C* __restrict__ tw, const ST& st,
                                               bool half = false) {
  const int S = L / R;
  const int nb = nlines * S;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = b % nlines, j = b / nlines;
    C v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = s[(j + m * S) * ps + line];
    if (j > 0) {
#pragma unroll
      for (int m = 1; m < R; ++m) v[m] = cmulc(ldc(&tw[j * (R - 1) + (m - 1)]), v[m]);
    }
    if constexpr (R % 2 == 0) {
      if (half) {
        dft_half<R, true, false, true>(v);
#pragma unroll
        for (int i = 0; i < R / 2; ++i) st(line, j + i * S, v[i]);
        continue;
      }
    }
    dft<R, true>(v);
#pragma unroll
    for (int i = 0; i < R; ++i) st(line, j + i * S, v[i]);
  }
}

template <typename C, int R, class ST>
__device__ __forceinline__ void stage_last_fwd(const C* s, int nlines, int ps, int L,
                                               const ST& st) {
  const int nb = nlines * (L / R);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = b % nlines, blk = b / nlines;
    C v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = s[(blk * R + i) * ps + line];
    dft<R, false>(v);
#pragma unroll
    for (int m = 0; m < R; ++m) st(line, blk * R + m, v[m]);
  }
}

template <typename C, int R, class LD>
__device__ __forceinline__ void stage_first_inv(C* s, int nlines, int ps, int L, const LD& ld) {
  const int nb = nlines * (L / R);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = b % nlines, blk = b / nlines;
    C v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = ld(line, blk * R + m);
    dft<R, true>(v);
#pragma unroll
    for (int i = 0; i < R; ++i) s[(blk * R + i) * ps + line] = v[i];
  }
  __syncthreads();
}

// Middle forward stages 1 .. nstage-2, or inverse stages nstage-2 .. 1.
template <typename C, bool INV>
__device__ __forceinline__ void fft_inner_stages(C* s, int nlines, int ps, const AxisPlan& P,
                                                 const C* __restrict__ tw) {
  for (int k = 1; k + 1 < P.nstage; ++k) {
    const int st = INV ? P.nstage - 1 - k : k;
    DDA_RADIX_DISPATCH(P.radix[st], (run_stage<C, INV, RR>(s, nlines, ps, P, st, tw)));
  }
}

// Forward transform of lines read from global memory, results written to
// global memory (needs nstage >= 2).
// half: the input lines hold at most L/2 values (zero above), see stage_first_fwd.
template <typename C, class LD, class ST>
__device__ void fft_global_fwd(C* s, int nlines, int ps, const AxisPlan& P,
                               const C* __restrict__ tw, const LD& ld, const ST& st,
                               bool half = false) {
  DDA_RADIX_DISPATCH(P.radix[0], (stage_first_fwd<C, RR>(s, nlines, ps, P.L, tw, ld, half)));
  fft_inner_stages<C, false>(s, nlines, ps, P, tw);
  DDA_RADIX_DISPATCH(P.radix[P.nstage - 1], (stage_last_fwd<C, RR>(s, nlines, ps, P.L, st)));
}

// Inverse transform of lines read from global memory (digit-reversed), natural
// order results written to global memory (needs nstage >= 2).
// half: only the first L/2 outputs of each line are kept, see stage_last_inv.
template <typename C, class LD, class ST>
__device__ void fft_global_inv(C* s, int nlines, int ps, const AxisPlan& P,
                               const C* __restrict__ tw, const LD& ld, const ST& st,
                               bool half = false) {
  DDA_RADIX_DISPATCH(P.radix[P.nstage - 1], (stage_first_inv<C, RR>(s, nlines, ps, P.L, ld)));
  fft_inner_stages<C, true>(s, nlines, ps, P, tw);
  DDA_RADIX_DISPATCH(P.radix[0], (stage_last_inv<C, RR>(s, nlines, ps, P.L, tw, st, half)));
}

}  // namespace dda
