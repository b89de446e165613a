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
template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = csub(a, b); a = cadd(a, b); b = t;
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C s02 = cadd(a0, a2), d02 = csub(a0, a2);
  C s13 = cadd(a1, a3), d13 = cmul_i<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C (&a)[8]) {
  using T = decltype(a[0].x);
  const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
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
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, w1); a[5] = csub(e1, w1);
  a[2] = cadd(e2, w2); a[6] = csub(e2, w2);
  a[3] = cadd(e3, w3); a[7] = csub(e3, w3);
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

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C (&v)[R]) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 5) dft5<INV>(v);
  else dft8<INV>(v);
}

// ---- one in-place stage ------------------------------------------------------
template <typename C, int R, bool INV>
__device__ __forceinline__ void fft_stage(C* s, int nlines, int pstride, int L, int B,
                                          const C* __restrict__ tw) {
  const int S = B / R;
  const int nb = nlines * (L / R);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = b % nlines, q = b / nlines;
    const int blk = q / S, j = q - blk * S;
    C* base = s + (blk * B + j) * pstride + line;
    C v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = base[i * S * pstride];
    if (!INV) {
      dft<R, false>(v);
      if (j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], __ldg(&tw[j * (R - 1) + (m - 1)]));
      }
    } else {
      if (j > 0) {
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmulc(__ldg(&tw[j * (R - 1) + (m - 1)]), v[m]);
      }
      dft<R, true>(v);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) base[i * S * pstride] = v[i];
  }
  __syncthreads();
}

template <typename C, bool INV, int R>
__device__ __forceinline__ void run_stage(C* s, int nlines, int pstride, const AxisPlan& P,
                                          int st, const C* __restrict__ tw) {
  fft_stage<C, R, INV>(s, nlines, pstride, P.L, P.blk[st], tw + P.tw_off[st]);
}

// Full transform of `nlines` lines in shared memory, in place.  Forward: natural
// -> digit-reversed; inverse (unnormalized): digit-reversed -> natural.
template <typename C, bool INV>
__device__ void fft_smem(C* s, int nlines, int pstride, const AxisPlan& P,
                         const C* __restrict__ tw) {
  for (int k = 0; k < P.nstage; ++k) {
    const int st = INV ? P.nstage - 1 - k : k;
    switch (P.radix[st]) {
      case 8: run_stage<C, INV, 8>(s, nlines, pstride, P, st, tw); break;
      case 4: run_stage<C, INV, 4>(s, nlines, pstride, P, st, tw); break;
      case 2: run_stage<C, INV, 2>(s, nlines, pstride, P, st, tw); break;
      case 3: run_stage<C, INV, 3>(s, nlines, pstride, P, st, tw); break;
      default: run_stage<C, INV, 5>(s, nlines, pstride, P, st, tw); break;
    }
  }
}

}  // namespace dda
