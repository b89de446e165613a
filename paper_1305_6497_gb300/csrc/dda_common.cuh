// Shared device/host definitions for the GB300 DDA library.
//
// Layouts (all device memory):
//  - box vectors: [R][3][nz][ny][nx] complex (R right-hand sides, 3 Cartesian
//    components), zero on vacant sites;
//  - spectral scratch: [R][3][nz][Ly][Lx] complex.  The x pass fills rows
//    y < ny, the y pass expands each (z, column) to Ly rows in place, the fused
//    z pass transforms along z, multiplies by the Green tensor transform and
//    transforms back in place, and the inverse y and x passes shrink back;
//  - Green tensor transform: one octant [Lz/2+1][Ly/2+1][Lx/2+1][6] complex
//    (components xx, xy, xz, yy, yz, zz side by side), the rest follows from
//    the parity of each component in each axis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {

constexpr int kMaxStages = 12;
constexpr int kMaxComp = 256;

// ---- double-float ("df64") arithmetic ----------------------------------------
// A value is the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2),
// about 48 significant bits.  FP64 runs at 1/58 of the FP32 rate on this part,
// so FFT passes that need FP64-level accuracy (the refinement's residual
// A.x) run in this arithmetic instead.  Sums use Knuth's TwoSum and Dekker's
// Fast2Sum, products the FMA-based exact product (Dekker; Ogita, Rump & Oishi
// 2005); the absolute error of a sum is ~2^-48 (|a| + |b|), enough for an FFT.
// The _rn intrinsics keep the compiler from contracting or reassociating.
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};
__device__ __forceinline__ df64 df_fast2sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast2sum(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast2sum(p, e);
}
__host__ __device__ __forceinline__ double df_to_double(df64 a) {
  return (double)a.hi + (double)a.lo;
}
struct __align__(16) df64c { df64 x, y; };

// Complex type for a real type.
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<df64> { using type = df64c; };
template <typename T> using cplx_t = typename Cplx<T>::type;

// Type of the box vectors a matvec reads and writes (the FFT scratch is
// cplx_t<T>): df64 passes take and return FP64 vectors.
template <typename T> struct IoT { using type = cplx_t<T>; };
template <> struct IoT<df64> { using type = double2; };
template <typename T> using io_t = typename IoT<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im);
template <> __host__ __device__ __forceinline__ float2 mk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 mk<double2>(double re, double im) {
  return make_double2(re, im);
}
template <> __host__ __device__ __forceinline__ df64c mk<df64c>(double re, double im) {
  df64c r;
  r.x = df64(re);
  r.y = df64(im);
  return r;
}

// box-vector element <-> FFT element
template <typename C, typename IO> __device__ __forceinline__ C from_io(IO v) { return v; }
template <> __device__ __forceinline__ df64c from_io<df64c, double2>(double2 v) {
  df64c r;
  r.x = df64(v.x);
  r.y = df64(v.y);
  return r;
}
template <typename IO, typename C> __device__ __forceinline__ IO to_io(C v) { return v; }
template <> __device__ __forceinline__ double2 to_io<double2, df64c>(df64c v) {
  return make_double2(df_to_double(v.x), df_to_double(v.y));
}

// read-only load of a complex value (tables)
template <typename C> __device__ __forceinline__ C ldc(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ df64c ldc<df64c>(const df64c* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  df64c r;
  r.x = df64(v.x, v.y);
  r.y = df64(v.z, v.w);
  return r;
}

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
  C r; r.x = a.x + b.x; r.y = a.y + b.y; return r;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
  C r; r.x = a.x - b.x; r.y = a.y - b.y; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) {
  C r; r.x = a.x * s; r.y = a.y * s; return r;
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __host__ __device__ __forceinline__ C cmul_i(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// One 1-D transform of length L = prod(radix[t]), in place.  Stage t works on
// blocks of blk[t] points with span blk[t]/radix[t]; its twiddles are
// tw[tw_off[t] + j*(radix[t]-1) + (m-1)] = exp(-2 pi i j m / blk[t]).
struct AxisPlan {
  int L;
  int nstage;
  int radix[kMaxStages];
  int blk[kMaxStages];
  int tw_off[kMaxStages];
  unsigned long long sdiv[kMaxStages];  // ceil(2^36 / span): q / span = (q * sdiv) >> 36
  int tw_len;
};

// q / d with m = ceil(2^36 / d): exact whenever q d <= 2^36, since m d - 2^36
// is below d.
__host__ __device__ __forceinline__ int fast_div(int q, unsigned long long m) {
  return (int)(((unsigned long long)q * m) >> 36);
}

// Everything a matvec kernel needs about one target's operator.
template <typename T> struct OpView {
  using C = cplx_t<T>;
  int nx, ny, nz;                 // box
  int Lx, Ly, Lz;                 // FFT grid
  int Hx, Hy, Hz;                 // octant sizes L/2 + 1
  int64_t nbox;                   // nx*ny*nz
  const uint8_t* comp;            // [nbox] 0 = vacant, else composition 1..ncomp
  const C* ghat;                  // [Hz][Hy][Hx][6], already divided by Lx*Ly*Lz
  const C* ainv;                  // [R][ncomp+1][3] alpha^{-1} per RHS and lattice axis
                                  // (the polarizability tensor's diagonal), entry 0 unused
  int ncomp1;                     // ncomp + 1
  const C* twx; const C* twy; const C* twz;
  const int* kx_at; const int* ky_at; const int* kz_at;  // frequency held at each
                                                          // digit-reversed position
  const int* ypos_at;             // position holding each y frequency (inverse of ky_at)
  const float2* twz_pair;         // z twiddles of the column-pair kernel's plan (FP32), or null
  int* zerr;                      // set to 1 by a kernel whose bounded wait on a copy ran out
  unsigned long long div_nx, div_ny, div_nz, div_Lx;     // fast_div magics
  AxisPlan px, py, pz;
};

// ---- asynchronous global -> shared copies (cp.async) ------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// BYTES = 4, 8 or 16; both addresses aligned to BYTES
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst_smem, const void* src_gmem) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst_smem)),
                 "l"(src_gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst_smem)),
                 "l"(src_gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace dda
