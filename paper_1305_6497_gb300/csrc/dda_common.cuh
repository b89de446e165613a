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

// Complex type for a real type.
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im);
template <> __host__ __device__ __forceinline__ float2 mk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 mk<double2>(double re, double im) {
  return make_double2(re, im);
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
  const C* ainv;                  // [R][ncomp+1] alpha^{-1} per RHS, entry 0 unused
  int ncomp1;                     // ncomp + 1
  const C* twx; const C* twy; const C* twz;
  const int* kx_at; const int* ky_at; const int* kz_at;  // frequency held at each
                                                          // digit-reversed position
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
