// Deterministic block reductions in FP64 (internal).
#pragma once

#include "dda_common.cuh"

namespace dda {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the block; thread 0 gets the totals in out[].
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (&out)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) sh[i][w] = s;
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? sh[i][lane] : 0.0;
      s = warp_sum(s);
      out[i] = s;
    }
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void write_partials(double (&acc)[NV], double* partials) {
  double tot[NV];
  block_sum<NV>(acc, tot);
  if (threadIdx.x == 0) {
    double* o = partials + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * NV;
#pragma unroll
    for (int i = 0; i < NV; ++i) o[i] = tot[i];
  }
}

// Fixed-order sum of the partials of RHS r (one block per RHS).
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, int nblk, int r,
                                             double (&tot)[NV]) {
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  const double* p = partials + (int64_t)r * nblk * NV;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += p[(int64_t)b * NV + i];
  }
  block_sum<NV>(acc, tot);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 tree over the block; thread 0 gets the totals.  Used only for the FP32
// inner solve's sums: FP64 arithmetic runs at 1/58 of the FP32 rate on this
// part, and an FP64 shuffle tree over every warp of every block costs more
// issue time on the FP64 pipe than the vector pass it closes.
template <int NV>
__device__ __forceinline__ void block_sum_f(float (&v)[NV], float (&out)[NV]) {
  __shared__ float shf[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float s = warp_sum_f(v[i]);
    if (lane == 0) shf[i][w] = s;
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float s = lane < nw ? shf[i][lane] : 0.0f;
      out[i] = warp_sum_f(s);
    }
  }
  __syncthreads();
}

// Per-RHS FP64 scalars as C.  For FP32 kernels the first N threads convert
// them and the block shares them through shared memory: the conversions issue
// on the slow FP64 pipe of this part, so one per block instead of one per
// thread.  Every thread of the block must reach the call.
template <typename C, int N>
__device__ __forceinline__ void block_scalars(const double2 (&v)[N], C (&out)[N]) {
  if constexpr (sizeof(C) == sizeof(double2)) {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = mk<C>(v[i].x, v[i].y);
  } else {
    __shared__ C sc[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (threadIdx.x == i) sc[i] = mk<C>(v[i].x, v[i].y);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = sc[i];
  }
}

// Per-thread accumulator for NV sums, closed by write<NOUT>(partials), which
// stores the block's first NOUT totals as FP64 partials (summed over the
// blocks in FP64, in a fixed order, by sum_partials).  FP64 data accumulate
// in FP64 throughout.  FP32 data (the inner solve's vectors) sum their
// products in FP32 over chunks of 8 elements, the chunks into a per-thread
// FP32 total, and the threads in an FP32 tree (5 levels per warp, up to 3
// across warps): for a thread holding k elements the relative error, against
// the sum of the magnitudes, stays below (k/8 + 15) 2^-24, about 1e-6 for
// the sizes solved, well inside what an FP32 Krylov iteration can use.
template <typename T, int NV> struct ChunkAcc;

template <int NV> struct ChunkAcc<double, NV> {
  double tot[NV];
  __device__ __forceinline__ ChunkAcc() {
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = 0.0;
  }
  __device__ __forceinline__ void add(int k, double v) { tot[k] += v; }
  __device__ __forceinline__ void step() {}
  template <int NOUT> __device__ __forceinline__ void write(double* partials) {
    static_assert(NOUT <= NV, "more outputs than sums");
    double v[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) v[i] = tot[i];
    write_partials<NOUT>(v, partials);
  }
};

template <int NV> struct ChunkAcc<float, NV> {
  float tot[NV], part[NV];
  int cnt;
  __device__ __forceinline__ ChunkAcc() : cnt(0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) { tot[i] = 0.0f; part[i] = 0.0f; }
  }
  __device__ __forceinline__ void add(int k, float v) { part[k] += v; }
  __device__ __forceinline__ void step() {
    if (++cnt == 8) {
#pragma unroll
      for (int i = 0; i < NV; ++i) { tot[i] += part[i]; part[i] = 0.0f; }
      cnt = 0;
    }
  }
  template <int NOUT> __device__ __forceinline__ void write(double* partials) {
    static_assert(NOUT <= NV, "more outputs than sums");
    float v[NOUT], out[NOUT];
#pragma unroll
    for (int i = 0; i < NOUT; ++i) v[i] = tot[i] + part[i];
    block_sum_f<NOUT>(v, out);
    if (threadIdx.x == 0) {
      double* o = partials + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * NOUT;
#pragma unroll
      for (int i = 0; i < NOUT; ++i) o[i] = (double)out[i];
    }
  }
};

#define GRID_LOOP(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

}  // namespace dda
