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

// Per-thread accumulator for NV sums.  FP64 data accumulate in FP64.  FP32
// data (the inner solve's vectors) form their products and sum them in FP32
// over chunks of 8 elements, and the chunks accumulate in FP64: FP64
// arithmetic runs at 1/58 of the FP32 rate on this part, and a chunk of 8
// FP32 products carries a relative error below 8 * 2^-24.
template <typename T, int NV> struct ChunkAcc {
  double tot[NV];
  T part[NV];
  int cnt;
  __device__ __forceinline__ ChunkAcc() : cnt(0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) { tot[i] = 0.0; part[i] = (T)0; }
  }
  __device__ __forceinline__ void add(int k, T v) { part[k] += v; }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int i = 0; i < NV; ++i) { tot[i] += (double)part[i]; part[i] = (T)0; }
    cnt = 0;
  }
  __device__ __forceinline__ void step() {
    if (sizeof(T) == 8 || ++cnt == 8) flush();
  }
};

#define GRID_LOOP(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

}  // namespace dda
