// Autotuning of the launch schedule of the FFT-matvec passes (host code that
// times the kernels of matvec_impl.cuh on live buffers).
#pragma once

#include "matvec_impl.cuh"

namespace dda {

// --------------------------------------------------------------------------
// autotuning of the launch schedule (tiles, lines, row pitch, Ghat staging)
// --------------------------------------------------------------------------
template <typename T>
static void fill_x(const OpView<T>& op, MatvecLaunch& L, int nl) {
  using C = cplx_t<T>;
  L.x_lines = nl;
  L.x_smem = (size_t)op.Lx * (nl + 1) * sizeof(C);
  L.xinv_smem = x_inv_smem_bytes(op.Lx, nl, op.nx, sizeof(C));
}
template <typename T>
static void fill_y(const OpView<T>& op, MatvecLaunch& L, int tile) {
  L.y_tile = tile;
  L.y_smem = (size_t)op.Ly * tile * sizeof(cplx_t<T>);
}
template <typename T>
static void fill_z(const OpView<T>& op, MatvecLaunch& L, int tile, int pad, bool gs) {
  using C = cplx_t<T>;
  L.z_tile = tile;
  L.z_ps = 3 * tile + pad;
  L.z_gs = gs;
  L.z_smem = (((size_t)op.Lz * L.z_ps * sizeof(C) + 15) & ~(size_t)15) +
             (gs ? (size_t)6 * op.Hz * tile * sizeof(C) : 0);
}

// Launch one pass `reps` times between two events; returns the mean in ms.
template <typename T>
// The x passes are timed in their fused forms (a vector-update prologue, an
// inner-product epilogue), which read more than the plain ones.
static float time_pass(const OpView<T>& op, const MatvecLaunch& L, int pass, int R,
                       const cplx_t<T>* x, cplx_t<T>* y, cplx_t<T>* scratch, cudaStream_t st,
                       cudaEvent_t e0, cudaEvent_t e1, int reps, const KState* ks,
                       double* part, FoldArgs fold) {
  auto launch = [&]() {
    switch (pass) {
      case 0: {
        XinArgs<T> xa{x, y, x, ks, nullptr, nullptr};  // s <- x - alpha x, into y
        launch_x_fwd_pass<T, XIN_S>(op, L, R, x, scratch, nullptr, xa, st);
        break;
      }
      case 1: launch_y_pass<T, false>(op, L, R, scratch, nullptr, st); break;
      case 2: launch_z_pass<T, false>(op, L, R, scratch, nullptr, st); break;
      case 3: launch_y_pass<T, true>(op, L, R, scratch, nullptr, st); break;
      default:  // with the scalar step its sums feed, as in the solves
        launch_x_inv_pass<T, XOUT_RV>(op, L, R, scratch, x, y, nullptr, x, part, st, fold);
    }
  };
  launch();  // warm-up
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps; ++i) launch();
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) return 1e30f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / reps;
}

template <typename T>
cudaError_t autotune_matvec(const OpView<T>& op, MatvecLaunch& L, int R, const cplx_t<T>* x,
                            cplx_t<T>* y, cplx_t<T>* scratch, cudaStream_t st) {
  using C = cplx_t<T>;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  // a zero Krylov state (alpha = 0) and partial sums for the fused x passes,
  // sized for the smallest line count tried (2 lines per CTA)
  // (and the tuner's own counters, group sums and active flags for the scalar
  // step the inverse x pass finishes; the step writes only these buffers)
  KState* ks = nullptr;
  double* part = nullptr;
  char* fb = nullptr;
  int* act = nullptr;
  const size_t nks = sizeof(KState) * (size_t)R;
  const size_t npart = sizeof(double) * 2 * (size_t)R * (3 * (size_t)op.nz * op.ny / 2 + 1);
  e = cudaMalloc(&ks, nks);
  if (e == cudaSuccess) e = cudaMalloc(&part, npart);
  if (e == cudaSuccess) e = cudaMalloc(&fb, fold_bytes(R));
  if (e == cudaSuccess) e = cudaMalloc(&act, sizeof(int) * (size_t)R);
  if (e == cudaSuccess) e = cudaMemsetAsync(ks, 0, nks, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(fb, 0, fold_gsum_offset(R), st);
  if (e != cudaSuccess) {
    cudaFree(ks); cudaFree(part); cudaFree(fb); cudaFree(act);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    return e;
  }
  const FoldArgs fold{ks, act, reinterpret_cast<unsigned*>(fb), FOLD_ALPHA,
                      reinterpret_cast<double*>(fb + fold_gsum_offset(R))};
  const int reps = 6;
  const size_t kMax = 200 * 1024;
  MatvecLaunch best = L;
  // Thread counts are tuned with the tiles: a CTA's stages have different
  // numbers of butterflies (e.g. 128-point lines as 16 x 8), and threads left
  // without one wait at the stage's barrier.
  // x passes (forward and inverse together)
  {
    float bt = time_pass<T>(op, best, 0, R, x, y, scratch, st, e0, e1, reps, ks, part, fold) +
               time_pass<T>(op, best, 4, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
    for (int nl : {2, 4, 8, 16, 32, 64})
      for (int th : {64, 96, 128, 192, 256}) {
        MatvecLaunch c = best;
        fill_x<T>(op, c, nl);
        c.x_threads = th;
        if (c.xinv_smem > kMax || nl > 3 * op.nz * op.ny) continue;
        const float tt = time_pass<T>(op, c, 0, R, x, y, scratch, st, e0, e1, reps, ks, part, fold) +
                         time_pass<T>(op, c, 4, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
        if (tt < bt) { bt = tt; best = c; }
      }
  }
  // y passes
  {
    float bt = time_pass<T>(op, best, 1, R, x, y, scratch, st, e0, e1, reps, ks, part, fold) +
               time_pass<T>(op, best, 3, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
    for (int tile : {2, 4, 8, 16, 32})
      for (int th : {64, 96, 128, 192, 256}) {
        MatvecLaunch c = best;
        fill_y<T>(op, c, tile);
        c.y_threads = th;
        if (c.y_smem > kMax) continue;
        const float tt = time_pass<T>(op, c, 1, R, x, y, scratch, st, e0, e1, reps, ks, part, fold) +
                         time_pass<T>(op, c, 3, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
        if (tt < bt) { bt = tt; best = c; }
      }
  }
  // z pass
  {
    float bt = time_pass<T>(op, best, 2, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
    for (int tile : {2, 4, 8, 16})
      for (int gs = 0; gs < 2; ++gs)
        for (int pad = 0; pad < 4; ++pad)
          for (int th : {64, 96, 128, 192, 256, 384}) {
            MatvecLaunch c = best;
            fill_z<T>(op, c, tile, pad, gs != 0);
            c.z_pair = 0;
            // a compiled-plan z kernel sets its own pitch: one pad value is enough
            if (std::is_same<T, float>::value && z_fixed_plan(op.pz) && pad != 0) continue;
            // 384 threads: compiled-plan z kernels only
            if (th > 256 && !(std::is_same<T, float>::value && z_fixed_applies(op.pz, tile)))
              continue;
            c.z_threads = th;
            if (c.z_smem > kMax) continue;
            if (std::is_same<T, float>::value && z_fixed_applies(op.pz, tile)) {
              // the compiled kernel's own pitch (see zc_pitch)
              const int pc = 3 * tile + (tile * 8 < 128 ? 1 : 0);
              const size_t zc = (((size_t)op.Lz * pc * 8 + 15) & ~(size_t)15) +
                                (gs ? (size_t)6 * op.Hz * tile * 8 : 0);
              if (zc > kMax) continue;
            }
            const float tt = time_pass<T>(op, c, 2, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
            if (tt < bt) { bt = tt; best = c; }
          }
    // the column-pair kernel (FP32, compiled z plans)
    if (std::is_same<T, float>::value)
      for (int tile : {4, 8})
        for (int gs = 0; gs < 2; ++gs)
        for (int tma = 0; tma < 2; ++tma) {
          const int th = kZPairThreads;
          if (!z_pair_applies(op.Lz, op.Lx, tile)) continue;
          if (tma && !z_pair_tma_applies(op.Lz, op.Lx, op.nz, tile)) continue;
          const size_t zs = zpair_smem_bytes(op.Lz, tile, gs != 0);
          if (zs > kMax) continue;
          MatvecLaunch c = best;
          fill_z<T>(op, c, tile, 0, gs != 0);
          c.z_pair = tma ? 2 : 1;
          c.z_smem = zs;
          c.z_threads = th;
          const float tt = time_pass<T>(op, c, 2, R, x, y, scratch, st, e0, e1, reps, ks, part, fold);
          if (tt < bt) { bt = tt; best = c; }
        }
  }
  (void)sizeof(C);
  cudaStreamSynchronize(st);
  cudaFree(ks);
  cudaFree(part);
  cudaFree(fb);
  cudaFree(act);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L = best;
  return cudaGetLastError();
}

}  // namespace dda
