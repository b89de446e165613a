// FFT-convolution matvec with FP64 box vectors and double-float FFT passes:
// the refinement's residual operator.  Kernels: matvec_impl.cuh.
#include "matvec_impl.cuh"

namespace dda {

cudaError_t launch_matvec_df(const OpView<df64>& op, const MatvecLaunch& L, int R,
                             const double2* x, double2* y, df64c* scratch, const int* active,
                             cudaStream_t st, const cudaEvent_t* ev) {
  // the x and y schedule of the FP64 passes (same element size); the z pass
  // has one variant here: 4 columns, Ghat read from global memory
  MatvecLaunch Ld = L;
  Ld.z_tile = 4;
  Ld.z_gs = false;
  Ld.z_ps = 3 * 4 + 1;
  Ld.z_smem = ((size_t)op.Lz * Ld.z_ps * sizeof(df64c) + 15) & ~(size_t)15;
  return matvec_passes<df64, XIN_PLAIN, XOUT_PLAIN>(op, Ld, R, x, y, scratch, active, st, ev,
                                                    XinArgs<df64>{}, nullptr, nullptr);
}

cudaError_t configure_matvec_kernels_df() {
  const void* k[] = {(const void*)k_fft_x_fwd<df64, XIN_PLAIN>,
                     (const void*)k_fft_x_inv<df64, XOUT_PLAIN>,
                     (const void*)k_fft_y<df64, false>, (const void*)k_fft_y<df64, true>,
                     (const void*)k_fft_z_mul<df64, 4, false>};
  for (const void* f : k) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               200 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dda
