// FFT-convolution matvec and its fused Krylov variants in FP64 (plain FP64
// solves, the Green-tensor setup transforms, the near field).  Kernels:
// matvec_impl.cuh.
#include "matvec_impl.cuh"
#include "matvec_tune.cuh"

namespace dda {

template cudaError_t autotune_matvec<double>(const OpView<double>&, MatvecLaunch&, int,
                                             const double2*, double2*, double2*, cudaStream_t);
template MatvecLaunch plan_matvec<double>(const OpView<double>&);
template cudaError_t configure_matvec_kernels<double>(const MatvecLaunch&);
template int matvec_partial_blocks<double>(const OpView<double>&, const MatvecLaunch&);
template cudaError_t launch_matvec_p<double>(const OpView<double>&, const MatvecLaunch&, int,
                                             const double2*, double2*, double2*,
                                             const double2*, double2*, const KState*, double*,
                                             const int*, cudaStream_t, const cudaEvent_t*, FoldArgs);
template cudaError_t launch_matvec_s<double>(const OpView<double>&, const MatvecLaunch&, int,
                                             const double2*, const double2*, double2*,
                                             double2*, double2*, const KState*, double*,
                                             const int*, cudaStream_t, const cudaEvent_t*, FoldArgs);
template cudaError_t launch_matvec_q<double>(const OpView<double>&, const MatvecLaunch&, int,
                                             const double2*, double2*, double2*, double2*,
                                             double2*, double2*, const KState*, double*,
                                             const int*, cudaStream_t, const cudaEvent_t*, FoldArgs);
template cudaError_t launch_matvec<double>(const OpView<double>&, const MatvecLaunch&, int,
                                           const double2*, double2*, double2*, const int*,
                                           cudaStream_t, const cudaEvent_t*);
template cudaError_t launch_field<double>(const OpView<double>&, const MatvecLaunch&, int,
                                          const double2*, double2*, double2*, cudaStream_t,
                                          bool);
template cudaError_t launch_x_fwd<double>(const OpView<double>&, const MatvecLaunch&, int,
                                          const double2*, double2*, cudaStream_t);

template cudaError_t launch_matvec_rv<double>(const OpView<double>&, const MatvecLaunch&, int,
                                            const double2*, double2*, const double2*, double2*, double*,
                                            const int*, cudaStream_t, const cudaEvent_t*);

}  // namespace dda
