// FFT-convolution matvec and its fused Krylov variants in FP32 (the inner
// solve of the refined precision mode).  Kernels: matvec_impl.cuh.
#include "matvec_impl.cuh"
#include "matvec_tune.cuh"

namespace dda {

template cudaError_t autotune_matvec<float>(const OpView<float>&, MatvecLaunch&, int,
                                            const float2*, float2*, float2*, cudaStream_t);
template MatvecLaunch plan_matvec<float>(const OpView<float>&);
template cudaError_t configure_matvec_kernels<float>(const MatvecLaunch&);
template int matvec_partial_blocks<float>(const OpView<float>&, const MatvecLaunch&);
template cudaError_t launch_matvec_p<float>(const OpView<float>&, const MatvecLaunch&, int,
                                            const float2*, float2*, float2*, const float2*,
                                            float2*, const KState*, double*, const int*,
                                            cudaStream_t, const cudaEvent_t*, FoldArgs);
template cudaError_t launch_matvec_s<float>(const OpView<float>&, const MatvecLaunch&, int,
                                            const float2*, const float2*, float2*, float2*,
                                            float2*, const KState*, double*, const int*,
                                            cudaStream_t, const cudaEvent_t*, FoldArgs);
template cudaError_t launch_matvec_q<float>(const OpView<float>&, const MatvecLaunch&, int,
                                            const float2*, float2*, float2*, float2*, float2*,
                                            float2*, const KState*, double*, const int*,
                                            cudaStream_t, const cudaEvent_t*, FoldArgs);
template cudaError_t launch_matvec<float>(const OpView<float>&, const MatvecLaunch&, int,
                                          const float2*, float2*, float2*, const int*,
                                          cudaStream_t, const cudaEvent_t*);

template cudaError_t launch_matvec_rv<float>(const OpView<float>&, const MatvecLaunch&, int,
                                            const float2*, float2*, const float2*, float2*, double*,
                                            const int*, cudaStream_t, const cudaEvent_t*);

}  // namespace dda
