// FP64 instantiations of the fused stage and upwind kernels.
#include "stage_kernels.cuh"

namespace hj {
cudaError_t launch_stage_f64(const StageParams& p, int scheme, cudaStream_t s) {
    return launch_stage_t<double>(p, scheme, s);
}
cudaError_t launch_upwind_f64(const UpwindParams& p, int scheme, cudaStream_t s) {
    return launch_upwind_t<double>(p, scheme, s);
}
}  // namespace hj
