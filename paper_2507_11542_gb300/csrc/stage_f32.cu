// FP32 instantiations of the fused stage and upwind kernels.
#include "stage_kernels.cuh"

namespace hj {
cudaError_t launch_stage_f32(const StageParams& p, int scheme, cudaStream_t s) {
    return launch_stage_t<float>(p, scheme, s);
}
cudaError_t launch_upwind_f32(const UpwindParams& p, int scheme, cudaStream_t s) {
    return launch_upwind_t<float>(p, scheme, s);
}
}  // namespace hj
