// FP32 instantiations of the row-tiled WENO5 stage kernel.
#include "rows_kernel.cuh"

namespace hj {
cudaError_t launch_rows_f32(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    HJ_ROWS_DISPATCH(launch_rows_dyn, float, p, c, s)
    return cudaErrorInvalidValue;
}
int rows_blocks_per_sm_f32(const StageParams& p, const RowsCfg& c) {
    HJ_ROWS_DISPATCH(rows_bps_dyn, float, p, c)
    return 0;
}
}  // namespace hj
