// FP32 instantiations of the row-tiled stage kernel with first- and
// third-order ENO.
#include "rows_kernel.cuh"

namespace hj {
cudaError_t launch_rows_f32_eno13(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    if (p.scheme == HJ_ENO1) {
        HJ_ROWS_DISPATCH(launch_rows_eno1, float, p, c, s)
    } else {
        HJ_ROWS_DISPATCH(launch_rows_eno3, float, p, c, s)
    }
    return cudaErrorInvalidValue;
}
int rows_blocks_per_sm_f32_eno13(const StageParams& p, const RowsCfg& c) {
    if (p.scheme == HJ_ENO1) {
        HJ_ROWS_DISPATCH(rows_bps_eno1, float, p, c)
    } else {
        HJ_ROWS_DISPATCH(rows_bps_eno3, float, p, c)
    }
    return 0;
}
}  // namespace hj
