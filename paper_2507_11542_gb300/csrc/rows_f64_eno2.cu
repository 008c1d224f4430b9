// FP64 instantiations of the row-tiled stage kernel with second-order ENO.
#include "rows_kernel.cuh"

namespace hj {
cudaError_t launch_rows_f64_eno2(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    HJ_ROWS_DISPATCH(launch_rows_eno2, double, p, c, s)
    return cudaErrorInvalidValue;
}
int rows_blocks_per_sm_f64_eno2(const StageParams& p, const RowsCfg& c) {
    HJ_ROWS_DISPATCH(rows_bps_eno2, double, p, c)
    return 0;
}
}  // namespace hj
