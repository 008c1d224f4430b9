// FP64 instantiations of the row-tiled stage kernel with Lax-Friedrichs
// dissipation local in p (HJ_ALPHA_BOX), every scheme, for the dynamics whose
// slopes depend on p (norm in 2-D and 3-D, air3D, rockets).
#include "rows_kernel.cuh"

namespace hj {
cudaError_t launch_rows_f64_box(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    switch (p.scheme) {
    case HJ_ENO1: HJ_ROWS_BOX_DISPATCH(launch_rows_eno1, double, p, c, s) break;
    case HJ_ENO2: HJ_ROWS_BOX_DISPATCH(launch_rows_eno2, double, p, c, s) break;
    case HJ_ENO3: HJ_ROWS_BOX_DISPATCH(launch_rows_eno3, double, p, c, s) break;
    default: HJ_ROWS_BOX_DISPATCH(launch_rows_weno5, double, p, c, s) break;
    }
    return cudaErrorInvalidValue;
}
int rows_blocks_per_sm_f64_box(const StageParams& p, const RowsCfg& c) {
    switch (p.scheme) {
    case HJ_ENO1: HJ_ROWS_BOX_DISPATCH(rows_bps_eno1, double, p, c) break;
    case HJ_ENO2: HJ_ROWS_BOX_DISPATCH(rows_bps_eno2, double, p, c) break;
    case HJ_ENO3: HJ_ROWS_BOX_DISPATCH(rows_bps_eno3, double, p, c) break;
    default: HJ_ROWS_BOX_DISPATCH(rows_bps_weno5, double, p, c) break;
    }
    return 0;
}
}  // namespace hj
