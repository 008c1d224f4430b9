// FP64 instantiations of the row-tiled stage kernel (WENO5 here, ENO2 in
// rows_f64_eno2.cu, ENO1 and ENO3 in rows_f64_eno13.cu), and the
// (dimension, dynamics) pairs it is built for.
#include "rows_kernel.cuh"

namespace hj {
bool rows_supported(int ndim, int dyn) {
    switch (ndim * 16 + dyn) {
    case 2 * 16 + HJ_DYN_DOUBLE_INTEGRATOR:
    case 2 * 16 + HJ_DYN_NORM:
    case 2 * 16 + HJ_DYN_ADVECT:
    case 2 * 16 + HJ_DYN_ROTATE:
    case 3 * 16 + HJ_DYN_AIR3D:
    case 3 * 16 + HJ_DYN_ROCKETS:
    case 3 * 16 + HJ_DYN_NORM:
    case 3 * 16 + HJ_DYN_ADVECT:
    case 3 * 16 + HJ_DYN_ROTATE:
    case 4 * 16 + HJ_DYN_DUBINS4D:
        return true;
    default:
        return false;
    }
}
cudaError_t launch_rows_f64_eno2(const StageParams& p, const RowsCfg& c, cudaStream_t s);
int rows_blocks_per_sm_f64_eno2(const StageParams& p, const RowsCfg& c);
cudaError_t launch_rows_f64_eno13(const StageParams& p, const RowsCfg& c, cudaStream_t s);
int rows_blocks_per_sm_f64_eno13(const StageParams& p, const RowsCfg& c);

cudaError_t launch_rows_f64_box(const StageParams& p, const RowsCfg& c, cudaStream_t s);
int rows_blocks_per_sm_f64_box(const StageParams& p, const RowsCfg& c);

cudaError_t launch_rows_f64(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    if (rows_box_variant(p)) return launch_rows_f64_box(p, c, s);
    if (p.scheme == HJ_ENO2) return launch_rows_f64_eno2(p, c, s);
    if (p.scheme == HJ_ENO1 || p.scheme == HJ_ENO3) return launch_rows_f64_eno13(p, c, s);
    HJ_ROWS_DISPATCH(launch_rows_weno5, double, p, c, s)
    return cudaErrorInvalidValue;
}
int rows_blocks_per_sm_f64(const StageParams& p, const RowsCfg& c) {
    if (rows_box_variant(p)) return rows_blocks_per_sm_f64_box(p, c);
    if (p.scheme == HJ_ENO2) return rows_blocks_per_sm_f64_eno2(p, c);
    if (p.scheme == HJ_ENO1 || p.scheme == HJ_ENO3) return rows_blocks_per_sm_f64_eno13(p, c);
    HJ_ROWS_DISPATCH(rows_bps_weno5, double, p, c)
    return 0;
}
}  // namespace hj
