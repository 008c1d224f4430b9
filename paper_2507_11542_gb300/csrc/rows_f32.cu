// FP32 instantiations of the row-tiled stage kernel (WENO5 here, ENO2 in
// rows_f32_eno2.cu, ENO1 and ENO3 in rows_f32_eno13.cu).
#include "rows_kernel.cuh"

namespace hj {
cudaError_t launch_rows_f32_eno2(const StageParams& p, const RowsCfg& c, cudaStream_t s);
int rows_blocks_per_sm_f32_eno2(const StageParams& p, const RowsCfg& c);
cudaError_t launch_rows_f32_eno13(const StageParams& p, const RowsCfg& c, cudaStream_t s);
int rows_blocks_per_sm_f32_eno13(const StageParams& p, const RowsCfg& c);

cudaError_t launch_rows_f32_box(const StageParams& p, const RowsCfg& c, cudaStream_t s);
int rows_blocks_per_sm_f32_box(const StageParams& p, const RowsCfg& c);

cudaError_t launch_rows_f32(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    if (rows_box_variant(p)) return launch_rows_f32_box(p, c, s);
    if (p.scheme == HJ_ENO2) return launch_rows_f32_eno2(p, c, s);
    if (p.scheme == HJ_ENO1 || p.scheme == HJ_ENO3) return launch_rows_f32_eno13(p, c, s);
    HJ_ROWS_DISPATCH(launch_rows_weno5, float, p, c, s)
    return cudaErrorInvalidValue;
}
int rows_blocks_per_sm_f32(const StageParams& p, const RowsCfg& c) {
    if (rows_box_variant(p)) return rows_blocks_per_sm_f32_box(p, c);
    if (p.scheme == HJ_ENO2) return rows_blocks_per_sm_f32_eno2(p, c);
    if (p.scheme == HJ_ENO1 || p.scheme == HJ_ENO3) return rows_blocks_per_sm_f32_eno13(p, c);
    HJ_ROWS_DISPATCH(rows_bps_weno5, float, p, c)
    return 0;
}
}  // namespace hj
