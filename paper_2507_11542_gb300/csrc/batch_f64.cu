// FP64 instantiations of the batched stage kernel.
#include "batch.cuh"

namespace hj {
cudaError_t launch_batch_stage_f64_eno2(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage,
                                        int ndim, int dynamics, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_batch_stage_f64_eno13(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage,
                                         int ndim, int dynamics, int scheme, int threads, size_t smem, cudaStream_t s);

cudaError_t launch_batch_stage_f64(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int ndim,
                                   int dynamics, int scheme, int threads, size_t smem, cudaStream_t s) {
    if (scheme == HJ_ENO2) return launch_batch_stage_f64_eno2(tiles, ntiles, insts, stage, ndim, dynamics, threads, smem, s);
    if (scheme == HJ_ENO1 || scheme == HJ_ENO3)
        return launch_batch_stage_f64_eno13(tiles, ntiles, insts, stage, ndim, dynamics, scheme, threads, smem, s);
    HJ_BATCH_DISPATCH(launch_batch_weno5, double)
}
}  // namespace hj
