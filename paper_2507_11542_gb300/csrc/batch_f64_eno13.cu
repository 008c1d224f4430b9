// FP64 instantiations of the batched stage kernel with first- and third-order ENO.
#include "batch.cuh"

namespace hj {
cudaError_t launch_batch_stage_f64_eno13(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage,
                                         int ndim, int dynamics, int scheme, int threads, size_t smem, cudaStream_t s) {
    if (scheme == HJ_ENO1) {
        HJ_BATCH_DISPATCH(launch_batch_eno1, double)
    }
    HJ_BATCH_DISPATCH(launch_batch_eno3, double)
}
}  // namespace hj
