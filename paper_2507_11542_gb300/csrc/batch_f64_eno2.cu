// FP64 instantiations of the batched stage kernel with second-order ENO.
#include "batch.cuh"

namespace hj {
cudaError_t launch_batch_stage_f64_eno2(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage,
                                        int ndim, int dynamics, int threads, size_t smem, cudaStream_t s) {
    HJ_BATCH_DISPATCH(launch_batch_eno2, double)
}
}  // namespace hj
