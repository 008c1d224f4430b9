// FP32 instantiations of the batched stage kernel, and the per-step advance kernel.
#include "batch.cuh"

namespace hj {

cudaError_t launch_batch_stage_f32(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int ndim,
                                   int dynamics, int threads, size_t smem, cudaStream_t s) {
    HJ_BATCH_DISPATCH(float)
}

// After stage 3 of a step: count the step, load the next step's dt and the
// slice (if any) that the next step completes.
__global__ void batch_advance_kernel(BatchInst* insts, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    BatchInst& I = insts[i];
    if (I.k >= I.steps_total) return;
    const int k = ++I.k;
    I.slice_out = nullptr;
    if (k < I.steps_total) {
        I.dt = I.dts[k];
        I.dt_f = (float)I.dt;
        if (I.cursor < I.n_ends && I.ends[I.cursor] == (long long)k + 1) {
            I.slice_out = static_cast<char*>(I.out) + (size_t)I.end_slice[I.cursor] * (size_t)I.nodes * I.elem;
            I.cursor += 1;
        }
    }
}

cudaError_t launch_batch_advance(BatchInst* insts, int n, cudaStream_t s) {
    batch_advance_kernel<<<(n + 127) / 128, 128, 0, s>>>(insts, n);
    return cudaGetLastError();
}

}  // namespace hj
