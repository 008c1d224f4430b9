// FP32 instantiations of the batched stage kernel, and the per-step advance kernel.
#include "batch.cuh"

namespace hj {

cudaError_t launch_batch_stage_f32_eno2(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage,
                                        int ndim, int dynamics, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_batch_stage_f32_eno13(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage,
                                         int ndim, int dynamics, int scheme, int threads, size_t smem, cudaStream_t s);

cudaError_t launch_batch_stage_f32(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int ndim,
                                   int dynamics, int scheme, int threads, size_t smem, cudaStream_t s) {
    if (scheme == HJ_ENO2) return launch_batch_stage_f32_eno2(tiles, ntiles, insts, stage, ndim, dynamics, threads, smem, s);
    if (scheme == HJ_ENO1 || scheme == HJ_ENO3)
        return launch_batch_stage_f32_eno13(tiles, ntiles, insts, stage, ndim, dynamics, scheme, threads, smem, s);
    HJ_BATCH_DISPATCH(launch_batch_weno5, float)
}

// After stage 3 of a step: count the step, and set up the next one. Every
// step uses dt_full except the one that completes a slice, which is clipped
// to land on the slice time (Listing 6) and also writes the slice output.
// Only instances of lanes lane_lo .. lane_hi took this step (the lane is
// tested first: other lanes' descriptors may be advancing concurrently).
__global__ void batch_advance_kernel(BatchInst* insts, int n, int lane_lo, int lane_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    BatchInst& I = insts[i];
    if (I.lane < lane_lo || I.lane > lane_hi) return;
    if (I.k >= I.steps_total) return;
    const int k = ++I.k;
    I.slice_out = nullptr;
    if (k < I.steps_total) {
        double dt = I.dt_full;
        if (I.cursor < I.n_ends && I.ends[I.cursor] == (long long)k + 1) {
            dt = I.end_dt[I.cursor];
            I.slice_out = static_cast<char*>(I.out) + (size_t)I.end_slice[I.cursor] * (size_t)I.nodes * I.elem;
            I.cursor += 1;
        }
        I.dt = dt;
        I.dt_f = (float)dt;
    }
}

cudaError_t launch_batch_advance(BatchInst* insts, int n, int lane_lo, int lane_hi, cudaStream_t s) {
    batch_advance_kernel<<<(n + 127) / 128, 128, 0, s>>>(insts, n, lane_lo, lane_hi);
    return cudaGetLastError();
}

}  // namespace hj
