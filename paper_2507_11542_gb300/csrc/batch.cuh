// batch.cuh -- the batched stage kernel: one launch advances one RK3 stage of
// every active instance of a batch. Each block owns one tile (a few full
// rows of one instance, through a chunk of planes) and runs the same tile
// body as the single-solve row kernel, with the instance's grid, dynamics,
// buffers and current dt read from its device descriptor.
#pragma once

#include "rows_kernel.cuh"

namespace hj {

template <typename T>
__device__ __forceinline__ T batch_dt(const BatchInst& I);
template <> __device__ __forceinline__ double batch_dt<double>(const BatchInst& I) { return I.dt; }
template <> __device__ __forceinline__ float batch_dt<float>(const BatchInst& I) { return I.dt_f; }

// KIND: kKindFirst for stage 1, kKindCombine for stages 2 and 3.
template <typename T, int D, int DYN, int SCHEME, int KIND>
__global__ void __launch_bounds__(RowsLimits<T>::kMaxThreads)
    batch_kernel(const BatchTile* __restrict__ tiles, const BatchInst* __restrict__ insts, const int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchTile t = tiles[blockIdx.x];
    const BatchInst& I = insts[t.inst];
    if (I.k >= I.steps_total) return;  // this instance has finished (block-uniform)
    StageRun<T> R;
    R.dt = batch_dt<T>(I);
    R.brt0 = I.brt == HJ_BRT_MIN0;
    R.also_out = nullptr;
    R.minv = false;
    if (stage == 1) {
        R.u = static_cast<const T*>(I.V);
        R.vn = nullptr;
        R.out = static_cast<T*>(I.V1);
        R.cv = T(0);
        R.cu = T(1);
    } else if (stage == 2) {
        R.u = static_cast<const T*>(I.V1);
        R.vn = static_cast<const T*>(I.V);
        R.out = static_cast<T*>(I.V2);
        R.cv = T(0.75);
        R.cu = T(0.25);
    } else {
        R.u = static_cast<const T*>(I.V2);
        R.vn = static_cast<const T*>(I.V);
        R.out = static_cast<T*>(I.V);
        R.also_out = static_cast<T*>(I.slice_out);
        R.cv = T(1.0 / 3.0);
        R.cu = T(2.0 / 3.0);
        R.minv = I.brt == HJ_BRT_MINV;
    }
    rows_tile<T, D, DYN, SCHEME, KIND>(I.P, R, I.ty, (int)blockDim.x, I.tz, t.row_tile, t.i2, t.chunk,
                                       (int)threadIdx.x, reinterpret_cast<T*>(smem_raw));
}

template <typename T, int D, int DYN, int SCHEME, int KIND>
cudaError_t launch_batch_kind(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int threads,
                              size_t smem, cudaStream_t s) {
    static std::atomic<unsigned long long> done{0};
    cudaError_t e = smem_optin(batch_kernel<T, D, DYN, SCHEME, KIND>, done);
    if (e != cudaSuccess) return e;
    batch_kernel<T, D, DYN, SCHEME, KIND><<<ntiles, threads, smem, s>>>(tiles, insts, stage);
    return cudaGetLastError();
}

template <typename T, int D, int DYN, int SCHEME>
cudaError_t launch_batch_scheme(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int threads,
                                size_t smem, cudaStream_t s) {
    return stage == 1
               ? launch_batch_kind<T, D, DYN, SCHEME, kKindFirst>(tiles, ntiles, insts, stage, threads, smem, s)
               : launch_batch_kind<T, D, DYN, SCHEME, kKindCombine>(tiles, ntiles, insts, stage, threads, smem, s);
}
template <typename T, int D, int DYN>
cudaError_t launch_batch_weno5(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int threads,
                               size_t smem, cudaStream_t s) {
    return launch_batch_scheme<T, D, DYN, HJ_WENO5>(tiles, ntiles, insts, stage, threads, smem, s);
}
template <typename T, int D, int DYN>
cudaError_t launch_batch_eno2(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int threads,
                              size_t smem, cudaStream_t s) {
    return launch_batch_scheme<T, D, DYN, HJ_ENO2>(tiles, ntiles, insts, stage, threads, smem, s);
}

template <typename T, int D, int DYN>
cudaError_t launch_batch_eno1(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int threads,
                              size_t smem, cudaStream_t s) {
    return launch_batch_scheme<T, D, DYN, HJ_ENO1>(tiles, ntiles, insts, stage, threads, smem, s);
}
template <typename T, int D, int DYN>
cudaError_t launch_batch_eno3(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int threads,
                              size_t smem, cudaStream_t s) {
    return launch_batch_scheme<T, D, DYN, HJ_ENO3>(tiles, ntiles, insts, stage, threads, smem, s);
}

#define HJ_BATCH_DISPATCH(FN, T)                                                                                   \
    switch (ndim * 16 + dynamics) {                                                                            \
    case 2 * 16 + HJ_DYN_DOUBLE_INTEGRATOR:                                                                    \
        return FN<T, 2, HJ_DYN_DOUBLE_INTEGRATOR>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 2 * 16 + HJ_DYN_NORM: return FN<T, 2, HJ_DYN_NORM>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 2 * 16 + HJ_DYN_ADVECT: return FN<T, 2, HJ_DYN_ADVECT>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 2 * 16 + HJ_DYN_ROTATE: return FN<T, 2, HJ_DYN_ROTATE>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 3 * 16 + HJ_DYN_AIR3D: return FN<T, 3, HJ_DYN_AIR3D>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 3 * 16 + HJ_DYN_ROCKETS: return FN<T, 3, HJ_DYN_ROCKETS>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 3 * 16 + HJ_DYN_NORM: return FN<T, 3, HJ_DYN_NORM>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 3 * 16 + HJ_DYN_ADVECT: return FN<T, 3, HJ_DYN_ADVECT>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 3 * 16 + HJ_DYN_ROTATE: return FN<T, 3, HJ_DYN_ROTATE>(tiles, ntiles, insts, stage, threads, smem, s); \
    case 4 * 16 + HJ_DYN_DUBINS4D: return FN<T, 4, HJ_DYN_DUBINS4D>(tiles, ntiles, insts, stage, threads, smem, s); \
    default: return cudaErrorInvalidValue;                                                                     \
    }

}  // namespace hj
