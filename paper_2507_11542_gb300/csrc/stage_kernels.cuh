// stage_kernels.cuh -- the fused RK stage kernel (Sec. 3-5): for every node,
// ghost-aware 7-point gathers along each dimension, upwind p-/p+ (ENO or
// WENO5), Lax-Friedrichs Hamiltonian, BRT clamp and the TVD-RK3 stage
// combination, in one pass. Included by one translation unit per element type.
#pragma once

#include "stencil.cuh"

namespace hj {

constexpr int kBX = 32, kBY = 8;

// One thread per node. Threads span (i0, i1); blockIdx.z strides over the
// combined index of dimensions 2 and 3.
template <typename T, int D, int SCHEME>
__global__ void __launch_bounds__(kBX * kBY) stage_kernel(const StageParams P) {
    const GridDev& g = P.g;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int i1 = (D > 1) ? (int)(blockIdx.y * blockDim.y + threadIdx.y) : 0;
    if (i0 >= g.n[0] || (D > 1 && i1 >= g.n[1])) return;
    const int nz = (D > 2 ? g.n[2] : 1) * (D > 3 ? g.n[3] : 1);
    const T* __restrict__ u = static_cast<const T*>(P.u);
    const T* __restrict__ vn = static_cast<const T*>(P.vn);
    T* __restrict__ out = static_cast<T*>(P.out);
    for (int z = blockIdx.z; z < nz; z += gridDim.z) {
        int idx[4] = {i0, i1, 0, 0};
        if (D > 2) { idx[2] = z % g.n[2]; }
        if (D > 3) { idx[3] = z / g.n[2]; }
        long long flat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) flat += (long long)idx[d] * g.stride[d];
        T pm[D], pp[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            T v[7];
            gather7<T>(u, flat, idx[d], g.n[d], g.stride[d], (g.periodic_mask >> d) & 1u, g.extrap, v);
            upwind_pair<T, SCHEME>(v, g.dx[d], g.inv_dx[d], SP<T>::floor(P, d), pm[d], pp[d]);
        }
        T y = lf_term<T, D>(P, idx, pm, pp);
        if (P.brt_min0) y = fmin(y, T(0));
        T r;
        if (P.mode == kTerm) {
            r = y;
        } else {
            const T w = ld(u + flat) + SP<T>::dt(P) * y;
            r = w;
            if (P.has_vn) {
                const T vv = ld(vn + flat);
                if (P.cv != 0.0) r = SP<T>::cv(P) * vv + SP<T>::cu(P) * w;
                if (P.minv_after) r = fmin(r, vv);
            }
        }
        out[flat] = r;
    }
}

template <typename T, int D, int SCHEME>
__global__ void __launch_bounds__(kBX * kBY) upwind_kernel(const UpwindParams P) {
    const GridDev& g = P.g;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int i1 = (D > 1) ? (int)(blockIdx.y * blockDim.y + threadIdx.y) : 0;
    if (i0 >= g.n[0] || (D > 1 && i1 >= g.n[1])) return;
    const int nz = (D > 2 ? g.n[2] : 1) * (D > 3 ? g.n[3] : 1);
    const T* __restrict__ u = static_cast<const T*>(P.u);
    for (int z = blockIdx.z; z < nz; z += gridDim.z) {
        int idx[4] = {i0, i1, 0, 0};
        if (D > 2) { idx[2] = z % g.n[2]; }
        if (D > 3) { idx[3] = z / g.n[2]; }
        long long flat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) flat += (long long)idx[d] * g.stride[d];
        const int d = P.dim;
        T v[7], pm, pp;
        gather7<T>(u, flat, idx[d], g.n[d], g.stride[d], (g.periodic_mask >> d) & 1u, g.extrap, v);
        upwind_pair<T, SCHEME>(v, g.dx[d], g.inv_dx[d], T(P.weno_floor), pm, pp);
        static_cast<T*>(P.pm)[flat] = pm;
        static_cast<T*>(P.pp)[flat] = pp;
    }
}

inline void launch_shape(const GridDev& g, dim3& grid, dim3& block) {
    if (g.ndim == 1) {
        block = dim3(kBX * kBY, 1, 1);
        grid = dim3((unsigned)((g.n[0] + kBX * kBY - 1) / (kBX * kBY)), 1, 1);
        return;
    }
    block = dim3(kBX, kBY, 1);
    long long nz = 1;
    for (int d = 2; d < g.ndim; ++d) nz *= g.n[d];
    grid = dim3((unsigned)((g.n[0] + kBX - 1) / kBX), (unsigned)((g.n[1] + kBY - 1) / kBY),
                (unsigned)(nz < 65535 ? nz : 65535));
}

template <typename T, int SCHEME>
cudaError_t launch_stage_scheme(const StageParams& p, cudaStream_t s) {
    dim3 grid, block;
    launch_shape(p.g, grid, block);
    switch (p.g.ndim) {
    case 1: stage_kernel<T, 1, SCHEME><<<grid, block, 0, s>>>(p); break;
    case 2: stage_kernel<T, 2, SCHEME><<<grid, block, 0, s>>>(p); break;
    case 3: stage_kernel<T, 3, SCHEME><<<grid, block, 0, s>>>(p); break;
    case 4: stage_kernel<T, 4, SCHEME><<<grid, block, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage_t(const StageParams& p, int scheme, cudaStream_t s) {
    switch (scheme) {
    case HJ_ENO1: return launch_stage_scheme<T, HJ_ENO1>(p, s);
    case HJ_ENO2: return launch_stage_scheme<T, HJ_ENO2>(p, s);
    case HJ_ENO3: return launch_stage_scheme<T, HJ_ENO3>(p, s);
    case HJ_WENO5: return launch_stage_scheme<T, HJ_WENO5>(p, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int SCHEME>
cudaError_t launch_upwind_scheme(const UpwindParams& p, cudaStream_t s) {
    dim3 grid, block;
    launch_shape(p.g, grid, block);
    switch (p.g.ndim) {
    case 1: upwind_kernel<T, 1, SCHEME><<<grid, block, 0, s>>>(p); break;
    case 2: upwind_kernel<T, 2, SCHEME><<<grid, block, 0, s>>>(p); break;
    case 3: upwind_kernel<T, 3, SCHEME><<<grid, block, 0, s>>>(p); break;
    case 4: upwind_kernel<T, 4, SCHEME><<<grid, block, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_upwind_t(const UpwindParams& p, int scheme, cudaStream_t s) {
    switch (scheme) {
    case HJ_ENO1: return launch_upwind_scheme<T, HJ_ENO1>(p, s);
    case HJ_ENO2: return launch_upwind_scheme<T, HJ_ENO2>(p, s);
    case HJ_ENO3: return launch_upwind_scheme<T, HJ_ENO3>(p, s);
    case HJ_WENO5: return launch_upwind_scheme<T, HJ_WENO5>(p, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hj
