// reduce.cu -- grid-wide reductions: the FP64 CFL bound (Sec. 4) and the
// non-finite check of value functions.
#include <cstdint>

#include "../../include/hj.h"
#include "hj_internal.h"

namespace hj {

// alpha_d(x), the maximum over the controls of |f_d| at the node, in FP64
// with every product and sum rounded separately (the plain left-to-right
// evaluation, bit for bit).
__device__ void node_alpha(const GridDev& g, int dyn, const double* q, const double* trig, const int* idx,
                           double* a) {
    double x[4];
    for (int d = 0; d < g.ndim; ++d) x[d] = __dadd_rn(g.lo[d], __dmul_rn((double)idx[d], g.dx[d]));
    for (int d = 0; d < 4; ++d) a[d] = 0.0;
    switch (dyn) {
    case HJ_DYN_DOUBLE_INTEGRATOR:
        a[0] = fabs(x[1]);
        a[1] = q[0];
        break;
    case HJ_DYN_AIR3D: {
        const double c = trig[idx[2]], s = trig[g.n[2] + idx[2]];
        a[0] = __dadd_rn(fabs(__dadd_rn(-q[0], __dmul_rn(q[1], c))), __dmul_rn(q[2], fabs(x[1])));
        a[1] = __dadd_rn(fabs(__dmul_rn(q[1], s)), __dmul_rn(q[2], fabs(x[0])));
        a[2] = __dadd_rn(q[2], q[3]);
        break;
    }
    case HJ_DYN_ROCKETS: {
        const double c = trig[idx[2]], s = trig[g.n[2] + idx[2]];
        a[0] = __dadd_rn(fabs(__dmul_rn(q[0], c)), __dmul_rn(q[2], fabs(x[0])));
        a[1] = __dadd_rn(fabs(__dadd_rn(__dadd_rn(__dmul_rn(q[0], s), q[0]), -q[1])), __dmul_rn(q[3], fabs(x[0])));
        a[2] = __dadd_rn(q[3], q[2]);
        break;
    }
    case HJ_DYN_DUBINS4D: {
        const double c = trig[idx[2]], s = trig[g.n[2] + idx[2]];
        a[0] = fabs(__dmul_rn(x[3], c));
        a[1] = fabs(__dmul_rn(x[3], s));
        a[2] = q[0];
        a[3] = q[1];
        break;
    }
    case HJ_DYN_NORM:
        for (int d = 0; d < g.ndim; ++d) a[d] = q[0];
        break;
    case HJ_DYN_ADVECT:
        for (int d = 0; d < g.ndim; ++d) a[d] = fabs(q[d]);
        break;
    case HJ_DYN_ROTATE:
        a[0] = fabs(__dmul_rn(q[0], x[1]));
        a[1] = fabs(__dmul_rn(q[0], x[0]));
        break;
    default:
        break;
    }
}

// alpha_d(x)/dx_d summed over d in the order alpha_0/dx_0 + alpha_1/dx_1 + ...
__device__ double node_bound(const GridDev& g, int dyn, const double* q, const double* trig, const int* idx) {
    double a[4];
    node_alpha(g, dyn, q, trig, idx, a);
    double s = 0.0;
    for (int d = 0; d < g.ndim; ++d) s = __dadd_rn(s, __ddiv_rn(a[d], g.dx[d]));
    return s;
}

struct BoundArgs {
    GridDev g;
    int dyn;
    int per_dim;  // 0: max over nodes of the sum (one word); 1: max over nodes of each alpha_d (ndim words)
    double q[8];
    const double* trig;
    unsigned long long* acc;
};

__device__ __forceinline__ double block_max(double v, double* scratch) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();  // scratch is reused across calls
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    double b = scratch[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, scratch[w]);
    return b;
}

__global__ void __launch_bounds__(256) step_bound_kernel(const BoundArgs A) {
    double best[4] = {0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long flat = (long long)blockIdx.x * blockDim.x + threadIdx.x; flat < A.g.total; flat += stride) {
        int idx[4] = {0, 0, 0, 0};
        long long r = flat;
        for (int d = 0; d < A.g.ndim; ++d) { idx[d] = (int)(r % A.g.n[d]); r /= A.g.n[d]; }
        if (A.per_dim) {
            double a[4];
            node_alpha(A.g, A.dyn, A.q, A.trig, idx, a);
            for (int d = 0; d < 4; ++d) best[d] = fmax(best[d], a[d]);
        } else {
            best[0] = fmax(best[0], node_bound(A.g, A.dyn, A.q, A.trig, idx));
        }
    }
    __shared__ double warp_best[8];
    const int words = A.per_dim ? A.g.ndim : 1;
    for (int d = 0; d < words; ++d) {
        const double b = block_max(best[d], warp_best);
        // non-negative doubles order like their bit patterns
        if (threadIdx.x == 0) atomicMax(A.acc + d, (unsigned long long)__double_as_longlong(b));
    }
}

// Streaming multiprocessors of the current device (grid-stride kernels size
// their grids in multiples of it), read once per device.
static int device_sms() {
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!sms[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        sms[dev] = n;  // benign race: every writer stores the same value
    }
    return sms[dev];
}

cudaError_t launch_step_bound(const GridDev& g, int dynamics, const double* params, const double* trig_d,
                              unsigned long long* acc, int per_dim, cudaStream_t s) {
    BoundArgs A;
    A.g = g;
    A.dyn = dynamics;
    A.per_dim = per_dim;
    for (int k = 0; k < 8; ++k) A.q[k] = params[k];
    A.trig = trig_d;
    A.acc = acc;
    long long blocks = (g.total + 255) / 256;
    const long long cap = 16LL * device_sms();  // a few waves of resident blocks
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    step_bound_kernel<<<(unsigned)blocks, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) nonfinite_kernel(const T* __restrict__ v, long long n, int* flag) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        bad |= !isfinite(v[i]);
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

template <typename T>
static cudaError_t launch_nonfinite(const T* v, long long n, int* flag, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    const long long cap = 8LL * device_sms();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    nonfinite_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(v, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite_f64(const double* v, long long n, int* flag, cudaStream_t s) {
    return launch_nonfinite<double>(v, n, flag, s);
}
cudaError_t launch_nonfinite_f32(const float* v, long long n, int* flag, cudaStream_t s) {
    return launch_nonfinite<float>(v, n, flag, s);
}

}  // namespace hj
