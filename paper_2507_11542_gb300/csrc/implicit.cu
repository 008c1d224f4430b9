// implicit.cu -- initial surfaces built on the device (Sec. 2.2: implicit
// surfaces on the grid container; geometric primitives combined by Boolean
// operations; the ellipsoid listing of that section).
//
// Blocks cover grid rows along dimension 0 (the row's coordinates along the
// other dimensions, and each primitive's contribution from them, are
// computed once per row), threads over the row so that every warp writes
// consecutive nodes. FP32 output is computed in FP32, FP64 output in FP64.
// The kernel only writes V: it is bound by HBM write bandwidth.
#include <cmath>
#include <cstring>

#include "ctx.h"

namespace hj {
namespace {

// A primitive in the kernel's precision (FP32 kernels convert nothing per node).
template <typename T>
struct ShapeT {
    int kind, op;
    unsigned mask;
    T c[kMaxDim], a[kMaxDim], r;
};

template <typename T>
ShapeT<T> shape_in(const hj_shape& s) {
    ShapeT<T> o;
    o.kind = s.kind;
    o.op = s.op;
    o.mask = s.dims_mask;
    for (int d = 0; d < kMaxDim; ++d) {
        o.c[d] = (T)s.center[d];
        o.a[d] = (T)s.axes[d];
    }
    o.r = (T)s.radius;
    return o;
}

template <typename T>
struct SurfaceArgs {
    GridDev g;
    int n;
    long long rows;  // prod(n[1..ndim-1])
    void* out;
    ShapeT<T> shp[HJ_MAX_SHAPES];
};

// A primitive's contribution from the dimensions >= 1 of one grid row (the
// same for every node of the row): partial sum of squares (sphere,
// ellipsoid) or partial maximum (rectangle; -inf if no dimension >= 1).
template <typename T>
__device__ __forceinline__ T shape_row_part(const ShapeT<T>& s, const T* xc) {
    T acc = (s.kind == HJ_SHAPE_RECTANGLE) ? T(-INFINITY) : T(0);
#pragma unroll
    for (int d = 1; d < kMaxDim; ++d) {
        if (!((s.mask >> d) & 1u)) continue;
        const T q = xc[d] - s.c[d];
        if (s.kind == HJ_SHAPE_RECTANGLE) acc = fmax(acc, fabs(q) - s.a[d]);
        else if (s.kind == HJ_SHAPE_ELLIPSOID) acc = acc + s.a[d] * (q * q);
        else acc = acc + q * q;
    }
    return acc;
}

// The primitive at a node of the row: dimension 0 joined to the row part.
// The sums run over dimensions in the order 1, 2, 3, then 0.
template <typename T>
__device__ __forceinline__ T shape_node(const ShapeT<T>& s, T part, T x0) {
    const bool on0 = s.mask & 1u;
    const T q = x0 - s.c[0];
    if (s.kind == HJ_SHAPE_RECTANGLE) return on0 ? fmax(part, fabs(q) - s.a[0]) : part;
    if (s.kind == HJ_SHAPE_ELLIPSOID) return (on0 ? part + s.a[0] * (q * q) : part) - s.r;
    return sqrt(on0 ? part + q * q : part) - s.r;
}

// Blocks: x over a row (dimension 0), y over dimension 1, z over the rest;
// each thread covers a few nodes of each row it visits. The row parts of the
// first kPre primitives are kept in registers, the others are recomputed per
// node.
constexpr int kPre = 4;

template <typename T>
__global__ void __launch_bounds__(128) surface_kernel(const SurfaceArgs<T> A) {
    const GridDev& g = A.g;
    const int nx = g.n[0];
    const int n1 = g.ndim > 1 ? g.n[1] : 1;
    const int n2 = g.ndim > 2 ? g.n[2] : 1;
    const long long nz = (long long)n2 * (g.ndim > 3 ? g.n[3] : 1);
    const T lo0 = T(g.lo[0]), dx0 = T(g.dx[0]);
    for (long long zz = blockIdx.z; zz < nz; zz += gridDim.z) {
        const int i2 = (int)(zz % n2), i3 = (int)(zz / n2);
        for (int i1 = blockIdx.y; i1 < n1; i1 += gridDim.y) {
            T xc[kMaxDim];
            xc[0] = T(0);
            xc[1] = g.ndim > 1 ? T(g.lo[1] + (double)i1 * g.dx[1]) : T(0);
            xc[2] = g.ndim > 2 ? T(g.lo[2] + (double)i2 * g.dx[2]) : T(0);
            xc[3] = g.ndim > 3 ? T(g.lo[3] + (double)i3 * g.dx[3]) : T(0);
            T pre[kPre];
#pragma unroll
            for (int k = 0; k < kPre; ++k) pre[k] = (k < A.n) ? shape_row_part<T>(A.shp[k], xc) : T(0);
            T* out = static_cast<T*>(A.out) + ((long long)zz * n1 + i1) * nx;
            for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < nx; i0 += gridDim.x * blockDim.x) {
                const T x0 = lo0 + T(i0) * dx0;
                T v = shape_node<T>(A.shp[0], pre[0], x0);
#pragma unroll
                for (int k = 1; k < kPre; ++k) {
                    if (k >= A.n) break;
                    const T sv = shape_node<T>(A.shp[k], pre[k], x0);
                    const int op = A.shp[k].op;
                    v = (op == HJ_SHAPE_UNION) ? fmin(v, sv) : (op == HJ_SHAPE_INTERSECT) ? fmax(v, sv) : fmax(v, -sv);
                }
                for (int k = kPre; k < A.n; ++k) {
                    const T sv = shape_node<T>(A.shp[k], shape_row_part<T>(A.shp[k], xc), x0);
                    const int op = A.shp[k].op;
                    v = (op == HJ_SHAPE_UNION) ? fmin(v, sv) : (op == HJ_SHAPE_INTERSECT) ? fmax(v, sv) : fmax(v, -sv);
                }
                out[i0] = v;
            }
        }
    }
}

bool finite4(const double* a) {
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(a[k])) return false;
    return true;
}

}  // namespace
}  // namespace hj

using namespace hj;

extern "C" hj_status hj_implicit_surface(hj_ctx* ctx, const hj_grid* grid, int32_t n_shapes, const hj_shape* shapes,
                                         int32_t dtype, void* out, int32_t out_on_device) {
    if (!ctx) return HJ_EINVAL;
    DeviceGuard guard(ctx->device);
    hj_status st = check_grid(ctx, grid);
    if (st) return st;
    const size_t es = elem_size(dtype);
    if (!es) return fail(ctx, HJ_EINVAL, "unknown dtype %d", dtype);
    if (!shapes || !out) return fail(ctx, HJ_EINVAL, "shapes and out must not be NULL");
    if (n_shapes < 1 || n_shapes > HJ_MAX_SHAPES)
        return fail(ctx, HJ_EINVAL, "n_shapes = %d is not in 1..%d", n_shapes, HJ_MAX_SHAPES);
    SurfaceArgs<double> A;
    SurfaceArgs<float> Af;
    std::memset(&A, 0, sizeof A);
    std::memset(&Af, 0, sizeof Af);
    A.g = make_grid(grid, HJ_EXTRAP_AWAY_FROM_ZERO);
    A.n = n_shapes;
    const uint32_t all = (1u << grid->ndim) - 1u;
    for (int k = 0; k < n_shapes; ++k) {
        const hj_shape& s = shapes[k];
        if (s.kind < HJ_SHAPE_SPHERE || s.kind > HJ_SHAPE_RECTANGLE)
            return fail(ctx, HJ_EINVAL, "shape %d: unknown kind %d", k, s.kind);
        if (k > 0 && (s.op < HJ_SHAPE_UNION || s.op > HJ_SHAPE_SUBTRACT))
            return fail(ctx, HJ_EINVAL, "shape %d: unknown operation %d", k, s.op);
        if (s.dims_mask == 0 || (s.dims_mask & ~all))
            return fail(ctx, HJ_EINVAL, "shape %d: dims_mask 0x%x does not fit a %d-D grid", k, s.dims_mask,
                        grid->ndim);
        if (!finite4(s.center) || !finite4(s.axes) || !std::isfinite(s.radius))
            return fail(ctx, HJ_EINVAL, "shape %d: non-finite parameter", k);
        for (int d = 0; d < grid->ndim; ++d) {
            if (!((s.dims_mask >> d) & 1u)) continue;
            if (s.kind == HJ_SHAPE_ELLIPSOID && !(s.axes[d] > 0.0))
                return fail(ctx, HJ_EINVAL, "shape %d: ellipsoid coefficient %d must be > 0", k, d);
            if (s.kind == HJ_SHAPE_RECTANGLE && !(s.axes[d] >= 0.0))
                return fail(ctx, HJ_EINVAL, "shape %d: rectangle half-width %d must be >= 0", k, d);
        }
        A.shp[k] = shape_in<double>(s);
        Af.shp[k] = shape_in<float>(s);
    }
    const long long N = A.g.total;
    A.rows = N / A.g.n[0];
    void* dst = out;
    if (!out_on_device) {
        st = ensure(ctx, &ctx->state, &ctx->state_bytes, (size_t)N * es);
        if (st) return st;
        dst = ctx->state;
    }
    A.out = dst;
    Af.g = A.g;
    Af.n = A.n;
    Af.rows = A.rows;
    Af.out = dst;
    const int threads = 128;
    const long long n1 = grid->ndim > 1 ? A.g.n[1] : 1;
    const long long nz = A.rows / n1;
    // about 4096 blocks of rows, each looping over its share
    const long long gz = std::min<long long>(nz, 4096);
    const long long gy = std::min<long long>(n1, std::max<long long>(1, 4096 / gz));
    const dim3 blocks((unsigned)((A.g.n[0] + 4 * threads - 1) / (4 * threads)), (unsigned)gy, (unsigned)gz);
    if (dtype == HJ_F64)
        surface_kernel<double><<<blocks, threads, 0, ctx->stream>>>(A);
    else
        surface_kernel<float><<<blocks, threads, 0, ctx->stream>>>(Af);
    ctx->launches += 1;
    HJ_CUDA(ctx, cudaGetLastError());
    if (!out_on_device) {
        HJ_CUDA(ctx, cudaMemcpyAsync(out, dst, (size_t)N * es, cudaMemcpyDeviceToHost, ctx->stream));
        HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return HJ_OK;
}
