// rows_kernel.cuh -- the fused RK stage kernel for WENO5 on 2-4 dimensional
// grids, tiled for GB300:
//
//  * A thread block owns TY full rows (all n0 nodes along dimension 0) of one
//    plane of dimensions (0, 1); threadIdx = (x, row), with n0 + 1 threads
//    per row and usually TY + 1 thread rows. The plane with three halo rows
//    above and below lives in shared memory.
//  * WENO5 is evaluated per interface (one interface gives p+ of a node and
//    p- of the next). Along dimension 0 thread x computes the interface
//    between nodes x-1 and x (the extra thread x = n0 the row's last one);
//    along dimension 1 thread row k the one between tile rows k-1 and k (the
//    extra thread row the tile's last one). So each node pays for about one
//    interface per dimension instead of two.
//  * For 3-D and 4-D grids the block streams along the last dimension through
//    a chunk of planes: each thread keeps six values of its column in
//    registers and carries the interface result p- to the next plane.
//  * In 4-D, dimension 2 is differentiated two-sided from 7-point loads.
//  * Ghost values (periodic wrap or slope continued away from zero, Sec. 2.1)
//    are produced where values are read; no padded array exists.
// Then: Hamiltonian + Lax-Friedrichs dissipation (Sec. 4), BRT clamp (Sec.
// 6.1) and the TVD-RK3 stage combination (Sec. 5), one store per node.
#pragma once

#include "stencil.cuh"
#include "weno_iface.cuh"

namespace hj {

// FP32 blocks may hold 1024 threads (<= 64 registers each); FP64 blocks at
// most 512 (<= 128 registers), since the FP64 interface math needs more.
template <typename T> struct RowsLimits;
template <> struct RowsLimits<float> { static constexpr int kMaxThreads = 1024; };
template <> struct RowsLimits<double> { static constexpr int kMaxThreads = 512; };

template <typename T>
__device__ __forceinline__ T ghost_value(T edge, T inner, int m, int extrap) {
    const T s = (extrap == HJ_EXTRAP_LINEAR) ? (edge - inner) : fabs(edge - inner) * sgn(edge);
    return add_rn(edge, mul_rn(T(m), s));
}

// Value at index i of a grid line (base pointer, n nodes, stride s), with the
// line's ghost rule outside [0, n).
template <typename T>
__device__ __forceinline__ T line_value(const T* __restrict__ base, int i, int n, long long s, bool periodic,
                                        int extrap) {
    if (i >= 0 && i < n) return ld(base + (long long)i * s);
    if (periodic) {
        int j = i % n;
        if (j < 0) j += n;
        return ld(base + (long long)j * s);
    }
    if (i < 0) return ghost_value(ld(base), ld(base + s), -i, extrap);
    return ghost_value(ld(base + (long long)(n - 1) * s), ld(base + (long long)(n - 2) * s), i - (n - 1), extrap);
}

// Value at index i of a shared-memory row of n nodes (ghosts from its ends).
template <typename T>
__device__ __forceinline__ T row_value(const T* row, int i, int n, bool periodic, int extrap) {
    if (i >= 0 && i < n) return row[i];
    if (periodic) {
        int j = i % n;
        if (j < 0) j += n;
        return row[j];
    }
    if (i < 0) return ghost_value(row[0], row[1], -i, extrap);
    return ghost_value(row[n - 1], row[n - 2], i - (n - 1), extrap);
}

// Values of one stage launch that differ between the three RK stages, in the
// kernel's precision (kept in registers).
template <typename T>
struct StageRun {
    const T* u;        // stencil input
    const T* vn;       // V^n (stages 2 and 3)
    T* out;            // result
    T* also_out;       // if not null, the result is written here as well (a time slice)
    T dt, cv, cu;
    bool has_vn, use_cv, minv, brt0, term;
};

template <typename T>
__device__ __forceinline__ StageRun<T> stage_run(const StageParams& P) {
    StageRun<T> R;
    R.u = static_cast<const T*>(P.u);
    R.vn = static_cast<const T*>(P.vn);
    R.out = static_cast<T*>(P.out);
    R.also_out = nullptr;
    R.dt = SP<T>::dt(P);
    R.cv = SP<T>::cv(P);
    R.cu = SP<T>::cu(P);
    R.has_vn = P.has_vn;
    R.use_cv = P.cv != 0.0;
    R.minv = P.minv_after;
    R.brt0 = P.brt_min0;
    R.term = P.mode == kTerm;
    return R;
}

// One tile: rows y0 = row_tile*TY .. +TY-1 of the plane(s) at dimension-2 index
// i2 (4-D) and the planes of chunk `chunk` along the streamed dimension
// (planes chunk*tz .. +tz-1). The block has NR thread rows; (x, r) is this
// thread's position, x in 0..n0, r in 0..NR-1 (threads with r >= NR only
// take part in the barriers). Per plane, the interfaces along dimensions 0
// and 1 are each evaluated once and shared through shared memory:
//   x-interfaces: n0+1 per node row (rows k = r, r+NR, ...),
//   y-interfaces: TY+1 per column (gaps k = r, r+NR, ...; gap k lies between
//                 tile rows k-1 and k),
// so with NR = TY+1 every thread evaluates at most one of each. The p- half
// of the interface a thread evaluates for its own row or gap belongs to its
// own node and stays in a register; the p+ half belongs to the neighbour
// (x-1 or row k-1) and goes through shared memory.
template <typename T, int D, int DYN>
__device__ __forceinline__ void rows_tile(const StageParams& P, const StageRun<T>& R, const int TY, const int NR,
                                          const int tz, const int row_tile, const int i2_in, const int chunk_in,
                                          const int x, const int r, T* const smem) {
    const GridDev& g = P.g;
    const int nx = g.n[0], ny = g.n[1];
    const int W = nx + 6;  // shared row: 3 ghost cells, nx nodes, 3 ghost cells
    // two buffers, alternating by plane: (TY + 6) rows x W, then p+ along
    // dimension 0 (TY rows of nx + 1) and along dimension 1 (TY + 1 rows of nx)
    const size_t buf_elems = rows_buf_elems(nx, TY);

    const T* __restrict__ u = R.u;
    const T* __restrict__ vn = R.vn;
    T* __restrict__ out = R.out;
    const T floor_raw = SP<T>::floor(P);
    const bool per0 = g.periodic_mask & 1u, per1 = (g.periodic_mask >> 1) & 1u;
    const int extrap = g.extrap;

    const int y0 = row_tile * TY;
    const int y = y0 + r;
    const int rows_valid = min(TY, ny - y0);
    const bool in_rows = r < NR;
    const bool node = (x < nx) && (r < rows_valid);

    const int i2 = (D == 4) ? i2_in : 0;
    const int chunk = (D >= 3) ? chunk_in : 0;
    constexpr int SD = (D >= 3) ? D - 1 : 0;  // streamed dimension
    const int ns = (D >= 3) ? g.n[SD] : 1;
    const int zbeg = (D >= 3) ? chunk * tz : 0;
    const int zend = (D >= 3) ? min(ns, zbeg + tz) : 1;
    const long long sS = (D >= 3) ? g.stride[SD] : 0;
    const bool perS = (D >= 3) ? ((g.periodic_mask >> SD) & 1u) : false;
    // the chunk's streamed-dimension reads stay inside the grid: no ghost logic needed
    const bool z_inside = (D < 3) || (zbeg >= 3 && zend + 3 <= ns);
    const T* __restrict__ uplane = u + ((D == 4) ? (long long)i2 * g.stride[2] : 0);
    const long long colbase = (long long)min(x, nx - 1) + (long long)min(y, ny - 1) * nx;  // within a plane

    const T inv_dx0 = SP<T>::inv_dx(P, 0);
    const T inv_dx1 = SP<T>::inv_dx(P, 1);
    const T inv_dxs = SP<T>::inv_dx(P, SD);
    const T dt = R.dt, cv = R.cv, cu = R.cu;
    const bool has_vn = R.has_vn, use_cv = R.use_cv, minv = R.minv, brt0 = R.brt0;
    const bool term_mode = R.term;
    T* __restrict__ also_out = R.also_out;

    // Halo rows (three above, three below, and rows past the grid edge in a
    // ragged last tile) are loaded by thread rows in turn: row h of n_extra.
    const int n_extra = 3 + (TY + 3 - rows_valid);

    // Streamed-dimension queue: q[k] = V at plane z-2+k (k = 0..5); carry = p- at z.
    // The loop starts one plane early (a warm-up iteration that only evaluates
    // the streamed interface) so that every interface goes through the same
    // code and results do not depend on where chunks start.
    T q[6];
    T carry = T(0);
    if (D >= 3 && node) {
#pragma unroll
        for (int k = 0; k < 5; ++k) q[k] = line_value(uplane + colbase, zbeg - 3 + k, ns, sS, perS, extrap);
    }
    const int zfirst = (D >= 3) ? zbeg - 1 : zbeg;

    for (int z = zfirst; z < zend; ++z) {
        const bool warm = z < zbeg;  // block-uniform
        const long long zoff = (D >= 3) ? (long long)z * sS : 0;
        const T* __restrict__ uz = uplane + zoff;
        T* const buf = smem + (size_t)((z - zfirst) & 1) * buf_elems;
        T* const plane = buf;
        T* const pxp = buf + (size_t)(TY + 6) * W;
        T* const pyp = pxp + (size_t)TY * (nx + 1);
        T center = T(0);
        T pm_x = T(0), pm_y = T(0);
        if (node) {
            if (D >= 3) {
                q[5] = z_inside ? ld(uplane + colbase + (long long)(z + 3) * sS)
                                : line_value(uplane + colbase, z + 3, ns, sS, perS, extrap);
                center = q[2];
            } else {
                center = ld(uz + colbase);
            }
        }
        if (!warm) {
            // stage the plane: node rows from the threads' own values, halo rows
            // from global memory (ghost rule along dimension 1), and the x-ghost
            // cells of each node row from its spare thread x == nx
            if (node) plane[(size_t)(r + 3) * W + 3 + x] = center;
            if (in_rows) {
                if (x < nx) {
                    for (int h = r; h < n_extra; h += NR) {
                        const int rr = (h < 3) ? h - 3 : rows_valid + (h - 3);
                        plane[(size_t)(rr + 3) * W + 3 + x] =
                            line_value(uz + x, y0 + rr, ny, (long long)nx, per1, extrap);
                    }
                } else if (r < rows_valid) {
                    const T* rowg = uz + (long long)y * nx;
                    T* rows = plane + (size_t)(r + 3) * W;
                    if (per0) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            rows[k] = ld(rowg + ((nx - 3 + k) % nx + nx) % nx);
                            rows[nx + 3 + k] = ld(rowg + k % nx);
                        }
                    } else {
                        const T e0 = ld(rowg), e1 = ld(rowg + 1), f0 = ld(rowg + nx - 1), f1 = ld(rowg + nx - 2);
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            rows[k] = ghost_value(e0, e1, 3 - k, extrap);
                            rows[nx + 3 + k] = ghost_value(f0, f1, k + 1, extrap);
                        }
                    }
                }
            }
            __syncthreads();
            // x-interface between nodes x-1 and x of row r (x = nx: the row's last one);
            // pxp slot r*(nx+1) + x receives p+ of node x-1 (slot 0 of a row is unused)
            if (in_rows && r < rows_valid) {
                const T* a = plane + (size_t)(r + 3) * W + x;  // a[m] = value at node x - 3 + m
                T ppj;
                weno_iface(a[1] - a[0], a[2] - a[1], a[3] - a[2], a[4] - a[3], a[5] - a[4], floor_raw, inv_dx0, ppj,
                           pm_x);
                pxp[(size_t)r * (nx + 1) + x] = ppj;
            }
            // y-interface of gap k (between tile rows k-1 and k) of column x, k = r;
            // pyp slot k*nx + x receives p+ of tile row k-1 (row 0 of pyp is unused)
            if (x < nx && in_rows && r <= rows_valid) {
                const T* c = plane + (size_t)r * W + 3 + x;  // c[m W] = tile row r - 3 + m
                T ppj;
                weno_iface(c[W] - c[0], c[2 * W] - c[W], c[3 * W] - c[2 * W], c[4 * W] - c[3 * W],
                           c[5 * W] - c[4 * W], floor_raw, inv_dx1, ppj, pm_y);
                pyp[(size_t)r * nx + x] = ppj;
            }
            // without an extra thread row (NR == TY), row 0 also takes the tile's last gap
            if (NR <= rows_valid && r == 0 && x < nx) {
                const T* c = plane + (size_t)NR * W + 3 + x;
                T ppj, unused;
                weno_iface(c[W] - c[0], c[2 * W] - c[W], c[3 * W] - c[2 * W], c[4 * W] - c[3 * W],
                           c[5 * W] - c[4 * W], floor_raw, inv_dx1, ppj, unused);
                pyp[(size_t)NR * nx + x] = ppj;
            }
            __syncthreads();
        }
        if (node) {
            T pm[D], pp[D];
            T next = T(0);
            if constexpr (D >= 3) {
                weno_iface(q[1] - q[0], q[2] - q[1], q[3] - q[2], q[4] - q[3], q[5] - q[4], floor_raw, inv_dxs,
                           pp[SD], next);
                pm[SD] = carry;
            }
            if (!warm) {
                pm[0] = pm_x;
                pp[0] = pxp[(size_t)r * (nx + 1) + x + 1];
                pm[1] = pm_y;
                pp[1] = pyp[(size_t)(r + 1) * nx + x];
                if constexpr (D == 4) {
                    T v[7];
                    gather7<T>(u, (long long)i2 * g.stride[2] + zoff + colbase, i2, g.n[2], g.stride[2],
                               (g.periodic_mask >> 2) & 1u, extrap, v);
                    weno5_pair<T>(v, SP<T>::dx(P, 2), floor_raw, pm[2], pp[2]);
                }
                int idx[4] = {x, y, 0, 0};
                if (D == 3) idx[2] = z;
                if (D == 4) { idx[2] = i2; idx[3] = z; }
                T yd = lf_term_dyn<T, D, DYN>(P, idx, pm, pp);
                if (brt0) yd = fmin(yd, T(0));
                const long long flat = (uz - u) + colbase;
                T res;
                if (term_mode) {
                    res = yd;
                } else {
                    const T w = center + dt * yd;
                    res = w;
                    if (has_vn) {
                        const T vv = ld(vn + flat);
                        if (use_cv) res = cv * vv + cu * w;
                        if (minv) res = fmin(res, vv);
                    }
                }
                out[flat] = res;
                if (also_out) also_out[flat] = res;
            }
            if constexpr (D >= 3) {
                carry = next;
#pragma unroll
                for (int k = 0; k < 5; ++k) q[k] = q[k + 1];
            }
        }
    }
}

template <typename T, int D, int DYN>
__global__ void __launch_bounds__(RowsLimits<T>::kMaxThreads) rows_kernel(const StageParams P, const RowsCfg C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const StageRun<T> R = stage_run<T>(P);
    const int i2 = (D == 4) ? (int)blockIdx.y : 0;
    const int chunk = (D == 3) ? (int)blockIdx.y : ((D == 4) ? (int)blockIdx.z : 0);
    rows_tile<T, D, DYN>(P, R, C.ty, C.nr, C.tz, blockIdx.x, i2, chunk, threadIdx.x, threadIdx.y,
                         reinterpret_cast<T*>(smem_raw));
}

// Shared memory of a rows_kernel block.
template <typename T>
inline size_t rows_smem_bytes(int nx, int ty) {
    return rows_smem(nx, ty, sizeof(T));
}

template <typename T, int D, int DYN>
inline void rows_shape(const StageParams& p, const RowsCfg& c, dim3& grid, dim3& block, size_t& smem) {
    block = dim3((unsigned)(p.g.n[0] + 1), (unsigned)c.nr, 1);
    grid = dim3((unsigned)c.row_tiles, 1, 1);
    if (D == 3) grid.y = (unsigned)c.nchunks;
    if (D == 4) { grid.y = (unsigned)p.g.n[2]; grid.z = (unsigned)c.nchunks; }
    smem = rows_smem_bytes<T>(p.g.n[0], c.ty);
}

template <typename T, int D, int DYN>
inline cudaError_t rows_prepare() {
    static bool done = false;  // benign race: setting the attribute twice is harmless
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(rows_kernel<T, D, DYN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

template <typename T, int D, int DYN>
cudaError_t launch_rows_dyn(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    dim3 grid, block;
    size_t smem;
    rows_shape<T, D, DYN>(p, c, grid, block, smem);
    cudaError_t e = rows_prepare<T, D, DYN>();
    if (e != cudaSuccess) return e;
    rows_kernel<T, D, DYN><<<grid, block, smem, s>>>(p, c);
    return cudaGetLastError();
}

template <typename T, int D, int DYN>
int rows_bps_dyn(const StageParams& p, const RowsCfg& c) {
    dim3 grid, block;
    size_t smem;
    rows_shape<T, D, DYN>(p, c, grid, block, smem);
    if (rows_prepare<T, D, DYN>() != cudaSuccess) return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rows_kernel<T, D, DYN>, (int)(block.x * block.y), smem) !=
        cudaSuccess)
        return 0;
    return bps;
}

// Dispatch over the (dimension, dynamics) pairs the row kernel is built for.
#define HJ_ROWS_DISPATCH(FN, T, ...)                                                   \
    switch (p.g.ndim * 16 + p.dynamics) {                                              \
    case 2 * 16 + HJ_DYN_DOUBLE_INTEGRATOR: return FN<T, 2, HJ_DYN_DOUBLE_INTEGRATOR>(__VA_ARGS__); \
    case 2 * 16 + HJ_DYN_NORM: return FN<T, 2, HJ_DYN_NORM>(__VA_ARGS__);             \
    case 2 * 16 + HJ_DYN_ADVECT: return FN<T, 2, HJ_DYN_ADVECT>(__VA_ARGS__);         \
    case 2 * 16 + HJ_DYN_ROTATE: return FN<T, 2, HJ_DYN_ROTATE>(__VA_ARGS__);         \
    case 3 * 16 + HJ_DYN_AIR3D: return FN<T, 3, HJ_DYN_AIR3D>(__VA_ARGS__);           \
    case 3 * 16 + HJ_DYN_NORM: return FN<T, 3, HJ_DYN_NORM>(__VA_ARGS__);             \
    case 3 * 16 + HJ_DYN_ADVECT: return FN<T, 3, HJ_DYN_ADVECT>(__VA_ARGS__);         \
    case 3 * 16 + HJ_DYN_ROTATE: return FN<T, 3, HJ_DYN_ROTATE>(__VA_ARGS__);         \
    case 4 * 16 + HJ_DYN_DUBINS4D: return FN<T, 4, HJ_DYN_DUBINS4D>(__VA_ARGS__);     \
    default: break;                                                                    \
    }

}  // namespace hj
