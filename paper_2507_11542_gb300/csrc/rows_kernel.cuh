// rows_kernel.cuh -- the fused RK stage kernel (WENO5, ENO1/2/3) on 2-4 dimensional
// grids, tiled for GB300:
//
//  * A thread block (1-D) owns TY full rows (all n0 nodes along dimension 0)
//    of one plane of dimensions (0, 1): one thread per node, one per row end
//    and, where the block has room, one per column for the tile's last
//    dimension-1 interface, each role in its own warps. The plane with
//    three halo rows above and below lives in shared memory.
//  * The upwind scheme (WENO5, ENO1/2/3) is evaluated per interface (one
//    interface gives p+ of a node and p- of the next). Along dimension 0 the
//    node thread x computes the interface between nodes x-1 and x (the row
//    end the row's last one); along dimension 1 the node thread of row k the
//    one between tile rows k-1 and k (the gap threads the tile's last one).
//    So each node pays for about one interface per dimension instead of two.
//  * For 3-D and 4-D grids the block streams along the last dimension through
//    a chunk of planes: each thread keeps six values of its column in
//    registers and carries the interface result p- to the next plane. Planes
//    are staged in shared memory two ahead of their use (asynchronous
//    copies), with one barrier per plane.
//  * In 4-D, dimension 2 is differentiated two-sided from 7-point loads.
//  * Ghost values (periodic wrap or slope continued away from zero, Sec. 2.1)
//    are produced where values are read; no padded array exists.
// Then: Hamiltonian + Lax-Friedrichs dissipation (Sec. 4), BRT clamp (Sec.
// 6.1) and the TVD-RK3 stage combination (Sec. 5), one store per node.
#pragma once

#include <atomic>
#include <type_traits>

#include "stencil.cuh"
#include "weno_iface.cuh"

namespace hj {

template <typename T> struct RowsLimits;
template <> struct RowsLimits<float> { static constexpr int kMaxThreads = kRowsMaxThreadsF32; };
template <> struct RowsLimits<double> { static constexpr int kMaxThreads = kRowsMaxThreadsF64; };
// Launch bounds of a row-kernel variant: OCC resident blocks per SM.
template <typename T, int OCC> struct RowsBounds {
    static constexpr int kThreads = OCC == 2 ? kRowsOcc2Threads : RowsLimits<T>::kMaxThreads;
};

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

// Values of one stage launch that differ between the three RK stages, in the
// kernel's precision (kept in registers).
template <typename T>
struct StageRun {
    const T* u;        // stencil input
    const T* vn;       // V^n (stages 2 and 3)
    T* out;            // result
    T* also_out;       // if not null, the result is written here as well (a time slice)
    T dt, cv, cu;
    bool minv, brt0;
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
    R.minv = P.minv_after;
    R.brt0 = P.brt_min0;
    return R;
}

// Asynchronous copy of one element from global to shared memory (cp.async:
// no register is involved). The issuing thread waits for its own copies with
// cp_async_wait_all; a barrier after that publishes them to the block.
template <typename T> __device__ __forceinline__ void cp_async_elem(T* dst, const T* src);
template <> __device__ __forceinline__ void cp_async_elem<float>(float* dst, const float* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    const size_t gsrc = __cvta_generic_to_global(src);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
template <> __device__ __forceinline__ void cp_async_elem<double>(double* dst, const double* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    const size_t gsrc = __cvta_generic_to_global(src);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }


// One tile: rows y0 = row_tile*TY .. +TY-1 of the plane(s) at dimension-2 index
// i2 (4-D) and the planes of chunk `chunk` along the streamed dimension
// (planes chunk*tz .. +tz-1), computed by the NT threads of a 1-D block.
// Thread t has one role, so that roles change only between whole warps
// (except one warp at each boundary):
//   t <  n0*TY          node (x, r) = (t mod n0, t div n0);
//   t <  n0*TY + TY     row end of row r = t - n0*TY (x = n0);
//   t <  n0*TY+TY+n0    gap thread of column x (present when the block has
//                       room: NT >= n0*TY + TY + n0);
//   others              barriers only.
// A block of exactly n0*TY threads has no row-end threads: node thread x of
// the last node row takes the end of row x as well (rows of n0 >= TY nodes).
//
// Interfaces along dimensions 0 and 1 are each evaluated once per plane and
// shared through shared memory:
//   x-interfaces: node (x, r) takes the one between nodes x-1 and x, the row
//                 end the row's last one;
//   y-interfaces: node (x, r) takes gap r (between tile rows r-1 and r), the
//                 gap thread of column x the tile's last gap (without gap
//                 threads: an idle node row of a ragged tile, else row 0).
// The p- half of the interface a thread evaluates for its own node stays in a
// register; the p+ half belongs to the neighbour (x-1 or row r-1) and goes
// through shared memory. Derivatives stay raw (undivided differences) until
// the node combines them, scaled by 1/(2 dx), into the means and half
// differences the Hamiltonian takes.
//
// Planes are software-pipelined through two shared buffers (plane p in
// buffer p mod 2) with one barrier per plane:
//   phase A(z): interfaces of plane z; ghost cells of plane z+1 from its row
//               ends; wait for this thread's copies into plane z+1
//   barrier
//   phase B(z): node updates of plane z; staging of plane z+2 (node values
//               from the column queues, halo rows and row ends copied
//               asynchronously), two planes ahead of its use.
// Flat indices are 32-bit (the grid has fewer than 2^31 nodes).
//
// IN: the tile is interior (all TY rows in the grid, its halo rows and the
// chunk's streamed-dimension reads inside the grid): no ghost or wrap logic
// is compiled for its staging and queue loads (a block-uniform dispatch).
template <typename T, int D, int DYN, int SCHEME, int KIND, bool IN = false>
__device__ __forceinline__ void rows_tile(const StageParams& P, const StageRun<T>& R, const int TY, const int NT,
                                          const int tz, const int row_tile, const int i2_in, const int chunk_in,
                                          const int t, T* const smem) {
    const GridDev& g = P.g;
    const int nx = g.n[0], ny = g.n[1];
    const int W = nx + 6;  // shared row: 3 ghost cells, nx nodes, 3 ghost cells
    // per buffer: (TY + 6) rows x W, p+ along dimension 0 (TY rows of nx + 1),
    // p+ along dimension 1 (TY + 1 rows of nx), row ends (4 per node row)
    const int buf_elems = (int)rows_buf_elems(nx, TY);
    const int o_pxp = (TY + 6) * W;
    const int o_pyp = o_pxp + TY * (nx + 1);
    const int o_ends = o_pyp + (TY + 1) * nx;

    const T* __restrict__ u = R.u;
    const T* __restrict__ vn = R.vn;
    T* __restrict__ out = R.out;
    const bool per0 = g.periodic_mask & 1u, per1 = (g.periodic_mask >> 1) & 1u;
    const int extrap = g.extrap;

    const int y0 = row_tile * TY;
    const int rows_valid = min(TY, ny - y0);
    // roles
    const int n_node = nx * TY;
    const int n_end = n_node + TY;
    const bool gaps = nx * TY + TY + nx <= NT;
    const bool is_node = t < n_node;
    const bool is_end = t >= n_node && t < n_end;
    const bool is_gap = gaps && t >= n_end && t < n_end + nx;
    int x, r;
    if (is_node) {
        r = t / nx;
        x = t - r * nx;
    } else if (is_end) {
        r = t - n_node;
        x = nx;
    } else {
        r = TY;
        x = is_gap ? t - n_end : nx;
    }
    const int y = y0 + r;
    const bool node = is_node && r < rows_valid;
    const bool do_xrow = (is_node || is_end) && r < rows_valid;
    // this thread's gap (tile row boundary) along dimension 1, or -1
    int gk = -1;
    if (is_node && r < rows_valid) gk = r;
    else if (is_gap) gk = rows_valid;
    else if (!gaps && is_node && r == rows_valid) gk = rows_valid;  // an idle row of a ragged tile
    const bool do_ylast = !gaps && rows_valid == TY && is_node && r == 0;  // full tile, no gap threads
    // The row-end role of a tile row er: the row's last dimension-0 interface,
    // its ghost sources and ghost cells. Row-end threads take it, or, in a
    // block of exactly n0*TY threads (no row-end threads), node thread x of the
    // last node row takes the end of row x: that row's threads evaluate one
    // interface fewer than row 0's, which also takes the tile's last gap.
    const bool merged = NT < n_end;
    const bool spare = merged ? (is_node && r == TY - 1 && x < rows_valid) : (is_end && r < rows_valid);
    const int er = merged ? x : r;
    const int ey = y0 + er;

    const int i2 = (D == 4) ? i2_in : 0;
    const int chunk = (D >= 3) ? chunk_in : 0;
    constexpr int SD = (D >= 3) ? D - 1 : 0;  // streamed dimension
    const T fl0 = SP<T>::floor(P, 0), fl1 = SP<T>::floor(P, 1), flS = SP<T>::floor(P, SD);
    const int ns = (D >= 3) ? g.n[SD] : 1;
    const int zbeg = (D >= 3) ? chunk * tz : 0;
    const int zend = (D >= 3) ? min(ns, zbeg + tz) : 1;
    const int sS = (D >= 3) ? (int)g.stride[SD] : 0;
    const bool perS = (D >= 3) ? ((g.periodic_mask >> SD) & 1u) : false;
    // the chunk's streamed-dimension reads stay inside the grid: no ghost logic needed
    const bool z_inside = IN || (D < 3) || (zbeg >= 3 && zend + 3 <= ns);
    const int plane0 = (D == 4) ? i2 * (int)g.stride[2] : 0;      // flat index of (0, 0, i2, 0)
    const int col = plane0 + min(x, nx - 1) + min(y, ny - 1) * nx;  // flat index of (x, y) at streamed index 0
    const T* __restrict__ ucol = u + col;

    // shared-memory offsets within a buffer
    const int s_center = (r + 3) * W + 3 + x;
    const int s_xrow = (r + 3) * W + x;        // value at node x - 3 of row r
    const int s_ycol = gk * W + 3 + x;         // value at tile row gk - 3 of column x
    const int s_ylast = TY * W + 3 + x;
    const int s_pxp = o_pxp + r * (nx + 1) + x;  // p+ of node x - 1 of row r (written); + 1: of node x (read)
    const int s_pyw = o_pyp + gk * nx + x;       // p+ of tile row gk - 1 (written)
    const int s_pyr = o_pyp + (r + 1) * nx + x;  // p+ of tile row r (read)

    // 1/(2 dx), or 1/(12 dx) where the interface evaluation returns six times the derivatives
    const auto half_inv = [&P](int d) -> T {
        if constexpr (iface_times6<T, SCHEME>()) return SP<T>::half_inv_dx6(P, d);
        else return SP<T>::half_inv_dx(P, d);
    };
    const T h0 = half_inv(0), h1 = half_inv(1), hS = half_inv(SD);
    const T dt = R.dt, cv = R.cv, cu = R.cu;
    const bool minv = R.minv;
    // BRT min(0, .) as a clamp (+inf: none), global dissipation as a flag, both read once
    const bool brt0 = R.brt0;
    const T clamp = brt0 ? T(0) : T(INFINITY);
    const bool alpha_global = P.alpha_global;
    T* __restrict__ also_out = R.also_out;
    // node coordinates that do not change along the streamed dimension
    T xc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) xc[d] = T(0);
    if constexpr (uses_coord<D, DYN>(0)) xc[0] = coord(SP<T>::lo(P, 0), x, SP<T>::dx(P, 0));
    if constexpr (uses_coord<D, DYN>(1)) xc[1] = coord(SP<T>::lo(P, 1), y, SP<T>::dx(P, 1));
    if constexpr (D == 4 && uses_coord<D, DYN>(2)) xc[2] = coord(SP<T>::lo(P, 2), i2, SP<T>::dx(P, 2));
    const T* __restrict__ trig = Trig<T>::get(P);       // cos of the dimension-2 coordinate
    const T* __restrict__ trig_s = uses_angle<D, DYN>() ? trig + g.n[2] : trig;  // sin
    T cos2 = T(0), sin2 = T(0);  // angle of dimension 2 (fixed for the block in 4-D)
    if constexpr (D == 4 && uses_angle<D, DYN>()) {
        cos2 = trig[i2];
        sin2 = trig_s[i2];
    }

    // Halo rows (three above, three below, and rows past the grid edge in a
    // ragged last tile): slot s = h * nx + hx of the n_extra * nx halo values
    // goes to thread s, s - NT, ... (node threads take their own column).
    const int n_extra = 3 + (TY + 3 - rows_valid);
    const int n_halo = n_extra * nx;

    // Plane p into buffer b, except the node values: halo rows (in-grid or
    // periodic rows copied asynchronously, rows past an extrapolated edge by
    // the ghost rule) and, from the row ends, the row's x-ghost sources
    // (periodic: the wrapped nodes into the ghost cells; extrapolated: the
    // two outermost nodes at each end into the row-end slots).
    auto halo_slot = [&](int sidx, int fp, T* b) {
        const int h = sidx / nx, hx = sidx - h * nx;
        const int rr = (h < 3) ? h - 3 : rows_valid + (h - 3);
        int yy = y0 + rr;
        T* dst = b + (rr + 3) * W + 3 + hx;
        if (!IN && per1 && (yy < 0 || yy >= ny)) yy = (yy % ny + ny) % ny;
        const T* base = u + plane0 + fp + hx;
        if (IN || (yy >= 0 && yy < ny)) cp_async_elem(dst, base + yy * nx);
        else *dst = line_value(base, yy, ny, (long long)nx, false, extrap);
    };
    // this thread's first halo slot (the same in every plane): destination and source
    const bool h0_on = t < n_halo;
    const int h0_h = t / nx, h0_x = t - (t / nx) * nx;
    const int h0_rr = (h0_h < 3) ? h0_h - 3 : rows_valid + (h0_h - 3);
    const int h0_dst = (h0_rr + 3) * W + 3 + h0_x;
    int h0_yy = y0 + h0_rr;
    if (!IN && per1 && (h0_yy < 0 || h0_yy >= ny)) h0_yy = (h0_yy % ny + ny) % ny;
    const bool h0_in = IN || (h0_yy >= 0 && h0_yy < ny);
    const int h0_src = plane0 + h0_x + (h0_in ? h0_yy * nx : 0);
    auto stage_rest = [&](int p, T* b) {
        const int fp = p * sS;
        if (h0_on) {
            if (h0_in) cp_async_elem(b + h0_dst, u + h0_src + fp);
            else b[h0_dst] = line_value(u + plane0 + fp + h0_x, h0_yy, ny, (long long)nx, false, extrap);
        }
        for (int sidx = t + NT; sidx < n_halo; sidx += NT) halo_slot(sidx, fp, b);  // small blocks, ragged tiles
        if (spare) {
            const T* rowg = u + plane0 + fp + ey * nx;
            if (per0) {
                T* rows = b + (er + 3) * W;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    cp_async_elem(rows + k, rowg + nx - 3 + k);
                    cp_async_elem(rows + nx + 3 + k, rowg + k);
                }
            } else {
                T* e = b + o_ends + 4 * er;
                cp_async_elem(e + 0, rowg);
                cp_async_elem(e + 1, rowg + 1);
                cp_async_elem(e + 2, rowg + nx - 1);
                cp_async_elem(e + 3, rowg + nx - 2);
            }
        }
    };
    // Row end, after its copies into b have landed: the extrapolated x-ghost cells of its row.
    auto finish_ghosts = [&](T* b) {
        if (spare && !per0) {
            const T* e = b + o_ends + 4 * er;
            T* rows = b + (er + 3) * W;
            const T e0 = e[0], e1 = e[1], f0 = e[2], f1 = e[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                rows[k] = ghost_value(e0, e1, 3 - k, extrap);
                rows[nx + 3 + k] = ghost_value(f0, f1, k + 1, extrap);
            }
        }
    };


    // Streamed-dimension queue: q[k] = V at plane z-2+k (k = 0..5); carry = raw p- at z.
    // A warm-up step evaluates the interface below the first plane, so that
    // every interface goes through the same code and results do not depend
    // on where chunks start.
    // In FP64 WENO5 the streamed-dimension interfaces slide along the column:
    // each reuses the differences of the one below it (Weno5Line, bit for bit
    // the same results as a full evaluation).
    constexpr bool kSlide = std::is_same<T, double>::value && SCHEME == HJ_WENO5 && D >= 3;
    T q[6];
    T carry = T(0);
    Weno5Line zline;
    if (D >= 3 && node) {
#pragma unroll
        for (int k = 0; k < 6; ++k)
            q[k] = IN ? ld(ucol + (zbeg - 3 + k) * sS) : line_value(ucol, zbeg - 3 + k, ns, (long long)sS, perS, extrap);
        T unused;
        if constexpr (kSlide) {
            zline.start(q[0], q[1], q[2], q[3], q[4], q[5]);
            zline.eval(flS, unused, carry);
        } else {
            iface_at<SCHEME>(q[0], q[1], q[2], q[3], q[4], q[5], flS, unused, carry);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) q[k] = q[k + 1];
    }

    // V^n of the node's next plane is loaded one plane ahead of its use (2-D
    // and 3-D grids), so that its global-memory latency is covered by a whole
    // plane of work. Where out aliases V^n, the value read is this thread's own
    // node, which it writes one plane later.
    constexpr bool kVnAhead = KIND == kKindCombine && D <= 3;
    T vn_next = T(0);
    if constexpr (kVnAhead) {
        if (node) vn_next = ld(vn + col + zbeg * sS);
    }

    // prologue: planes zbeg and zbeg+1 (ghost cells of zbeg+1 follow in phase A(zbeg))
    {
        T* const b0 = smem;
        if (node) b0[s_center] = (D >= 3) ? q[2] : ld(ucol);
        stage_rest(zbeg, b0);
        if (zbeg + 1 < zend) {
            T* const b1 = smem + buf_elems;
            if (node) b1[s_center] = q[3];
            stage_rest(zbeg + 1, b1);
        }
        cp_async_wait_all();
        finish_ghosts(b0);
        __syncthreads();
    }

    for (int z = zbeg; z < zend; ++z) {
        const int fz = z * sS;
        T* const bz = smem + ((z - zbeg) & 1) * buf_elems;        // plane z (and z+2)
        T* const bn = smem + ((z - zbeg + 1) & 1) * buf_elems;    // plane z+1
        T cosz = cos2, sinz = sin2;
        if constexpr (D == 3 && uses_angle<D, DYN>()) {
            cosz = trig[z];
            sinz = trig_s[z];
        }
        if (D >= 3 && node)
            q[5] = z_inside ? ld(ucol + fz + 3 * sS) : line_value(ucol, z + 3, ns, (long long)sS, perS, extrap);
        T vv = T(0);
        if constexpr (kVnAhead) {
            if (node) {
                vv = vn_next;
                if (z + 1 < zend) vn_next = ld(vn + col + fz + sS);
            }
        }

        // phase A: interfaces of plane z along dimensions 0 and 1
        T pmx = T(0), pmy = T(0);
        // x-interface between nodes x-1 and x of row r (x = nx: the row's last one)
        if (do_xrow) {
            const T* a = bz + s_xrow;
            T ppj;
            iface_at<SCHEME>(a[0], a[1], a[2], a[3], a[4], a[5], fl0, ppj, pmx);
            bz[s_pxp] = ppj;
        }
        // merged blocks: the last interface of row er (between node n0-1 and the ghost n0)
        if (merged && spare) {
            const T* a = bz + (er + 3) * W + nx;
            T ppj, unused;
            iface_at<SCHEME>(a[0], a[1], a[2], a[3], a[4], a[5], fl0, ppj, unused);
            bz[o_pxp + er * (nx + 1) + nx] = ppj;
        }
        // y-interface of gap gk (between tile rows gk-1 and gk) of column x
        if (gk >= 0) {
            const T* c = bz + s_ycol;
            T ppj;
            iface_at<SCHEME>(c[0], c[W], c[2 * W], c[3 * W], c[4 * W], c[5 * W], fl1, ppj, pmy);
            bz[s_pyw] = ppj;
        }
        if (do_ylast) {
            const T* c = bz + s_ylast;
            T ppj, unused;
            iface_at<SCHEME>(c[0], c[W], c[2 * W], c[3 * W], c[4 * W], c[5 * W], fl1, ppj, unused);
            bz[o_pyp + TY * nx + x] = ppj;
        }
        cp_async_wait_all();  // this thread's copies into plane z+1
        if (z + 1 < zend) finish_ghosts(bn);
        __syncthreads();

        // phase B: staging of plane z+2, then the node update of plane z
        if (z + 2 < zend) {
            if (node) bz[s_center] = q[4];
            stage_rest(z + 2, bz);
        }
        if (node) {
            const T center = (D >= 3) ? q[2] : ld(ucol);
            // raw sums and differences of the one-sided derivatives, and 1/(2 dx)
            T sm[D], df[D], hh[D];
            const T ppx = bz[s_pxp + 1];
            const T ppy = bz[s_pyr];
            sm[0] = pmx + ppx;
            df[0] = ppx - pmx;
            hh[0] = h0;
            sm[1] = pmy + ppy;
            df[1] = ppy - pmy;
            hh[1] = h1;
            T next = T(0);
            if constexpr (D >= 3) {
                T pps;
                if constexpr (kSlide) {
                    zline.slide(q[4], q[5]);
                    zline.eval(flS, pps, next);
                } else {
                    iface_at<SCHEME>(q[0], q[1], q[2], q[3], q[4], q[5], flS, pps, next);
                }
                sm[SD] = carry + pps;
                df[SD] = pps - carry;
                hh[SD] = hS;
            }
            if constexpr (D == 4) {
                // dimension 2: both interfaces of the node from a 7-point line
                T v[7];
                gather7<T>(u, (long long)(col + fz), i2, g.n[2], g.stride[2], (g.periodic_mask >> 2) & 1u, extrap, v);
                T pm2, pp2, unused0, unused1;
                const T fl2 = SP<T>::floor(P, 2);
                iface_at<SCHEME>(v[0], v[1], v[2], v[3], v[4], v[5], fl2, unused0, pm2);
                iface_at<SCHEME>(v[1], v[2], v[3], v[4], v[5], v[6], fl2, pp2, unused1);
                sm[2] = pm2 + pp2;
                df[2] = pp2 - pm2;
                hh[2] = half_inv(2);
                if constexpr (uses_coord<D, DYN>(3)) xc[3] = coord(SP<T>::lo(P, 3), z, SP<T>::dx(P, 3));
            }
            if constexpr (D == 3 && uses_coord<D, DYN>(2)) xc[2] = coord(SP<T>::lo(P, 2), z, SP<T>::dx(P, 2));
            T yd = lf_combine_raw<T, D, DYN>(P, xc, cosz, sinz, sm, df, hh, alpha_global);
            if constexpr (std::is_same<T, double>::value) {
                // BRT min(0, .) on the bit pattern: positive values (and +NaN) become 0
                if (brt0 && __double_as_longlong(yd) > 0) yd = 0.0;
            } else {
                yd = fminf(yd, clamp);
            }
            const int flat = col + fz;
            T res;
            if constexpr (KIND == kKindTerm) {
                res = yd;
            } else if constexpr (KIND == kKindFirst) {
                res = center + dt * yd;
            } else {
                if constexpr (!kVnAhead) vv = ld(vn + flat);
                res = cv * vv + cu * (center + dt * yd);
                if (minv) res = fmin(res, vv);
            }
            out[flat] = res;
            if (also_out) also_out[flat] = res;
            if constexpr (D >= 3) {
                carry = next;
#pragma unroll
                for (int k = 0; k < 5; ++k) q[k] = q[k + 1];
            }
        }
    }
}

// Whether tile (row_tile, chunk) is interior: all its TY rows and three halo
// rows on each side inside the grid along dimension 1, and its chunk's planes
// with three on each side inside the grid along the streamed dimension.
template <int D>
__device__ __forceinline__ bool rows_interior(const GridDev& g, int ty, int tz, int row_tile, int chunk) {
    const int y0 = row_tile * ty;
    bool in = y0 >= 3 && y0 + ty + 3 <= g.n[1];
    if constexpr (D >= 3) {
        const int zbeg = chunk * tz, zend = min(g.n[D - 1], zbeg + tz);
        in = in && zbeg >= 3 && zend + 3 <= g.n[D - 1];
    }
    return in;
}

template <typename T, int D, int DYN, int SCHEME, int KIND, int OCC>
__global__ void __launch_bounds__(RowsBounds<T, OCC>::kThreads, OCC) rows_kernel(const StageParams P, const RowsCfg C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const StageRun<T> R = stage_run<T>(P);
    const int i2 = (D == 4) ? (int)blockIdx.y : 0;
    const int chunk = (D == 3) ? (int)blockIdx.y : ((D == 4) ? (int)blockIdx.z : 0);
    // the interior body is compiled for the ENO schemes only: there it pays
    // (their per-node arithmetic is small beside the staging logic), while a
    // second WENO5 body measured slower in FP32 and no faster in FP64
    if constexpr (SCHEME != HJ_WENO5) {
        if (C.split && rows_interior<D>(P.g, C.ty, C.tz, blockIdx.x, chunk)) {
            rows_tile<T, D, DYN, SCHEME, KIND, true>(P, R, C.ty, C.nt, C.tz, blockIdx.x, i2, chunk, threadIdx.x,
                                                     reinterpret_cast<T*>(smem_raw));
            return;
        }
    }
    rows_tile<T, D, DYN, SCHEME, KIND, false>(P, R, C.ty, C.nt, C.tz, blockIdx.x, i2, chunk, threadIdx.x,
                                              reinterpret_cast<T*>(smem_raw));
}

// Shared memory of a rows_kernel block.
template <typename T>
inline size_t rows_smem_bytes(int nx, int ty) {
    return rows_smem(nx, ty, sizeof(T));
}

template <typename T, int D, int DYN>
inline void rows_shape(const StageParams& p, const RowsCfg& c, dim3& grid, dim3& block, size_t& smem) {
    block = dim3((unsigned)c.nt, 1, 1);
    grid = dim3((unsigned)c.row_tiles, 1, 1);
    if (D == 3) grid.y = (unsigned)c.nchunks;
    if (D == 4) { grid.y = (unsigned)p.g.n[2]; grid.z = (unsigned)c.nchunks; }
    smem = rows_smem_bytes<T>(p.g.n[0], c.ty);
}

// Opts a kernel into 200 KiB of dynamic shared memory, once per device (the
// attribute belongs to the current device's copy of the kernel); `done` holds
// one bit per device already set (devices 0..63; others are set every call).
template <typename K>
inline cudaError_t smem_optin(K* kernel, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    done.fetch_or(bit, std::memory_order_relaxed);  // setting the attribute twice (a race) is harmless
    return cudaSuccess;
}

template <typename T, int D, int DYN, int SCHEME, int KIND, int OCC>
inline cudaError_t rows_prepare() {
    static std::atomic<unsigned long long> done{0};
    return smem_optin(rows_kernel<T, D, DYN, SCHEME, KIND, OCC>, done);
}

template <typename T, int D, int DYN, int SCHEME, int KIND, int OCC>
cudaError_t launch_rows_occ(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    dim3 grid, block;
    size_t smem;
    rows_shape<T, D, DYN>(p, c, grid, block, smem);
    cudaError_t e = rows_prepare<T, D, DYN, SCHEME, KIND, OCC>();
    if (e != cudaSuccess) return e;
    rows_kernel<T, D, DYN, SCHEME, KIND, OCC><<<grid, block, smem, s>>>(p, c);
    return cudaGetLastError();
}

// The variant for two blocks per SM exists for FP32 only.
template <typename T, int D, int DYN, int SCHEME, int KIND>
cudaError_t launch_rows_kind(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (c.occ == 2) return launch_rows_occ<T, D, DYN, SCHEME, KIND, 2>(p, c, s);
    }
    return launch_rows_occ<T, D, DYN, SCHEME, KIND, 1>(p, c, s);
}

template <typename T, int D, int DYN, int SCHEME>
cudaError_t launch_rows_scheme(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    switch (stage_kind(p)) {
    case kKindTerm: return launch_rows_kind<T, D, DYN, SCHEME, kKindTerm>(p, c, s);
    case kKindFirst: return launch_rows_kind<T, D, DYN, SCHEME, kKindFirst>(p, c, s);
    default: return launch_rows_kind<T, D, DYN, SCHEME, kKindCombine>(p, c, s);
    }
}
template <typename T, int D, int DYN>
cudaError_t launch_rows_weno5(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    return launch_rows_scheme<T, D, DYN, HJ_WENO5>(p, c, s);
}
template <typename T, int D, int DYN>
cudaError_t launch_rows_eno2(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    return launch_rows_scheme<T, D, DYN, HJ_ENO2>(p, c, s);
}
template <typename T, int D, int DYN>
cudaError_t launch_rows_eno1(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    return launch_rows_scheme<T, D, DYN, HJ_ENO1>(p, c, s);
}
template <typename T, int D, int DYN>
cudaError_t launch_rows_eno3(const StageParams& p, const RowsCfg& c, cudaStream_t s) {
    return launch_rows_scheme<T, D, DYN, HJ_ENO3>(p, c, s);
}

template <typename T, int D, int DYN, int SCHEME, int OCC>
int rows_bps_occ(const StageParams& p, const RowsCfg& c) {
    dim3 grid, block;
    size_t smem;
    rows_shape<T, D, DYN>(p, c, grid, block, smem);
    if ((int)block.x > RowsBounds<T, OCC>::kThreads) return 0;
    if (rows_prepare<T, D, DYN, SCHEME, kKindCombine, OCC>() != cudaSuccess) return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rows_kernel<T, D, DYN, SCHEME, kKindCombine, OCC>,
                                                      (int)block.x, smem) != cudaSuccess)
        return 0;
    return bps;
}

// Resident blocks per SM of the stage kernels of a configuration (the
// combining stages, the largest of the three kinds); 0 if it cannot launch.
template <typename T, int D, int DYN, int SCHEME>
int rows_bps_scheme(const StageParams& p, const RowsCfg& c) {
    if constexpr (std::is_same<T, float>::value) {
        if (c.occ == 2) return rows_bps_occ<T, D, DYN, SCHEME, 2>(p, c);
    }
    return rows_bps_occ<T, D, DYN, SCHEME, 1>(p, c);
}
template <typename T, int D, int DYN>
int rows_bps_weno5(const StageParams& p, const RowsCfg& c) {
    return rows_bps_scheme<T, D, DYN, HJ_WENO5>(p, c);
}
template <typename T, int D, int DYN>
int rows_bps_eno2(const StageParams& p, const RowsCfg& c) {
    return rows_bps_scheme<T, D, DYN, HJ_ENO2>(p, c);
}
template <typename T, int D, int DYN>
int rows_bps_eno1(const StageParams& p, const RowsCfg& c) {
    return rows_bps_scheme<T, D, DYN, HJ_ENO1>(p, c);
}
template <typename T, int D, int DYN>
int rows_bps_eno3(const StageParams& p, const RowsCfg& c) {
    return rows_bps_scheme<T, D, DYN, HJ_ENO3>(p, c);
}

// Dispatch over the (dimension, dynamics) pairs the row kernel is built for.
#define HJ_ROWS_DISPATCH(FN, T, ...)                                                   \
    switch (p.g.ndim * 16 + p.dynamics) {                                              \
    case 2 * 16 + HJ_DYN_DOUBLE_INTEGRATOR: return FN<T, 2, HJ_DYN_DOUBLE_INTEGRATOR>(__VA_ARGS__); \
    case 2 * 16 + HJ_DYN_NORM: return FN<T, 2, HJ_DYN_NORM>(__VA_ARGS__);             \
    case 2 * 16 + HJ_DYN_ADVECT: return FN<T, 2, HJ_DYN_ADVECT>(__VA_ARGS__);         \
    case 2 * 16 + HJ_DYN_ROTATE: return FN<T, 2, HJ_DYN_ROTATE>(__VA_ARGS__);         \
    case 3 * 16 + HJ_DYN_AIR3D: return FN<T, 3, HJ_DYN_AIR3D>(__VA_ARGS__);           \
    case 3 * 16 + HJ_DYN_ROCKETS: return FN<T, 3, HJ_DYN_ROCKETS>(__VA_ARGS__);       \
    case 3 * 16 + HJ_DYN_NORM: return FN<T, 3, HJ_DYN_NORM>(__VA_ARGS__);             \
    case 3 * 16 + HJ_DYN_ADVECT: return FN<T, 3, HJ_DYN_ADVECT>(__VA_ARGS__);         \
    case 3 * 16 + HJ_DYN_ROTATE: return FN<T, 3, HJ_DYN_ROTATE>(__VA_ARGS__);         \
    case 4 * 16 + HJ_DYN_DUBINS4D: return FN<T, 4, HJ_DYN_DUBINS4D>(__VA_ARGS__);     \
    default: break;                                                                    \
    }

// The variants with dissipation local in p (HJ_ALPHA_BOX) of the dynamics
// whose slopes depend on p; instantiated in translation units of their own.
#define HJ_ROWS_BOX_DISPATCH(FN, T, ...)                                                                  \
    switch (p.g.ndim * 16 + p.dynamics) {                                                                  \
    case 2 * 16 + HJ_DYN_NORM: return FN<T, 2, HJ_DYN_NORM + kDynBox>(__VA_ARGS__);                        \
    case 3 * 16 + HJ_DYN_NORM: return FN<T, 3, HJ_DYN_NORM + kDynBox>(__VA_ARGS__);                        \
    case 3 * 16 + HJ_DYN_AIR3D: return FN<T, 3, HJ_DYN_AIR3D + kDynBox>(__VA_ARGS__);                      \
    case 3 * 16 + HJ_DYN_ROCKETS: return FN<T, 3, HJ_DYN_ROCKETS + kDynBox>(__VA_ARGS__);                  \
    default: break;                                                                                        \
    }


}  // namespace hj
