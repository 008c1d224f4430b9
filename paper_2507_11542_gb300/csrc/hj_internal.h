// hj_internal.h -- host/device shared declarations of the GB300 level-set
// library (not part of the public ABI; the ABI is include/hj.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace hj {

constexpr int kMaxDim = 4;

// WENO5 epsilon floor of FP32 kernels, in raw-difference units: 1e-99 (the
// FP64 floor) underflows in FP32; with 1e-18 the squared sums stay normal.
constexpr float kWenoFloorF32 = 1e-18f;

// Row and batch kernels take the dynamics as a template parameter. For the
// Hamiltonians whose |dHg/dp_d| depends on p (norm, air3D, rockets), the
// variant with Lax-Friedrichs dissipation local in p (HJ_ALPHA_BOX) is the
// dynamics id plus kDynBox; the other dynamics need no such variant (their
// box maximum is the maximum over every p).
constexpr int kDynBox = 8;
__host__ __device__ constexpr int dyn_base(int dyn) { return dyn & (kDynBox - 1); }
__host__ __device__ constexpr bool dyn_is_box(int dyn) { return (dyn & kDynBox) != 0; }
__host__ __device__ inline bool box_differs(int dyn) {
    return dyn == 4 /* HJ_DYN_NORM */ || dyn == 2 /* HJ_DYN_AIR3D */ || dyn == 7 /* HJ_DYN_ROCKETS */;
}

// A named NVTX range for the lifetime of the object: solves, steps, batched
// graph replays and server admissions show up as ranges in a profiler's
// timeline (header-only NVTX: inert unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Largest block of the row-tiled kernels: FP32 blocks may hold 1024 threads
// (<= 64 registers each), FP64 blocks 512 (<= 128 registers), since the FP64
// interface arithmetic needs more registers.
constexpr int kRowsMaxThreadsF32 = 1024;
constexpr int kRowsMaxThreadsF64 = 512;
inline int rows_max_threads(int dtype_is_f64) { return dtype_is_f64 ? kRowsMaxThreadsF64 : kRowsMaxThreadsF32; }
// The FP32 row kernel also exists compiled for two resident blocks per SM
// (<= 56 registers a thread) of at most this many threads.
constexpr int kRowsOcc2Threads = 544;

// Grid as the kernels see it. Spacing and its inverse are computed once on
// the host from the hj_grid (periodic: (hi-lo)/n, else (hi-lo)/(n-1)).
struct GridDev {
    int ndim;
    int n[kMaxDim];
    long long stride[kMaxDim];
    long long total;
    double lo[kMaxDim];
    double dx[kMaxDim];
    double inv_dx[kMaxDim];
    unsigned periodic_mask;
    int extrap;  // HJ_EXTRAP_*
};

// What one launch of the fused stage kernel computes at every node:
//   w   = U + dt * ydot(U)            (mode kStage*)  or  w = ydot(U)  (mode kTerm)
//   out = cv * Vn + cu * w            (cv == 0: out = w)
//   out = min(out, Vn)                (minv_after: BRT "min(V, V_prev)" rule)
enum StageMode { kTerm = 0, kStage = 1 };

struct StageParams {
    GridDev g;
    int dynamics;
    double params[8];
    int brt_min0;     // clamp ydot at zero (BRT min(0, H))
    int minv_after;   // out = min(out, Vn)
    int mode;         // StageMode
    int scheme;       // HJ_ENO1/2/3 or HJ_WENO5 (row kernel); the one-node kernel takes it as an argument
    double dt;
    double cv, cu;    // stage combination coefficients
    const void* u;    // stencil input
    const void* vn;   // V^n (read at the node only); may be null when cv == 0 and !minv_after
    void* out;
    const double* trig_d;  // cos, sin of the dimension-2 coordinate: [cos(0..n2-1), sin(0..n2-1)]
    const float* trig_f;
    double weno_floor[kMaxDim];   // additive floor of the WENO5 epsilon per dimension, in raw-difference units
    double half_inv_dx[kMaxDim];  // 1 / (2 dx): raw differences to (p- + p+)/2 and (p+ - p-)/2
    double half_inv_dx6[kMaxDim]; // 1 / (12 dx): the same from six times the raw differences (WENO5)
    int alpha_global;             // dissipation alpha_d = alpha_g[d] (global LF) instead of alpha_d(x)
    double alpha_g[kMaxDim];
    int alpha_box;                // dissipation alpha_d = max |dHg/dp_d| over the node's box of gradients
    // FP32 copies of the scalars above, so that FP32 kernels do no FP64 arithmetic
    float lo_f[kMaxDim], dx_f[kMaxDim], inv_dx_f[kMaxDim], half_inv_dx_f[kMaxDim], half_inv_dx6_f[kMaxDim];
    float alpha_g_f[kMaxDim];
    float weno_floor_f[kMaxDim];
    float params_f[8];
    float dt_f, cv_f, cu_f;
    int has_vn;            // the stage reads Vn (cv != 0 or minv_after)
};

// Whether a row-kernel launch takes a variant with dissipation local in p
// (rows_f32_box.cu, rows_f64_box.cu).
inline bool rows_box_variant(const StageParams& p) { return p.alpha_box && box_differs(p.dynamics); }

// Fills the FP32 copies and has_vn from the FP64 fields (call before launching).
inline StageParams finalize(StageParams p) {
    for (int d = 0; d < kMaxDim; ++d) {
        p.lo_f[d] = (float)p.g.lo[d];
        p.dx_f[d] = (float)p.g.dx[d];
        p.inv_dx_f[d] = (float)p.g.inv_dx[d];
        p.half_inv_dx[d] = 0.5 * p.g.inv_dx[d];
        p.half_inv_dx6[d] = p.half_inv_dx[d] / 6.0;
        p.half_inv_dx6_f[d] = (float)p.half_inv_dx6[d];
        p.half_inv_dx_f[d] = (float)p.half_inv_dx[d];
        p.alpha_g_f[d] = (float)p.alpha_g[d];
        p.weno_floor_f[d] = (float)p.weno_floor[d];
    }
    for (int k = 0; k < 8; ++k) p.params_f[k] = (float)p.params[k];
    p.dt_f = (float)p.dt;
    p.cv_f = (float)p.cv;
    p.cu_f = (float)p.cu;
    p.has_vn = (p.mode == kStage) && (p.cv != 0.0 || p.minv_after);
    return p;
}

// What the row kernels store per node, by launch (a template parameter, so
// that no per-node branch remains): the stage term alone, the first RK
// stage (no V^n), or a combination with V^n (stages 2 and 3).
enum StageKind { kKindTerm = 0, kKindFirst = 1, kKindCombine = 2 };
inline int stage_kind(const StageParams& p) {  // p finalized
    return p.mode == kTerm ? kKindTerm : (p.has_vn ? kKindCombine : kKindFirst);
}

struct UpwindParams {
    GridDev g;
    int dim;
    const void* u;
    void* pm;
    void* pp;
    double weno_floor;
};

// Launch configuration of the row-tiled stage kernel (rows_kernel.cuh).
struct RowsCfg {
    int ty;         // node rows per tile
    int nt;         // threads per block (1-D): rows_block_threads(n0, ty, ...), or n0*ty (no row-end threads)
    int tz;         // planes per chunk along the streamed (last) dimension
    int nchunks;    // chunks along the streamed dimension
    int row_tiles;  // ceil(n1 / ty)
    int occ;        // 1, or 2: FP32 kernel compiled for two resident blocks of <= kRowsOcc2Threads threads per SM
    int split;      // 1: interior tiles take the body compiled without ghost and wrap logic (ENO schemes)
};

// Threads of a row-kernel block with ty node rows of n0 nodes: one thread per
// node, one per row for the row's last dimension-0 interface and ghost cells,
// and, where the block size allows it, one per column for the tile's last
// dimension-1 interface (without them thread row 0 evaluates those).
inline bool rows_gap_threads(int nx, int ty, int threads) { return nx * ty + ty + nx <= threads; }
inline int rows_block_threads(int nx, int ty, int max_threads) {
    return nx * ty + ty + (rows_gap_threads(nx, ty, max_threads) ? nx : 0);
}

// Elements of one of the two alternating shared buffers of a rows_kernel
// block: (ty + 6) padded rows of n0 + 6, then p+ along dimension 0 (ty rows
// of n0 + 1), along dimension 1 (ty + 1 rows of n0), and the two outermost
// values at each end of every node row (4 per row, for the ghost cells).
__host__ __device__ inline size_t rows_buf_elems(int nx, int ty) {
    return (size_t)(ty + 6) * (size_t)(nx + 6) + (size_t)ty * (size_t)(nx + 1) + (size_t)(ty + 1) * (size_t)nx +
           4 * (size_t)ty;
}

// Dynamic shared memory of a rows_kernel block (element size es).
inline size_t rows_smem(int nx, int ty, size_t es) {
    return 2 * es * rows_buf_elems(nx, ty);
}

// Launchers (one translation unit per element type). Return the launch error.
cudaError_t launch_stage_f64(const StageParams& p, int scheme, cudaStream_t s);
cudaError_t launch_stage_f32(const StageParams& p, int scheme, cudaStream_t s);
cudaError_t launch_upwind_f64(const UpwindParams& p, int scheme, cudaStream_t s);
cudaError_t launch_upwind_f32(const UpwindParams& p, int scheme, cudaStream_t s);

// Row-tiled stage kernel (every scheme): defined for D = 2 (double integrator, norm,
// advection, rotation), D = 3 (air3D, rockets, norm, advection, rotation), D = 4 (Dubins4D).
bool rows_supported(int ndim, int dynamics);
cudaError_t launch_rows_f64(const StageParams& p, const RowsCfg& c, cudaStream_t s);
cudaError_t launch_rows_f32(const StageParams& p, const RowsCfg& c, cudaStream_t s);
// resident blocks per SM of a configuration (0 if it cannot launch)
int rows_blocks_per_sm_f64(const StageParams& p, const RowsCfg& c);
int rows_blocks_per_sm_f32(const StageParams& p, const RowsCfg& c);

// ---------------------------------------------------------------------------
// Batched solves: many instances advanced together by one launch per stage
// over a list of tiles (batch.cuh).
// ---------------------------------------------------------------------------
struct BatchTile {
    int inst;      // instance index
    int row_tile;  // rows row_tile*ty .. of the instance's planes
    int i2;        // dimension-2 index (4-D instances)
    int chunk;     // chunk along the streamed dimension
};

struct BatchInst {
    StageParams P;            // grid, dynamics, parameters (FP64 + FP32), angle tables, WENO floor
    int ty, tz;               // tile shape of this instance
    int steps_total;          // RK3 steps of the whole solve
    int k;                    // steps completed (advanced on the device)
    double dt;                // dt of the current step
    float dt_f;
    int brt;                  // HJ_BRT_*
    void* V;                  // value function (in place)
    void* V1;                 // stage buffers
    void* V2;
    void* slice_out;          // stage 3 of the current step also writes here, or null
    double dt_full;           // dt of every step that does not end a slice: min(max_step, cfl/stepBoundInv)
    const long long* ends;    // distinct positive step counts at which slices are taken, ascending
    const int* end_slice;     // slice index written at each of those
    const double* end_dt;     // dt of the step that completes each of those (clipped to the slice time)
    int n_ends;
    int cursor;               // next entry of ends not yet scheduled
    void* out;                // slice outputs: n_slices x nodes elements
    long long nodes;
    int elem;                 // element size in bytes
    int lane;                 // rate class: advanced by the step graphs of lanes 0 .. lane
};

cudaError_t launch_batch_stage_f32(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int ndim,
                                   int dynamics, int scheme, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_batch_stage_f64(const BatchTile* tiles, int ntiles, const BatchInst* insts, int stage, int ndim,
                                   int dynamics, int scheme, int threads, size_t smem, cudaStream_t s);
// Advances the instances of lanes lane_lo .. lane_hi (BatchInst::lane).
cudaError_t launch_batch_advance(BatchInst* insts, int n, int lane_lo, int lane_hi, cudaStream_t s);

// max over nodes of sum_d alpha_d(x)/dx_d, as the FP64 bit pattern, atomically
// max-ed into *acc (which the caller zeroes first).
cudaError_t launch_step_bound(const GridDev& g, int dynamics, const double* params, const double* trig_d,
                              unsigned long long* acc, int per_dim, cudaStream_t s);
// Sets *flag to 1 if any of the n elements is NaN or +-Inf.
cudaError_t launch_nonfinite_f64(const double* v, long long n, int* flag, cudaStream_t s);
cudaError_t launch_nonfinite_f32(const float* v, long long n, int* flag, cudaStream_t s);

}  // namespace hj
