// static_step.cu -- hj_rk3_step_static: one TVD-RK3 step that allocates no
// memory. Its two stage buffers and the heading-angle tables live in one
// file-scope __device__ array of fixed size, shared by every call in the
// process.
//
// Why: some callers may not allocate device memory once they are running --
// a real-time control loop (a safety filter re-solving its reachable set
// every cycle) that forbids allocation after start-up because cudaMalloc can
// block and fragment, or a host application that owns the GPU's memory pool
// and forbids any other allocator. This entry point lets them step a value
// function in a buffer they already own.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/hj.h"
#include "hj_internal.h"

namespace {

using namespace hj;

constexpr size_t kStageBytes = (size_t)HJ_STATIC_MAX_NODES * sizeof(double);  // one stage buffer, FP64 worth
constexpr size_t kAngleBytes = (size_t)HJ_STATIC_MAX_ANGLES * 2 * (sizeof(double) + sizeof(float));
constexpr size_t kScratchBytes = 2 * kStageBytes + kAngleBytes;

// The scratch. In host code this name is only a stand-in for the symbol; the
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
// (n, lo, dx) of the angle tables last written into each device's scratch
double g_angle_key[kMaxDevices][3];
bool g_angle_valid[kMaxDevices] = {false};
// host staging of the tables (filled under g_mutex; consumed by the copy before it returns)
double g_angle_host_d[2 * HJ_STATIC_MAX_ANGLES];
float g_angle_host_f[2 * HJ_STATIC_MAX_ANGLES];

// Device address of the scratch on `device` (which must be current).
hj_status scratch_address(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HJ_ECUDA;
        g_scratch_ptr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
    return HJ_OK;
}

// cos and sin of the dimension-2 coordinate, both precisions, from the host
// math library (the values every other entry point uses), written into the
// scratch on `stream` when the device's tables hold other angles. The copy
// from pageable host memory has consumed its source when it returns.
hj_status angle_tables(int device, int n, double lo, double dx, double* td, float* tf, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g_mutex);
    double* key = g_angle_key[device];
    if (g_angle_valid[device] && key[0] == (double)n && key[1] == lo && key[2] == dx) return HJ_OK;
    for (int i = 0; i < n; ++i) {
        const double x = lo + (double)i * dx;
        g_angle_host_d[i] = std::cos(x);
        g_angle_host_d[n + i] = std::sin(x);
        g_angle_host_f[i] = (float)g_angle_host_d[i];
        g_angle_host_f[n + i] = (float)g_angle_host_d[n + i];
    }
    g_angle_valid[device] = false;
    if (cudaMemcpyAsync(td, g_angle_host_d, 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(tf, g_angle_host_f, 2 * (size_t)n * sizeof(float), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess)
        return HJ_ECUDA;
    key[0] = (double)n;
    key[1] = lo;
    key[2] = dx;
    g_angle_valid[device] = true;
    return HJ_OK;
}

bool grid_valid(const hj_grid* g) {
    if (!g || g->ndim < 1 || g->ndim > 4 || (g->periodic_mask >> g->ndim)) return false;
    for (int d = 0; d < g->ndim; ++d) {
        const bool periodic = (g->periodic_mask >> d) & 1u;
        if (g->n[d] < (periodic ? 1 : 2)) return false;
        if (!std::isfinite(g->lo[d]) || !std::isfinite(g->hi[d]) || !(g->hi[d] > g->lo[d])) return false;
    }
    return true;
}

bool method_valid(const hj_grid* g, const hj_method* m) {
    if (!m) return false;
    if (m->scheme != HJ_ENO1 && m->scheme != HJ_ENO2 && m->scheme != HJ_ENO3 && m->scheme != HJ_WENO5) return false;
    if (m->brt < HJ_BRT_NONE || m->brt > HJ_BRT_MINV) return false;
    if (m->extrap != HJ_EXTRAP_AWAY_FROM_ZERO && m->extrap != HJ_EXTRAP_LINEAR) return false;
    for (int k = 0; k < 8; ++k)
        if (!std::isfinite(m->params[k])) return false;
    if ((m->order != 0 && m->order != 3) || m->alpha_mode != HJ_ALPHA_NODE) return false;
    if (m->kernel != HJ_KERNEL_AUTO && m->kernel != HJ_KERNEL_NODE) return false;
    for (int k = 0; k < 4; ++k)
        if (m->tile_override[k] != 0) return false;
    const int D = g->ndim;
    switch (m->dynamics) {
    case HJ_DYN_DOUBLE_INTEGRATOR: return D == 2 && m->params[0] >= 0;
    case HJ_DYN_AIR3D: return D == 3 && m->params[2] >= 0 && m->params[3] >= 0;
    case HJ_DYN_DUBINS4D: return D == 4 && m->params[0] >= 0 && m->params[1] >= 0;
    case HJ_DYN_NORM: return D <= 3 && m->params[0] >= 0;
    case HJ_DYN_ADVECT: return D <= 3;
    case HJ_DYN_ROTATE: return D >= 2 && D <= 3;
    case HJ_DYN_ROCKETS: return D == 3 && m->params[2] >= 0 && m->params[3] >= 0;
    default: return false;
    }
}

// Launch shape of the row kernel without timing: the fewest rows per tile
// that give at least 256 threads, and planes per chunk so that the blocks
// fill the SMs about twice.
bool pick_rows(const StageParams& P, int dtype, int sm_count, RowsCfg* c) {
    const GridDev& G = P.g;
    const int D = G.ndim;
    if (!rows_supported(D, P.dynamics)) return false;
    for (int d = 0; d < D; ++d)
        if (G.n[d] < 4) return false;
    const int max_threads = rows_max_threads(dtype == HJ_F64);
    const int nx = G.n[0], ny = G.n[1];
    if (nx + 1 > max_threads) return false;
    int ty = 1;
    while (ty < ny && (nx + 1) * (ty + 2) <= max_threads && (nx + 1) * ty < 256) ++ty;
    const size_t es = dtype == HJ_F64 ? 8 : 4;
    if (rows_smem(nx, ty, es) > 200 * 1024) return false;
    c->ty = ty;
    c->nt = rows_block_threads(nx, ty, max_threads);
    c->occ = 1;
    c->split = 1;  // interior tiles on the body without ghost logic (the same bits either way)
    c->row_tiles = (ny + ty - 1) / ty;
    const int ns = D >= 3 ? G.n[D - 1] : 1;
    const long long per_plane = (long long)c->row_tiles * (D == 4 ? G.n[2] : 1);
    int tz = ns;
    if (D >= 3) {
        const long long want = 2LL * sm_count;
        const long long chunks = (want + per_plane - 1) / per_plane;
        tz = (int)std::max(1LL, (ns + chunks - 1) / std::max(1LL, chunks));
    }
    c->tz = D >= 3 ? tz : 1;
    c->nchunks = D >= 3 ? (ns + c->tz - 1) / c->tz : 1;
    if (c->nchunks > 65535) return false;
    const int bps = dtype == HJ_F64 ? rows_blocks_per_sm_f64(P, *c) : rows_blocks_per_sm_f32(P, *c);
    return bps > 0;
}

}  // namespace

extern "C" hj_status hj_rk3_step_static(void* cuda_stream, int32_t device, const hj_grid* grid,
                                        const hj_method* method, int32_t dtype, void* v, double dt) {
    if (!grid_valid(grid) || !method_valid(grid, method)) return HJ_EINVAL;
    if (dtype != HJ_F32 && dtype != HJ_F64) return HJ_EINVAL;
    if (!v || !(dt >= 0.0) || !std::isfinite(dt)) return HJ_EINVAL;
    if (device < 0 || device >= kMaxDevices) return HJ_EINVAL;
    long long total = 1;
    for (int d = 0; d < grid->ndim; ++d) {
        if (grid->n[d] > HJ_STATIC_MAX_NODES) return HJ_EINVAL;  // checked before the product can overflow
        total *= grid->n[d];
        if (total > HJ_STATIC_MAX_NODES) return HJ_EINVAL;  // beyond the fixed scratch
    }
    const bool angles = method->dynamics == HJ_DYN_AIR3D || method->dynamics == HJ_DYN_DUBINS4D ||
                        method->dynamics == HJ_DYN_ROCKETS;
    if (angles && grid->n[2] > HJ_STATIC_MAX_ANGLES) return HJ_EINVAL;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return HJ_ECUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return HJ_ECUDA;
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, device};

    unsigned char* base = nullptr;
    hj_status st = scratch_address(device, &base);
    if (st != HJ_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // the kernels' view of the grid (same spacing rule as every other entry point)
    StageParams P;
    std::memset(&P, 0, sizeof P);
    GridDev& G = P.g;
    G.ndim = grid->ndim;
    long long stride = 1;
    for (int d = 0; d < 4; ++d) {
        if (d < grid->ndim) {
            const bool periodic = (grid->periodic_mask >> d) & 1u;
            G.n[d] = (int)grid->n[d];
            G.stride[d] = stride;
            stride *= grid->n[d];
            G.lo[d] = grid->lo[d];
            G.dx[d] = (grid->hi[d] - grid->lo[d]) / (periodic ? (double)grid->n[d] : (double)(grid->n[d] - 1));
            G.inv_dx[d] = 1.0 / G.dx[d];
        } else {
            G.n[d] = 1;
            G.stride[d] = stride;
            G.dx[d] = 1.0;
            G.inv_dx[d] = 1.0;
        }
    }
    G.total = stride;
    G.periodic_mask = grid->periodic_mask;
    G.extrap = method->extrap;
    P.dynamics = method->dynamics;
    for (int k = 0; k < 8; ++k) P.params[k] = method->params[k];
    P.brt_min0 = method->brt == HJ_BRT_MIN0;
    // WENO5 epsilon floor per dimension in raw-difference units (1e-99 on divided differences in FP64)
    for (int d = 0; d < 4; ++d) P.weno_floor[d] = dtype == HJ_F32 ? (double)kWenoFloorF32 : 1e-99 * G.dx[d] * G.dx[d];

    void* w1 = base;
    void* w2 = base + kStageBytes;
    double* td = reinterpret_cast<double*>(base + 2 * kStageBytes);
    float* tf = reinterpret_cast<float*>(base + 2 * kStageBytes + (size_t)HJ_STATIC_MAX_ANGLES * 2 * sizeof(double));
    if (angles && (st = angle_tables(device, G.n[2], G.lo[2], G.dx[2], td, tf, stream)) != HJ_OK) return st;
    P.trig_d = td;
    P.trig_f = tf;

    int sm_count = 0;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HJ_ECUDA;
    RowsCfg cfg;
    P.scheme = method->scheme;
    // every scheme has a row-kernel variant; kernel = HJ_KERNEL_NODE asks for the other kernel
    const bool rows = method->kernel != HJ_KERNEL_NODE && pick_rows(P, dtype, sm_count, &cfg);

    // stage 1: w1 = v + dt L(v); stage 2: w2 = 3/4 v + 1/4 (w1 + dt L(w1));
    // stage 3: v = 1/3 v + 2/3 (w2 + dt L(w2)) [then min(., v) for the min-V rule]
    const void* ins[3] = {v, w1, w2};
    void* outs[3] = {w1, w2, v};
    const double cvs[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cus[3] = {1.0, 0.25, 2.0 / 3.0};
    P.mode = kStage;
    P.dt = dt;
    for (int s = 0; s < 3; ++s) {
        P.u = ins[s];
        P.vn = s == 0 ? nullptr : v;
        P.out = outs[s];
        P.cv = cvs[s];
        P.cu = cus[s];
        P.minv_after = (s == 2 && method->brt == HJ_BRT_MINV);
        const StageParams Q = finalize(P);
        cudaError_t e;
        if (rows) e = dtype == HJ_F64 ? launch_rows_f64(Q, cfg, stream) : launch_rows_f32(Q, cfg, stream);
        else e = dtype == HJ_F64 ? launch_stage_f64(Q, method->scheme, stream) : launch_stage_f32(Q, method->scheme, stream);
        if (e != cudaSuccess) return HJ_ECUDA;
    }
    return HJ_OK;
}
