// hj_api.cu -- the C ABI of include/hj.h: context, argument validation, the
// per-row entry points and the time loop of Sec. 5 (Listing 6).
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/hj.h"
#include "hj_internal.h"
#include "ctx.h"
#include "engine.h"


namespace hj {

hj_status fail(hj_ctx* ctx, hj_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

hj_status cuda_fail(hj_ctx* ctx, cudaError_t e, const char* what) {
    // A failed allocation is not sticky, but the runtime also records it as the
    // thread's last error: clear it, or the next launch check would report it.
    if (e == cudaErrorMemoryAllocation) (void)cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? HJ_ENOMEM : HJ_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}


size_t elem_size(int dtype) { return dtype == HJ_F64 ? 8 : (dtype == HJ_F32 ? 4 : 0); }

hj_status check_grid(hj_ctx* ctx, const hj_grid* g) {
    if (!g) return fail(ctx, HJ_EINVAL, "grid is NULL");
    if (g->ndim < 1 || g->ndim > 4) return fail(ctx, HJ_EINVAL, "ndim %d not in 1..4", g->ndim);
    long long total = 1;
    for (int d = 0; d < g->ndim; ++d) {
        const bool periodic = (g->periodic_mask >> d) & 1u;
        if (g->n[d] < (periodic ? 1 : 2)) return fail(ctx, HJ_EINVAL, "n[%d] = %lld too small", d, (long long)g->n[d]);
        if (g->n[d] > (1ll << 30)) return fail(ctx, HJ_EINVAL, "n[%d] too large", d);
        if (!std::isfinite(g->lo[d]) || !std::isfinite(g->hi[d]) || !(g->hi[d] > g->lo[d]))
            return fail(ctx, HJ_EINVAL, "bounds of dimension %d are not finite with hi > lo", d);
        total *= g->n[d];
        if (total > (1ll << 40)) return fail(ctx, HJ_EINVAL, "grid too large");
    }
    if (g->periodic_mask >> g->ndim) return fail(ctx, HJ_EINVAL, "periodic_mask names a dimension >= ndim");
    return HJ_OK;
}

hj_status check_method(hj_ctx* ctx, const hj_grid* g, const hj_method* m) {
    if (!m) return fail(ctx, HJ_EINVAL, "method is NULL");
    if (m->scheme != HJ_ENO1 && m->scheme != HJ_ENO2 && m->scheme != HJ_ENO3 && m->scheme != HJ_WENO5)
        return fail(ctx, HJ_EINVAL, "unknown scheme %d", m->scheme);
    if (m->brt < HJ_BRT_NONE || m->brt > HJ_BRT_MINV) return fail(ctx, HJ_EINVAL, "unknown brt mode %d", m->brt);
    if (m->extrap != HJ_EXTRAP_AWAY_FROM_ZERO && m->extrap != HJ_EXTRAP_LINEAR)
        return fail(ctx, HJ_EINVAL, "unknown extrapolation %d", m->extrap);
    for (int k = 0; k < 8; ++k)
        if (!std::isfinite(m->params[k])) return fail(ctx, HJ_EINVAL, "params[%d] is not finite", k);
    if (m->order < 0 || m->order > 3) return fail(ctx, HJ_EINVAL, "order %d not in 1..3 (0 = 3)", m->order);
    if (m->alpha_mode != HJ_ALPHA_NODE && m->alpha_mode != HJ_ALPHA_GLOBAL && m->alpha_mode != HJ_ALPHA_BOX)
        return fail(ctx, HJ_EINVAL, "unknown alpha_mode %d", m->alpha_mode);
    if (m->kernel != HJ_KERNEL_AUTO && m->kernel != HJ_KERNEL_ROWS && m->kernel != HJ_KERNEL_NODE)
        return fail(ctx, HJ_EINVAL, "unknown kernel %d", m->kernel);
    const int32_t* to = m->tile_override;
    if (to[0] < 0 || to[1] < 0 || to[2] < 0 || to[2] > 2 || to[3] < 0 || to[3] > 3)
        return fail(ctx, HJ_EINVAL, "tile_override {%d, %d, %d, %d} malformed", to[0], to[1], to[2], to[3]);
    if (to[0] == 0 && (to[1] || to[2] || to[3]))
        return fail(ctx, HJ_EINVAL, "tile_override needs ty >= 1 (all zero: tuned)");
    if (to[0] > 0 && m->kernel == HJ_KERNEL_NODE)
        return fail(ctx, HJ_EINVAL, "tile_override applies to the row kernel, not to kernel = HJ_KERNEL_NODE");
    const int D = g->ndim;
    const double* q = m->params;
    switch (m->dynamics) {
    case HJ_DYN_DOUBLE_INTEGRATOR:
        if (D != 2) return fail(ctx, HJ_EINVAL, "double integrator needs ndim 2");
        if (q[0] < 0) return fail(ctx, HJ_EINVAL, "umax < 0");
        break;
    case HJ_DYN_AIR3D:
        if (D != 3) return fail(ctx, HJ_EINVAL, "air3D needs ndim 3");
        if (q[2] < 0 || q[3] < 0) return fail(ctx, HJ_EINVAL, "control bounds < 0");
        break;
    case HJ_DYN_DUBINS4D:
        if (D != 4) return fail(ctx, HJ_EINVAL, "Dubins4D needs ndim 4");
        if (q[0] < 0 || q[1] < 0) return fail(ctx, HJ_EINVAL, "control bounds < 0");
        break;
    case HJ_DYN_NORM:
        if (D > 3) return fail(ctx, HJ_EINVAL, "norm Hamiltonian supports ndim 1..3");
        if (q[0] < 0) return fail(ctx, HJ_EINVAL, "speed < 0");
        break;
    case HJ_DYN_ADVECT:
        if (D > 3) return fail(ctx, HJ_EINVAL, "advection supports ndim 1..3");
        break;
    case HJ_DYN_ROTATE:
        if (D < 2 || D > 3) return fail(ctx, HJ_EINVAL, "rotation supports ndim 2..3");
        break;
    case HJ_DYN_ROCKETS:
        if (D != 3) return fail(ctx, HJ_EINVAL, "rockets needs ndim 3");
        if (q[2] < 0 || q[3] < 0) return fail(ctx, HJ_EINVAL, "control bounds < 0");
        break;
    default:
        return fail(ctx, HJ_EINVAL, "unknown dynamics %d", m->dynamics);
    }
    return HJ_OK;
}

hj_status check_solver_settings(hj_ctx* ctx, const hj_method* m) {
    if (!(m->cfl > 0.0) || !(m->cfl <= 1.0)) return fail(ctx, HJ_EINVAL, "cfl must be in (0, 1]");
    if (!(m->max_step > 0.0)) return fail(ctx, HJ_EINVAL, "max_step must be > 0");
    return HJ_OK;
}

GridDev make_grid(const hj_grid* g, int extrap) {
    GridDev G;
    std::memset(&G, 0, sizeof G);
    G.ndim = g->ndim;
    long long stride = 1;
    for (int d = 0; d < 4; ++d) {
        if (d < g->ndim) {
            const bool periodic = (g->periodic_mask >> d) & 1u;
            G.n[d] = (int)g->n[d];
            G.stride[d] = stride;
            stride *= g->n[d];
            G.lo[d] = g->lo[d];
            G.dx[d] = (g->hi[d] - g->lo[d]) / (periodic ? (double)g->n[d] : (double)(g->n[d] - 1));
            G.inv_dx[d] = 1.0 / G.dx[d];
        } else {
            G.n[d] = 1;
            G.stride[d] = stride;
            G.dx[d] = 1.0;
            G.inv_dx[d] = 1.0;
        }
    }
    G.total = stride;
    G.periodic_mask = g->periodic_mask;
    G.extrap = extrap;
    return G;
}

// WENO5 epsilon floor in raw-difference units along dimension d: FP64 uses
// 1e-99 on divided differences (Sec. 3.3, Jiang-Peng), so 1e-99 dx_d^2 on raw
// ones; FP32 uses 1e-18 directly so that the squared sums stay normal numbers.
double weno_floor(const GridDev& g, int dtype, int d) {
    if (dtype == HJ_F32) return (double)kWenoFloorF32;
    return 1e-99 * g.dx[d] * g.dx[d];
}

bool default_launch(const hj_method* m) {
    return m->kernel == HJ_KERNEL_AUTO && m->tile_override[0] == 0;
}

hj_status ensure(hj_ctx* ctx, void** p, size_t* cap, size_t bytes) {
    if (*cap >= bytes && *p) return HJ_OK;
    if (*p) {
        HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(ctx, e, "cudaMalloc");
    }
    *cap = bytes;
    return HJ_OK;
}

hj_status ensure_work(hj_ctx* ctx, size_t bytes) {
    if (ctx->work_bytes >= bytes && ctx->work[0]) return HJ_OK;
    if (ctx->work[0]) {
        HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->work[0]);
        cudaFree(ctx->work[1]);
        ctx->work[0] = ctx->work[1] = nullptr;
        ctx->work_bytes = 0;
    }
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMalloc(&ctx->work[k], bytes);
        if (e != cudaSuccess) {
            cudaFree(ctx->work[0]);
            ctx->work[0] = ctx->work[1] = nullptr;
            return cuda_fail(ctx, e, "cudaMalloc(stage buffers)");
        }
    }
    ctx->work_bytes = bytes;
    return HJ_OK;
}

// cos/sin of the dimension-2 coordinate (the heading angle of air3D and
// Dubins4D), from the host math library, in both precisions.
void angle_table(const hj_grid* g, std::vector<double>* out) {
    const int n = (int)g->n[2];
    const bool periodic = (g->periodic_mask >> 2) & 1u;
    const double dx = (g->hi[2] - g->lo[2]) / (periodic ? (double)n : (double)(n - 1));
    out->assign(2 * (size_t)n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double x = g->lo[2] + (double)i * dx;
        (*out)[i] = std::cos(x);
        (*out)[n + i] = std::sin(x);
    }
}

hj_status check_slices(hj_ctx* ctx, int n_slices, const double* slice_times, double t0) {
    if (n_slices < 1 || !slice_times) return fail(ctx, HJ_EINVAL, "need at least one slice time");
    if (!(t0 >= 0.0) || !std::isfinite(t0)) return fail(ctx, HJ_EINVAL, "t0 must be finite and >= 0");
    for (int s = 0; s < n_slices; ++s) {
        const double ts = slice_times[s];
        if (!(ts >= t0) || !std::isfinite(ts)) return fail(ctx, HJ_EINVAL, "slice time %d invalid (before t0?)", s);
        if (s > 0 && ts < slice_times[s - 1]) return fail(ctx, HJ_EINVAL, "slice times must not decrease");
    }
    return HJ_OK;
}

// Listing 6: dt = min(t_f - t, maxStep, cfl * stepBound), stepBound = 1/stepBoundInv,
// while t_f - t >= eps t_f; alpha depends on x only, so stepBound is the same at
// every step and the whole schedule is known before the first step.
void plan_schedule(const hj_method* m, double sbi, int n_slices, const double* slice_times, double t0,
                   Schedule* S) {
    S->dts.clear();
    S->slice_steps.assign(n_slices, 0);
    S->slice_t.assign(n_slices, t0);
    const double step_bound_v = 1.0 / sbi;
    const double eps = 100.0 * DBL_EPSILON;
    double t = t0;
    for (int s = 0; s < n_slices; ++s) {
        const double ts = slice_times[s];
        while (ts > t && ts - t >= eps * ts) {
            double dt = ts - t;
            if (m->max_step < dt) dt = m->max_step;
            if (m->cfl * step_bound_v < dt) dt = m->cfl * step_bound_v;
            S->dts.push_back(dt);
            t += dt;
        }
        S->slice_steps[s] = (long long)S->dts.size();
        S->slice_t[s] = t;
    }
}

hj_status upload_trig(hj_ctx* ctx, const hj_grid* g, int dynamics) {
    if (dynamics != HJ_DYN_AIR3D && dynamics != HJ_DYN_DUBINS4D && dynamics != HJ_DYN_ROCKETS) return HJ_OK;
    const int n = (int)g->n[2];
    const bool periodic = (g->periodic_mask >> 2) & 1u;
    const double dx = (g->hi[2] - g->lo[2]) / (periodic ? (double)n : (double)(n - 1));
    if (ctx->trig_valid && ctx->trig_key[0] == (double)n && ctx->trig_key[1] == g->lo[2] && ctx->trig_key[2] == dx)
        return HJ_OK;  // the tables on the device already hold these angles
    std::vector<double> hd;
    angle_table(g, &hd);
    std::vector<float> hf(hd.begin(), hd.end());
    const size_t need = 2 * (size_t)n;
    if (ctx->trig_cap < need) {
        HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->trig_d);
        cudaFree(ctx->trig_f);
        ctx->trig_d = nullptr;
        ctx->trig_f = nullptr;
        ctx->trig_cap = 0;
        HJ_CUDA(ctx, cudaMalloc(&ctx->trig_d, need * sizeof(double)));
        HJ_CUDA(ctx, cudaMalloc(&ctx->trig_f, need * sizeof(float)));
        ctx->trig_cap = need;
    }
    // copies ordered after earlier kernels on the stream; waited for because the host vectors die at return
    ctx->trig_valid = false;
    HJ_CUDA(ctx, cudaMemcpyAsync(ctx->trig_d, hd.data(), need * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    HJ_CUDA(ctx, cudaMemcpyAsync(ctx->trig_f, hf.data(), need * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->trig_key[0] = (double)n;
    ctx->trig_key[1] = g->lo[2];
    ctx->trig_key[2] = dx;
    ctx->trig_valid = true;
    return HJ_OK;
}

StageParams stage_params(hj_ctx* ctx, const GridDev& G, const hj_method* m, int dtype) {
    StageParams P;
    std::memset(&P, 0, sizeof P);
    P.g = G;
    P.dynamics = m->dynamics;
    for (int k = 0; k < 8; ++k) P.params[k] = m->params[k];
    P.brt_min0 = (m->brt == HJ_BRT_MIN0);
    P.trig_d = ctx->trig_d;
    P.trig_f = ctx->trig_f;
    for (int d = 0; d < kMaxDim; ++d) P.weno_floor[d] = weno_floor(G, dtype, d);
    P.alpha_box = (m->alpha_mode == HJ_ALPHA_BOX);
    return P;
}

// ---------------------------------------------------------------------------
// Row-tiled stage kernel: eligibility, launch-shape tuning, dispatch
// ---------------------------------------------------------------------------


bool rows_eligible(const GridDev& G, int scheme, int dynamics, int dtype, int kernel) {
    if ((scheme != HJ_WENO5 && scheme != HJ_ENO1 && scheme != HJ_ENO2 && scheme != HJ_ENO3) ||
        !rows_supported(G.ndim, dynamics) || kernel == HJ_KERNEL_NODE)
        return false;
    for (int d = 0; d < G.ndim; ++d)
        if (G.n[d] < 4) return false;
    if (G.n[0] + 1 > rows_max_threads(dtype == HJ_F64)) return false;
    if (G.ndim == 4 && G.n[2] > 65535) return false;
    if (G.total >= (1LL << 31)) return false;  // the row kernel indexes with 32-bit integers
    return true;
}

RowsCfg make_rows_cfg(const GridDev& G, int ty, int tz, int dtype) {
    RowsCfg c;
    c.ty = ty;
    c.nt = rows_block_threads(G.n[0], ty, rows_max_threads(dtype == HJ_F64));
    c.occ = 1;
    c.split = 0;
    c.row_tiles = (G.n[1] + ty - 1) / ty;
    const int ns = G.ndim >= 3 ? G.n[G.ndim - 1] : 1;
    c.tz = G.ndim >= 3 ? tz : 1;
    c.nchunks = G.ndim >= 3 ? (ns + c.tz - 1) / c.tz : 1;
    return c;
}

int rows_bps(const StageParams& P, const RowsCfg& c, int dtype) {
    return dtype == HJ_F64 ? rows_blocks_per_sm_f64(P, c) : rows_blocks_per_sm_f32(P, c);
}

cudaError_t rows_launch(hj_ctx* ctx, const StageParams& P0, const RowsCfg& c, int dtype) {
    ctx->launches += 1;
    const StageParams P = finalize(P0);
    return dtype == HJ_F64 ? launch_rows_f64(P, c, ctx->stream) : launch_rows_f32(P, c, ctx->stream);
}

// Candidate shapes ranked by a simple cost model: whole waves of resident
// blocks times the work of a block (warps x planes, plus one plane of
// prologue per chunk and the halo rows per plane). The sixteen best blocks
// with row-end threads and the eight best of n0*ty threads (the last node row
// taking the row ends) are timed.
std::vector<RowsCfg> rows_candidates(hj_ctx* ctx, const StageParams& P, int dtype) {
    const GridDev& G = P.g;
    const int nx = G.n[0], ny = G.n[1];
    const int D = G.ndim;
    const int ns = D >= 3 ? G.n[D - 1] : 1;
    const size_t es = dtype == HJ_F64 ? 8 : 4;
    static const int tys[] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 24, 32};
    static const int tzs[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 128, 256};
    std::vector<std::pair<double, RowsCfg>> scored, scored_merged;
    for (int ty : tys) {
        if (ty > ny || ty > nx || nx * ty > rows_max_threads(dtype == HJ_F64)) continue;
        if (rows_smem(nx, ty, es) > 200 * 1024) continue;
        std::vector<int> zs;
        if (D >= 3) {
            for (int tz : tzs)
                if (tz < ns) zs.push_back(tz);
            zs.push_back(ns);
        } else {
            zs.push_back(1);
        }
        for (int k = 0; k < 4 * (int)zs.size(); ++k) {
            const int tz = zs[k / 4];
            const bool merged = (k % 4) >= 2;  // a block of n0*ty threads: the last node row takes the row ends
            if (!merged && (nx + 1) * ty > rows_max_threads(dtype == HJ_F64)) continue;
            RowsCfg c = make_rows_cfg(G, ty, tz, dtype);
            if (merged) c.nt = nx * ty;
            if (k % 2 == 1) {  // the FP32 variant for two blocks per SM
                if (dtype == HJ_F64 || c.nt > kRowsOcc2Threads) continue;
                c.occ = 2;
            }
            if (c.nchunks > 65535 || c.row_tiles > (1 << 30)) continue;
            const int bps = rows_bps(P, c, dtype);
            if (bps <= 0) continue;
            const double blocks = (double)c.row_tiles * c.nchunks * (D == 4 ? G.n[2] : 1);
            const double slots = (double)ctx->sm_count * bps;
            const double waves = std::ceil(blocks / slots);
            const double warps = std::ceil((double)c.nt / 32.0);
            const double rows_valid = std::min(ty, ny);
            const double plane = warps * (1.0 + 0.1 * (6.0 + ty - rows_valid) / ty);
            const double planes = D >= 3 ? (double)std::min(tz, ns) + 1.0 : 1.0;
            (merged ? scored_merged : scored).push_back({waves * std::min((double)bps, blocks) * plane * planes, c});
        }
    }
    const auto by_cost = [](const std::pair<double, RowsCfg>& a, const std::pair<double, RowsCfg>& b) {
        return a.first < b.first;
    };
    std::sort(scored.begin(), scored.end(), by_cost);
    std::sort(scored_merged.begin(), scored_merged.end(), by_cost);
    std::vector<RowsCfg> out;
    for (size_t k = 0; k < scored.size() && k < 16; ++k) out.push_back(scored[k].second);
    for (size_t k = 0; k < scored_merged.size() && k < 8; ++k) out.push_back(scored_merged[k].second);
    return out;
}

// The launch shape for this grid: measured once per (shape, dtype, dynamics,
// scheme, dissipation) over the model's best candidates (groups of
// first-stage launches writing to a scratch buffer, best of two groups), then
// cached in the context. A tile override {ty, tz, occ, merged} (ty >= 1)
// pins the shape instead; it is validated once and cached like a tuned one.
hj_status rows_config(hj_ctx* ctx, const StageParams& P, int dtype, const int32_t* tile, RowsCfg* out) {
    const GridDev& G = P.g;
    std::vector<long long> key = {G.ndim, P.dynamics, P.scheme, dtype, G.n[0], G.n[1], G.n[2], G.n[3],
                                  rows_box_variant(P) ? 1 : 0};
    if (tile && tile[0] > 0) {
        std::vector<long long> pkey = key;
        for (int k = 0; k < 4; ++k) pkey.push_back(-1 - (long long)tile[k]);
        auto hit = ctx->rows_cache.find(pkey);
        if (hit != ctx->rows_cache.end()) {
            *out = hit->second;
            return HJ_OK;
        }
        const int ty = tile[0], tz = tile[1] > 0 ? tile[1] : 1, occ = tile[2] > 0 ? tile[2] : 1;
        const int merged = tile[3] & 1, split = (tile[3] & 2) ? 0 : 1;
        if (ty <= G.n[1] && ty <= G.n[0] && (G.n[0] + 1 - merged) * ty <= rows_max_threads(dtype == HJ_F64)) {
            *out = make_rows_cfg(G, ty, tz, dtype);
            if (merged) out->nt = G.n[0] * ty;
            out->occ = occ;
            out->split = split;
            if (occ == 2 && (dtype == HJ_F64 || out->nt > kRowsOcc2Threads)) out->occ = 0;
            if (out->occ && out->nchunks <= 65535 && rows_bps(P, *out, dtype) > 0) {
                ctx->rows_cache[pkey] = *out;
                return HJ_OK;
            }
        }
        return fail(ctx, HJ_EINVAL, "tile_override {%d, %d, %d, %d} does not fit this grid", tile[0], tile[1],
                    tile[2], tile[3]);
    }
    auto it = ctx->rows_cache.find(key);
    if (it != ctx->rows_cache.end()) {
        *out = it->second;
        return HJ_OK;
    }
    std::vector<RowsCfg> cands = rows_candidates(ctx, P, dtype);
    if (cands.empty()) return fail(ctx, HJ_EINVAL, "no launch shape fits the row kernel");
    RowsCfg best = cands[0];
    if (cands.size() > 1) {
        const size_t bytes = (size_t)G.total * (dtype == HJ_F64 ? 8 : 4);
        hj_status st = ensure(ctx, &ctx->tune_buf, &ctx->tune_bytes, bytes);
        if (st) return st;
        // timed as a first RK stage (reads u, writes the scratch buffer)
        StageParams T = P;
        T.mode = kStage;
        T.vn = nullptr;
        T.cv = 0.0;
        T.cu = 1.0;
        T.minv_after = 0;
        T.out = ctx->tune_buf;
        cudaEvent_t e0, e1;
        HJ_CUDA(ctx, cudaEventCreate(&e0));
        HJ_CUDA(ctx, cudaEventCreate(&e1));
        // FP32 launches of a few tens of microseconds are timed in groups: the
        // event clock advances in steps of about two microseconds.
        const int group = dtype == HJ_F64 ? 1 : (G.total < (4LL << 20) ? 6 : 2);
        float best_ms = 1e30f;
        for (const RowsCfg& c : cands) {
            cudaError_t e = rows_launch(ctx, T, c, dtype);  // warm-up
            float ms_min = 1e30f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, ctx->stream);
                for (int k = 0; k < group && e == cudaSuccess; ++k) e = rows_launch(ctx, T, c, dtype);
                cudaEventRecord(e1, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                ms_min = std::min(ms_min, ms);
            }
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(ctx, e, "tuning launch");
            }
            if (ms_min < best_ms) {
                best_ms = ms_min;
                best = c;
            }
        }
        // the ENO schemes: the best shape once more with interior tiles on
        // their own body (the WENO5 kernels have no second body)
        cudaError_t e = cudaSuccess;
        if (P.scheme != HJ_WENO5) {
            RowsCfg c = best;
            c.split = 1;
            e = rows_launch(ctx, T, c, dtype);
            float ms_min = 1e30f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, ctx->stream);
                for (int k = 0; k < group && e == cudaSuccess; ++k) e = rows_launch(ctx, T, c, dtype);
                cudaEventRecord(e1, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                ms_min = std::min(ms_min, ms);
            }
            if (e == cudaSuccess && ms_min < best_ms) best = c;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tuning launch");
    }
    ctx->rows_cache[key] = best;
    *out = best;
    return HJ_OK;
}

// Which kernel runs a method's stages, and the row kernel's pinned shape
// (hj_method.kernel and tile_override).
struct KernelPick {
    int kernel = HJ_KERNEL_AUTO;
    int32_t tile[4] = {0, 0, 0, 0};
};
KernelPick pick_of(const hj_method* m) {
    KernelPick k;
    k.kernel = m->kernel;
    for (int i = 0; i < 4; ++i) k.tile[i] = m->tile_override[i];
    return k;
}

// Refuses a kernel choice the grid cannot take (before anything is enqueued).
hj_status check_pick(hj_ctx* ctx, const GridDev& G, const hj_method* m, int dtype) {
    const bool rows = rows_eligible(G, m->scheme, m->dynamics, dtype, m->kernel);
    if (m->kernel == HJ_KERNEL_ROWS && !rows)
        return fail(ctx, HJ_EINVAL, "kernel = HJ_KERNEL_ROWS: the row kernel cannot take this grid");
    if (m->tile_override[0] > 0 && !rows)
        return fail(ctx, HJ_EINVAL, "tile_override: the row kernel cannot take this grid");
    return HJ_OK;
}

// Launches one stage; HJ_EINVAL (with the context's message set) if a pinned
// shape does not fit.
hj_status launch_stage(hj_ctx* ctx, const StageParams& P, int scheme, int dtype, const KernelPick& k) {
    if (rows_eligible(P.g, scheme, P.dynamics, dtype, k.kernel)) {
        StageParams Q = P;
        Q.scheme = scheme;
        RowsCfg c;
        hj_status st = rows_config(ctx, Q, dtype, k.tile, &c);
        if (st) return st;
        cudaError_t e = rows_launch(ctx, Q, c, dtype);
        return e == cudaSuccess ? HJ_OK : cuda_fail(ctx, e, "stage launch");
    }
    ctx->launches += 1;
    const StageParams Q = finalize(P);
    cudaError_t e = dtype == HJ_F64 ? launch_stage_f64(Q, scheme, ctx->stream)
                                    : launch_stage_f32(Q, scheme, ctx->stream);
    return e == cudaSuccess ? HJ_OK : cuda_fail(ctx, e, "stage launch");
}

// Three fused stage launches of one TVD-RK3 step (Listing 6):
//   V1 = V + dt L(V);  V2 = 3/4 V + 1/4 (V1 + dt L(V1));  V <- 1/3 V + 2/3 (V2 + dt L(V2))
// with V <- min(V_new, V_old) in the last stage for the BRT min-V rule.
hj_status rk3_launch(hj_ctx* ctx, StageParams P, int scheme, int dtype, int brt, void* v, double dt,
                     const KernelPick& k);

// One TVD-RK step of order 1, 2 or 3 (0 = 3), in place on v:
//   1: v <- v + dt L(v)                              (one launch, then a copy)
//   2: V1 = v + dt L(v);  v <- 1/2 v + 1/2 (V1 + dt L(V1))
//   3: rk3_launch
// with v <- min(v_new, v_old) for the BRT min-V rule.
hj_status rk_launch(hj_ctx* ctx, const StageParams& P0, int scheme, int dtype, int brt, int order, void* v,
                    double dt, size_t bytes, const KernelPick& k) {
    if (order == 0 || order == 3) return rk3_launch(ctx, P0, scheme, dtype, brt, v, dt, k);
    StageParams P = P0;
    P.mode = kStage;
    P.dt = dt;
    hj_status st;
    if (order == 1) {
        P.u = v; P.out = ctx->work[0]; P.cv = 0.0; P.cu = 1.0;
        P.minv_after = (brt == HJ_BRT_MINV);
        P.vn = P.minv_after ? v : nullptr;
        if ((st = launch_stage(ctx, P, scheme, dtype, k))) return st;
        HJ_CUDA(ctx, cudaMemcpyAsync(v, ctx->work[0], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return HJ_OK;
    }
    P.u = v; P.vn = nullptr; P.out = ctx->work[0]; P.cv = 0.0; P.cu = 1.0; P.minv_after = 0;
    if ((st = launch_stage(ctx, P, scheme, dtype, k))) return st;
    P.u = ctx->work[0]; P.vn = v; P.out = v; P.cv = 0.5; P.cu = 0.5;
    P.minv_after = (brt == HJ_BRT_MINV);
    return launch_stage(ctx, P, scheme, dtype, k);
}

hj_status rk3_launch(hj_ctx* ctx, StageParams P, int scheme, int dtype, int brt, void* v, double dt,
                     const KernelPick& k) {
    P.mode = kStage;
    P.dt = dt;
    hj_status st;
    P.u = v; P.vn = nullptr; P.out = ctx->work[0]; P.cv = 0.0; P.cu = 1.0; P.minv_after = 0;
    if ((st = launch_stage(ctx, P, scheme, dtype, k))) return st;
    P.u = ctx->work[0]; P.vn = v; P.out = ctx->work[1]; P.cv = 0.75; P.cu = 0.25;
    if ((st = launch_stage(ctx, P, scheme, dtype, k))) return st;
    P.u = ctx->work[1]; P.vn = v; P.out = v; P.cv = 1.0 / 3.0; P.cu = 2.0 / 3.0;
    P.minv_after = (brt == HJ_BRT_MINV);
    return launch_stage(ctx, P, scheme, dtype, k);
}

// alpha_max[d] = max over the grid of alpha_d(x) (global Lax-Friedrichs).
// Synchronises the stream.
hj_status alpha_max(hj_ctx* ctx, const hj_grid* g, const hj_method* m, double* amax) {
    hj_status st = upload_trig(ctx, g, m->dynamics);
    if (st) return st;
    const GridDev G = make_grid(g, m->extrap);
    unsigned long long* acc = ctx->aux + 2;
    HJ_CUDA(ctx, cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long), ctx->stream));
    cudaError_t e = launch_step_bound(G, m->dynamics, m->params, ctx->trig_d, acc, 1, ctx->stream);
    ctx->launches += 1;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "alpha maximum launch");
    unsigned long long bits[4] = {0, 0, 0, 0};
    HJ_CUDA(ctx, cudaMemcpyAsync(bits, acc, sizeof bits, cudaMemcpyDeviceToHost, ctx->stream));
    HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int d = 0; d < 4; ++d) std::memcpy(&amax[d], &bits[d], sizeof(double));
    for (int d = G.ndim; d < 4; ++d) amax[d] = 0.0;
    return HJ_OK;
}

// CFL bound: max over nodes of sum_d alpha_d(x)/dx_d, or with global
// dissipation sum_d max_x alpha_d / dx_d (left to right, as the oracle).
hj_status step_bound(hj_ctx* ctx, const hj_grid* g, const hj_method* m, double* out) {
    if (m->alpha_mode == HJ_ALPHA_GLOBAL) {
        double amax[4];
        hj_status st = alpha_max(ctx, g, m, amax);
        if (st) return st;
        const GridDev G = make_grid(g, m->extrap);
        double s = 0.0;
        for (int d = 0; d < G.ndim; ++d) s += amax[d] / G.dx[d];
        *out = s;
        return HJ_OK;
    }
    hj_status st = upload_trig(ctx, g, m->dynamics);
    if (st) return st;
    const GridDev G = make_grid(g, m->extrap);
    HJ_CUDA(ctx, cudaMemsetAsync(ctx->aux, 0, sizeof(unsigned long long), ctx->stream));
    cudaError_t e = launch_step_bound(G, m->dynamics, m->params, ctx->trig_d, ctx->aux, 0, ctx->stream);
    ctx->launches += 1;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step bound launch");
    unsigned long long bits = 0;
    HJ_CUDA(ctx, cudaMemcpyAsync(&bits, ctx->aux, sizeof bits, cudaMemcpyDeviceToHost, ctx->stream));
    HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double v;
    std::memcpy(&v, &bits, sizeof v);
    *out = v;
    return HJ_OK;
}

// The launch parameters of a method on a grid: with global dissipation, the
// grid maxima of alpha (one reduction).
hj_status method_params(hj_ctx* ctx, const hj_grid* g, const GridDev& G, const hj_method* m, int dtype,
                        StageParams* P) {
    *P = stage_params(ctx, G, m, dtype);
    if (m->alpha_mode == HJ_ALPHA_GLOBAL) {
        hj_status st = alpha_max(ctx, g, m, P->alpha_g);
        if (st) return st;
        P->alpha_global = 1;
    }
    return HJ_OK;
}

hj_status nonfinite(hj_ctx* ctx, const void* v, long long n, int dtype, bool* bad) {
    int* flag = reinterpret_cast<int*>(ctx->aux + 1);
    HJ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    cudaError_t e = dtype == HJ_F64 ? launch_nonfinite_f64(static_cast<const double*>(v), n, flag, ctx->stream)
                                    : launch_nonfinite_f32(static_cast<const float*>(v), n, flag, ctx->stream);
    ctx->launches += 1;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "non-finite check launch");
    int h = 0;
    HJ_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *bad = h != 0;
    return HJ_OK;
}


}  // namespace hj

using namespace hj;

extern "C" {

const char* hj_version(void) { return "hj-gb300 0.1 sm_103a"; }

const char* hj_status_str(hj_status s) {
    switch (s) {
    case HJ_OK: return "ok";
    case HJ_EINVAL: return "invalid argument";
    case HJ_ENOMEM: return "out of memory";
    case HJ_ECUDA: return "CUDA error";
    case HJ_ENONFINITE: return "non-finite value";
    case HJ_ETIMEOUT: return "timed out";
    case HJ_ECANCELLED: return "cancelled";
    case HJ_EBUSY: return "busy";
    default: return "unknown status";
    }
}

const char* hj_ctx_last_error(const hj_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "context is NULL"; }

hj_status hj_ctx_create(int32_t device, void* cuda_stream, hj_ctx** out) {
    if (!out) return HJ_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) return HJ_ECUDA;
    if (device < 0 || device >= count) return HJ_EINVAL;
    hj_ctx* ctx = new (std::nothrow) hj_ctx();
    if (!ctx) return HJ_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    DeviceGuard guard(device);
    if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete ctx;
        return HJ_ECUDA;
    }
    if (cudaMalloc(&ctx->aux, 256) != cudaSuccess) {
        (void)cudaGetLastError();  // not sticky: leave no recorded error behind
        delete ctx;
        return HJ_ENOMEM;
    }
    *out = ctx;
    return HJ_OK;
}

void hj_ctx_destroy(hj_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->work[0]);
    cudaFree(ctx->work[1]);
    cudaFree(ctx->state);
    cudaFree(ctx->aux);
    cudaFree(ctx->trig_d);
    cudaFree(ctx->trig_f);
    cudaFree(ctx->tune_buf);
    delete ctx->batch_engine;
    delete ctx;
}

hj_status hj_upwind(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype, const void* v,
                    int32_t dim, void* pm, void* pp) {
    if (!ctx) return HJ_EINVAL;
    hj_status st = check_grid(ctx, grid);
    if (st) return st;
    if (!method) return fail(ctx, HJ_EINVAL, "method is NULL");
    if (!elem_size(dtype)) return fail(ctx, HJ_EINVAL, "unknown dtype %d", dtype);
    if (method->scheme != HJ_ENO1 && method->scheme != HJ_ENO2 && method->scheme != HJ_ENO3 &&
        method->scheme != HJ_WENO5)
        return fail(ctx, HJ_EINVAL, "unknown scheme %d", method->scheme);
    if (method->extrap != HJ_EXTRAP_AWAY_FROM_ZERO && method->extrap != HJ_EXTRAP_LINEAR)
        return fail(ctx, HJ_EINVAL, "unknown extrapolation %d", method->extrap);
    if (dim < 0 || dim >= grid->ndim) return fail(ctx, HJ_EINVAL, "dim %d out of range", dim);
    if (!v || !pm || !pp) return fail(ctx, HJ_EINVAL, "NULL array");
    DeviceGuard guard(ctx->device);
    UpwindParams P;
    std::memset(&P, 0, sizeof P);
    P.g = make_grid(grid, method->extrap);
    P.dim = dim;
    P.u = v;
    P.pm = pm;
    P.pp = pp;
    P.weno_floor = weno_floor(P.g, dtype, dim);
    ctx->launches += 1;
    cudaError_t e = dtype == HJ_F64 ? launch_upwind_f64(P, method->scheme, ctx->stream)
                                    : launch_upwind_f32(P, method->scheme, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upwind launch");
    return HJ_OK;
}

hj_status hj_term(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype, const void* v,
                  void* ydot) {
    if (!ctx) return HJ_EINVAL;
    hj_status st = check_grid(ctx, grid);
    if (st) return st;
    if ((st = check_method(ctx, grid, method))) return st;
    if (!elem_size(dtype)) return fail(ctx, HJ_EINVAL, "unknown dtype %d", dtype);
    if (!v || !ydot) return fail(ctx, HJ_EINVAL, "NULL array");
    DeviceGuard guard(ctx->device);
    if ((st = upload_trig(ctx, grid, method->dynamics))) return st;
    StageParams P;
    const GridDev G = make_grid(grid, method->extrap);
    if ((st = check_pick(ctx, G, method, dtype))) return st;
    if ((st = method_params(ctx, grid, G, method, dtype, &P))) return st;
    P.mode = kTerm;
    P.u = v;
    P.out = ydot;
    return launch_stage(ctx, P, method->scheme, dtype, pick_of(method));
}

hj_status hj_step_bound(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, double* out) {
    if (!ctx) return HJ_EINVAL;
    hj_status st = check_grid(ctx, grid);
    if (st) return st;
    if ((st = check_method(ctx, grid, method))) return st;
    if (!out) return fail(ctx, HJ_EINVAL, "out is NULL");
    DeviceGuard guard(ctx->device);
    return step_bound(ctx, grid, method, out);
}

hj_status hj_rk3_step(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype, void* v,
                      double dt) {
    hj::NvtxRange range("hj_rk3_step");
    if (!ctx) return HJ_EINVAL;
    hj_status st = check_grid(ctx, grid);
    if (st) return st;
    if ((st = check_method(ctx, grid, method))) return st;
    if (!elem_size(dtype)) return fail(ctx, HJ_EINVAL, "unknown dtype %d", dtype);
    if (!v) return fail(ctx, HJ_EINVAL, "NULL array");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(ctx, HJ_EINVAL, "dt must be finite and >= 0");
    DeviceGuard guard(ctx->device);
    const GridDev G = make_grid(grid, method->extrap);
    if ((st = check_pick(ctx, G, method, dtype))) return st;
    if ((st = ensure_work(ctx, (size_t)G.total * elem_size(dtype)))) return st;
    if ((st = upload_trig(ctx, grid, method->dynamics))) return st;
    StageParams P;
    if ((st = method_params(ctx, grid, G, method, dtype, &P))) return st;
    return rk_launch(ctx, P, method->scheme, dtype, method->brt, method->order, v, dt,
                     (size_t)G.total * elem_size(dtype), pick_of(method));
}

hj_status hj_rk3_stage(hj_ctx* ctx, const hj_grid* grid, const hj_method* method, int32_t dtype, int32_t stage,
                       const void* u, const void* vn, void* out, double dt) {
    if (!ctx) return HJ_EINVAL;
    hj_status st = check_grid(ctx, grid);
    if (st) return st;
    if ((st = check_method(ctx, grid, method))) return st;
    if (!elem_size(dtype)) return fail(ctx, HJ_EINVAL, "unknown dtype %d", dtype);
    if (stage < 1 || stage > 3) return fail(ctx, HJ_EINVAL, "stage %d not in 1..3", stage);
    if (!u || !out || (stage > 1 && !vn)) return fail(ctx, HJ_EINVAL, "NULL array");
    if (out == u) return fail(ctx, HJ_EINVAL, "out must not alias u");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(ctx, HJ_EINVAL, "dt must be finite and >= 0");
    DeviceGuard guard(ctx->device);
    if ((st = upload_trig(ctx, grid, method->dynamics))) return st;
    StageParams P;
    const GridDev G = make_grid(grid, method->extrap);
    if ((st = check_pick(ctx, G, method, dtype))) return st;
    if ((st = method_params(ctx, grid, G, method, dtype, &P))) return st;
    P.mode = kStage;
    P.dt = dt;
    P.u = u;
    P.vn = vn;
    P.out = out;
    P.cv = stage == 1 ? 0.0 : (stage == 2 ? 0.75 : 1.0 / 3.0);
    P.cu = stage == 1 ? 1.0 : (stage == 2 ? 0.25 : 2.0 / 3.0);
    P.minv_after = (stage == 3 && method->brt == HJ_BRT_MINV);
    return launch_stage(ctx, P, method->scheme, dtype, pick_of(method));
}

hj_status hj_solve(hj_ctx* ctx, const hj_problem* pr, void* out_slices, int32_t out_on_device, double* out_times,
                   hj_stats* stats) {
    hj::NvtxRange range("hj_solve");
    if (!ctx) return HJ_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    if (!pr) return fail(ctx, HJ_EINVAL, "problem is NULL");
    hj_status st = check_grid(ctx, &pr->grid);
    if (st) return st;
    if ((st = check_method(ctx, &pr->grid, &pr->method))) return st;
    if ((st = check_solver_settings(ctx, &pr->method))) return st;
    const size_t es = elem_size(pr->dtype);
    if (!es) return fail(ctx, HJ_EINVAL, "unknown dtype %d", pr->dtype);
    if (!pr->v0 || !out_slices) return fail(ctx, HJ_EINVAL, "NULL v0 or output");
    if ((st = check_slices(ctx, pr->n_slices, pr->slice_times, pr->t0))) return st;
    DeviceGuard guard(ctx->device);
    const GridDev G = make_grid(&pr->grid, pr->method.extrap);
    if ((st = check_pick(ctx, G, &pr->method, pr->dtype))) return st;
    const size_t bytes = (size_t)G.total * es;
    const long long launches0 = ctx->launches;
    if ((st = ensure_work(ctx, bytes))) return st;
    if ((st = ensure(ctx, &ctx->state, &ctx->state_bytes, bytes))) return st;
    void* V = ctx->state;
    HJ_CUDA(ctx, cudaMemcpyAsync(V, pr->v0, bytes, pr->v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 ctx->stream));
    bool bad = false;
    if ((st = nonfinite(ctx, V, G.total, pr->dtype, &bad))) return st;
    if (bad) return fail(ctx, HJ_ENONFINITE, "v0 holds NaN or Inf");
    double sbi = 0.0;
    if ((st = step_bound(ctx, &pr->grid, &pr->method, &sbi))) return st;  // also uploads the angle tables
    StageParams P;
    if ((st = method_params(ctx, &pr->grid, G, &pr->method, pr->dtype, &P))) return st;
    Schedule S;
    plan_schedule(&pr->method, sbi, pr->n_slices, pr->slice_times, pr->t0, &S);
    const cudaMemcpyKind out_kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t k = 0;
    for (int s = 0; s < pr->n_slices; ++s) {
        for (; k < (size_t)S.slice_steps[s]; ++k)
            if ((st = rk_launch(ctx, P, pr->method.scheme, pr->dtype, pr->method.brt, pr->method.order, V, S.dts[k],
                                bytes, pick_of(&pr->method))))
                return st;
        HJ_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(out_slices) + (size_t)s * bytes, V, bytes, out_kind,
                                     ctx->stream));
        if (out_times) out_times[s] = S.slice_t[s];
    }
    const long long steps = (long long)S.dts.size();
    const double t = S.slice_t[pr->n_slices - 1];
    if ((st = nonfinite(ctx, V, G.total, pr->dtype, &bad))) return st;  // synchronises the stream
    if (bad) return fail(ctx, HJ_ENONFINITE, "the solution became non-finite");
    if (stats) {
        stats->steps = steps;
        stats->cell_updates = steps * G.total;
        stats->kernel_launches = ctx->launches - launches0;
        stats->step_bound_inv = sbi;
        stats->t_final = t;
        stats->elapsed_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats->queued_ms = 0.0;
    }
    return HJ_OK;
}

}  // extern "C"
