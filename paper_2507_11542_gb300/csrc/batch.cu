// batch.cu -- hj_solve_batch: many independent solves advanced together.
//
// Every eligible instance (WENO5, a dimension/dynamics pair of the row
// kernel) gets a device descriptor (grid, dynamics, its three arrays, its dt
// schedule and slice cursor). Instances are grouped by (element type,
// dimension, dynamics); one launch per group and RK stage covers all tiles of
// the group's active instances, and one small kernel per step advances every
// instance's step counter, dt and slice output. Blocks of K steps are
// captured once as a CUDA graph and replayed; the tile lists are rebuilt
// whenever finished instances leave a quarter of the tiles idle.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace hj {
namespace {

constexpr size_t kAlign = 256;
constexpr int kGraphSteps = 16;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Inst {
    int idx = 0;               // problem index
    GridDev G;
    int dtype = 0;
    size_t es = 0;
    long long N = 0;
    bool angles = false;
    int group = -1;
    Schedule S;
    double sbi = 0.0;
    std::vector<long long> ends;
    std::vector<int> end_slice;
    // arena 1 offsets
    size_t off_v = 0, off_v1 = 0, off_v2 = 0, off_td = 0, off_tf = 0, off_stage = 0;
    // arena 2 offsets
    size_t off_dts = 0, off_ends = 0, off_end_slice = 0;
    int ty = 1, tz = 1;
};

struct Group {
    int dtype, ndim, dyn;
    std::vector<int> members;  // indices into the instance list
    int threads = 0;
    int tz_target = 8;
    size_t smem = 0;
    std::vector<BatchTile> tiles;
    size_t off_tiles = 0;      // arena 2 offset of this group's tile list
    size_t tile_cap = 0;       // capacity in tiles
};

int max_block_threads(int dtype) { return dtype == HJ_F64 ? 512 : 1024; }

void shape_for(const Inst& in, int threads, int tz_target, int* ty, int* tz) {
    const int nx = in.G.n[0], ny = in.G.n[1];
    int t = std::max(1, threads / (nx + 1));
    t = std::min(t, ny);
    while (t > 1 && rows_smem(nx, t, in.es) > 200 * 1024) --t;
    *ty = t;
    const int D = in.G.ndim;
    *tz = D >= 3 ? std::max(1, std::min(tz_target, in.G.n[D - 1])) : 1;
}

void build_tiles(const std::vector<Inst>& insts, Group& g, long long gstep, std::vector<int>* order_out) {
    g.tiles.clear();
    std::vector<int> order;
    for (int m : g.members)
        if ((long long)insts[m].S.dts.size() > gstep) order.push_back(m);
    // largest instances first: their many tiles start early, small ones fill the tail
    std::sort(order.begin(), order.end(), [&](int a, int b) { return insts[a].N > insts[b].N; });
    for (int m : order) {
        const Inst& in = insts[m];
        const int D = in.G.ndim;
        const int rt = (in.G.n[1] + in.ty - 1) / in.ty;
        const int ns = D >= 3 ? in.G.n[D - 1] : 1;
        const int nch = D >= 3 ? (ns + in.tz - 1) / in.tz : 1;
        const int n2 = D == 4 ? in.G.n[2] : 1;
        for (int c = 0; c < nch; ++c)
            for (int j = 0; j < n2; ++j)
                for (int t = 0; t < rt; ++t) g.tiles.push_back(BatchTile{m, t, j, c});
    }
    if (order_out) *order_out = order;
}

cudaError_t launch_group_stage(hj_ctx* ctx, const Group& g, const BatchInst* d_insts, unsigned char* arena2, int stage,
                               cudaStream_t s, bool count = true) {
    if (g.tiles.empty()) return cudaSuccess;
    const BatchTile* tiles = reinterpret_cast<const BatchTile*>(arena2 + g.off_tiles);
    if (count) ctx->launches += 1;
    return g.dtype == HJ_F64 ? launch_batch_stage_f64(tiles, (int)g.tiles.size(), d_insts, stage, g.ndim, g.dyn,
                                                      g.threads, g.smem, s)
                             : launch_batch_stage_f32(tiles, (int)g.tiles.size(), d_insts, stage, g.ndim, g.dyn,
                                                      g.threads, g.smem, s);
}

// One RK3 step of every active instance: each group's three stages, then the advance kernel.
// (count = false while capturing: a captured launch runs at each replay instead)
cudaError_t enqueue_step(hj_ctx* ctx, const std::vector<Group>& groups, BatchInst* d_insts, int n_insts,
                         unsigned char* arena2, cudaStream_t s, bool count) {
    for (int stage = 1; stage <= 3; ++stage)
        for (const Group& g : groups) {
            cudaError_t e = launch_group_stage(ctx, g, d_insts, arena2, stage, s, count);
            if (e != cudaSuccess) return e;
        }
    if (count) ctx->launches += 1;
    return launch_batch_advance(d_insts, n_insts, s);
}

long long launches_per_step(const std::vector<Group>& groups) {
    long long k = 1;
    for (const Group& g : groups)
        if (!g.tiles.empty()) k += 3;
    return k;
}

}  // namespace
}  // namespace hj

using namespace hj;

extern "C" hj_status hj_solve_batch(hj_ctx* ctx, int32_t n, const hj_problem* problems, void* const* out_slices,
                                    const int32_t* out_on_device, double* const* out_times, hj_stats* stats) {
    if (!ctx) return HJ_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    if (n < 0 || (n > 0 && (!problems || !out_slices || !out_on_device)))
        return fail(ctx, HJ_EINVAL, "batch needs problems, outputs and output placement flags");
    if (n == 0) return HJ_OK;
    // ---- validate everything before any work
    for (int i = 0; i < n; ++i) {
        const hj_problem* pr = &problems[i];
        hj_status st;
        if ((st = check_grid(ctx, &pr->grid)) || (st = check_method(ctx, &pr->grid, &pr->method)) ||
            (st = check_solver_settings(ctx, &pr->method)) || (st = check_slices(ctx, pr->n_slices, pr->slice_times))) {
            const std::string msg = ctx->last_error;
            return fail(ctx, st, "problem %d: %s", i, msg.c_str());
        }
        if (!elem_size(pr->dtype)) return fail(ctx, HJ_EINVAL, "problem %d: unknown dtype", i);
        if (!pr->v0 || !out_slices[i]) return fail(ctx, HJ_EINVAL, "problem %d: NULL v0 or output", i);
    }
    DeviceGuard guard(ctx->device);
    const long long launches0 = ctx->launches;

    // ---- instances the batched kernel serves; the others are solved one by one afterwards
    std::vector<Inst> insts;
    std::vector<int> single;
    for (int i = 0; i < n; ++i) {
        const hj_problem* pr = &problems[i];
        Inst in;
        in.idx = i;
        in.G = make_grid(&pr->grid, pr->method.extrap);
        in.dtype = pr->dtype;
        in.es = elem_size(pr->dtype);
        in.N = in.G.total;
        in.angles = pr->method.dynamics == HJ_DYN_AIR3D || pr->method.dynamics == HJ_DYN_DUBINS4D;
        if (rows_eligible(in.G, pr->method.scheme, pr->method.dynamics, pr->dtype) &&
            in.G.n[0] + 1 <= max_block_threads(pr->dtype))
            insts.push_back(in);
        else
            single.push_back(i);
    }

    hj_status st = HJ_OK;
    if (!insts.empty()) {
        // ---- arena 1: arrays, angle tables, slice staging, reduction slots
        size_t off = 0;
        for (Inst& in : insts) {
            const size_t bytes = align_up((size_t)in.N * in.es);
            in.off_v = off; off += bytes;
            in.off_v1 = off; off += bytes;
            in.off_v2 = off; off += bytes;
            if (in.angles) {
                in.off_td = off; off += align_up(2 * (size_t)in.G.n[2] * sizeof(double));
                in.off_tf = off; off += align_up(2 * (size_t)in.G.n[2] * sizeof(float));
            }
            if (!out_on_device[in.idx]) {  // slices staged on the device, copied to the host at the end
                in.off_stage = off;
                off += align_up((size_t)problems[in.idx].n_slices * in.N * in.es);
            }
        }
        const size_t off_slots = off;  // per instance: step-bound accumulator (8 B) + non-finite flag (8 B)
        off += align_up(insts.size() * 16);
        if ((st = ensure(ctx, &ctx->batch_arena, &ctx->batch_bytes, off))) return st;
        unsigned char* A = static_cast<unsigned char*>(ctx->batch_arena);
        unsigned long long* slots = reinterpret_cast<unsigned long long*>(A + off_slots);
        HJ_CUDA(ctx, cudaMemsetAsync(slots, 0, insts.size() * 16, ctx->stream));
        std::vector<std::vector<double>> tables(insts.size());
        std::vector<std::vector<float>> tables_f(insts.size());  // alive until the stream is synchronised below
        for (size_t j = 0; j < insts.size(); ++j) {
            Inst& in = insts[j];
            const hj_problem* pr = &problems[in.idx];
            HJ_CUDA(ctx, cudaMemcpyAsync(A + in.off_v, pr->v0, (size_t)in.N * in.es,
                                         pr->v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                         ctx->stream));
            if (in.angles) {
                angle_table(&pr->grid, &tables[j]);
                tables_f[j].assign(tables[j].begin(), tables[j].end());
                HJ_CUDA(ctx, cudaMemcpyAsync(A + in.off_td, tables[j].data(), tables[j].size() * sizeof(double),
                                             cudaMemcpyHostToDevice, ctx->stream));
                HJ_CUDA(ctx, cudaMemcpyAsync(A + in.off_tf, tables_f[j].data(), tables_f[j].size() * sizeof(float),
                                             cudaMemcpyHostToDevice, ctx->stream));
            }
            int* flag = reinterpret_cast<int*>(slots + 2 * j + 1);
            cudaError_t e = in.dtype == HJ_F64
                                ? launch_nonfinite_f64(reinterpret_cast<const double*>(A + in.off_v), in.N, flag, ctx->stream)
                                : launch_nonfinite_f32(reinterpret_cast<const float*>(A + in.off_v), in.N, flag, ctx->stream);
            if (e == cudaSuccess)
                e = launch_step_bound(in.G, pr->method.dynamics, pr->method.params,
                                      in.angles ? reinterpret_cast<const double*>(A + in.off_td) : nullptr,
                                      slots + 2 * j, ctx->stream);
            ctx->launches += 2;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batch set-up launch");
        }
        std::vector<unsigned long long> hslots(2 * insts.size());
        HJ_CUDA(ctx, cudaMemcpyAsync(hslots.data(), slots, hslots.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (size_t j = 0; j < insts.size(); ++j) {
            Inst& in = insts[j];
            if (hslots[2 * j + 1] & 0xffffffffull) return fail(ctx, HJ_ENONFINITE, "problem %d: v0 holds NaN or Inf", in.idx);
            std::memcpy(&in.sbi, &hslots[2 * j], sizeof(double));
            const hj_problem* pr = &problems[in.idx];
            plan_schedule(&pr->method, in.sbi, pr->n_slices, pr->slice_times, &in.S);
            for (int s = 0; s < pr->n_slices; ++s) {
                const long long e = in.S.slice_steps[s];
                if (e > 0 && (in.ends.empty() || in.ends.back() != e)) {
                    in.ends.push_back(e);
                    in.end_slice.push_back(s);
                }
            }
        }

        // ---- groups by (dtype, dimension, dynamics)
        std::vector<Group> groups;
        for (size_t j = 0; j < insts.size(); ++j) {
            Inst& in = insts[j];
            const int dyn = problems[in.idx].method.dynamics;
            int gi = -1;
            for (size_t k = 0; k < groups.size(); ++k)
                if (groups[k].dtype == in.dtype && groups[k].ndim == in.G.ndim && groups[k].dyn == dyn) gi = (int)k;
            if (gi < 0) {
                groups.push_back(Group{in.dtype, in.G.ndim, dyn});
                gi = (int)groups.size() - 1;
            }
            in.group = gi;
            groups[gi].members.push_back((int)j);
        }

        // ---- arena 2: descriptors, schedules, tile lists
        size_t off2 = align_up(insts.size() * sizeof(BatchInst));
        for (Inst& in : insts) {
            in.off_dts = off2; off2 += align_up(std::max<size_t>(1, in.S.dts.size()) * sizeof(double));
            in.off_ends = off2; off2 += align_up(std::max<size_t>(1, in.ends.size()) * sizeof(long long));
            in.off_end_slice = off2; off2 += align_up(std::max<size_t>(1, in.end_slice.size()) * sizeof(int));
        }
        for (Group& g : groups) {
            // the most tiles any shape below can produce: one row per tile, one plane per chunk
            size_t cap = 0;
            for (int m : g.members) {
                const GridDev& G = insts[m].G;
                cap += (size_t)G.n[1] * (G.ndim >= 3 ? G.n[G.ndim - 1] : 1) * (G.ndim == 4 ? G.n[2] : 1);
            }
            g.tile_cap = cap;
            g.off_tiles = off2;
            off2 += align_up(cap * sizeof(BatchTile));
        }
        if ((st = ensure(ctx, &ctx->batch_aux, &ctx->batch_aux_bytes, off2))) return st;
        unsigned char* B = static_cast<unsigned char*>(ctx->batch_aux);
        BatchInst* d_insts = reinterpret_cast<BatchInst*>(B);

        std::vector<BatchInst> hdesc(insts.size());
        for (size_t j = 0; j < insts.size(); ++j) {
            Inst& in = insts[j];
            const hj_problem* pr = &problems[in.idx];
            BatchInst& D = hdesc[j];
            std::memset(&D, 0, sizeof D);
            StageParams P = stage_params(ctx, in.G, &pr->method, in.dtype);
            P.trig_d = in.angles ? reinterpret_cast<const double*>(A + in.off_td) : nullptr;
            P.trig_f = in.angles ? reinterpret_cast<const float*>(A + in.off_tf) : nullptr;
            P.mode = kStage;
            D.P = finalize(P);
            D.steps_total = (int)in.S.dts.size();
            D.k = 0;
            D.dt = in.S.dts.empty() ? 0.0 : in.S.dts[0];
            D.dt_f = (float)D.dt;
            D.brt = pr->method.brt;
            D.V = A + in.off_v;
            D.V1 = A + in.off_v1;
            D.V2 = A + in.off_v2;
            D.dts = reinterpret_cast<const double*>(B + in.off_dts);
            D.ends = reinterpret_cast<const long long*>(B + in.off_ends);
            D.end_slice = reinterpret_cast<const int*>(B + in.off_end_slice);
            D.n_ends = (int)in.ends.size();
            D.out = out_on_device[in.idx] ? out_slices[in.idx] : (void*)(A + in.off_stage);
            D.nodes = in.N;
            D.elem = (int)in.es;
            D.cursor = 0;
            D.slice_out = nullptr;
            if (!in.ends.empty() && in.ends[0] == 1) {
                D.slice_out = static_cast<char*>(D.out) + (size_t)in.end_slice[0] * in.N * in.es;
                D.cursor = 1;
            }
            if (!in.S.dts.empty())
                HJ_CUDA(ctx, cudaMemcpyAsync(B + in.off_dts, in.S.dts.data(), in.S.dts.size() * sizeof(double),
                                             cudaMemcpyHostToDevice, ctx->stream));
            if (!in.ends.empty()) {
                HJ_CUDA(ctx, cudaMemcpyAsync(B + in.off_ends, in.ends.data(), in.ends.size() * sizeof(long long),
                                             cudaMemcpyHostToDevice, ctx->stream));
                HJ_CUDA(ctx, cudaMemcpyAsync(B + in.off_end_slice, in.end_slice.data(),
                                             in.end_slice.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
            }
            // slices taken before any step hold V0
            for (int s = 0; s < pr->n_slices; ++s)
                if (in.S.slice_steps[s] == 0)
                    HJ_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(D.out) + (size_t)s * in.N * in.es, A + in.off_v,
                                                 (size_t)in.N * in.es, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        HJ_CUDA(ctx, cudaMemcpyAsync(d_insts, hdesc.data(), hdesc.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                                     ctx->stream));

        // ---- launch shape per group: measured once per (dtype, dimension, dynamics) and context
        for (Group& g : groups) {
            int max_nx = 0;
            for (int m : g.members) max_nx = std::max(max_nx, insts[m].G.n[0]);
            const std::vector<long long> key = {g.dtype, g.ndim, g.dyn};
            auto set_shape = [&](int threads, int tzt) {
                g.threads = threads;
                g.tz_target = tzt;
                g.smem = 0;
                for (int m : g.members) {
                    shape_for(insts[m], threads, tzt, &insts[m].ty, &insts[m].tz);
                    g.smem = std::max(g.smem, rows_smem(insts[m].G.n[0], insts[m].ty, insts[m].es));
                }
            };
            auto it = ctx->batch_shape.find(key);
            if (it != ctx->batch_shape.end() && it->second.first >= max_nx + 1) {
                set_shape(it->second.first, it->second.second);
                continue;
            }
            std::vector<std::pair<int, int>> cands;
            for (int threads : {256, 512, 1024})
                if (threads <= max_block_threads(g.dtype) && threads >= max_nx + 1)
                    for (int tzt : {4, 8, 16, 32}) cands.push_back({threads, tzt});
            if (cands.empty()) {
                const int t = ((max_nx + 1 + 31) / 32) * 32;
                cands.push_back({std::min(t, max_block_threads(g.dtype)), 8});
            }
            std::pair<int, int> best = cands[0];
            if (cands.size() > 1) {
                cudaEvent_t e0, e1;
                HJ_CUDA(ctx, cudaEventCreate(&e0));
                HJ_CUDA(ctx, cudaEventCreate(&e1));
                float best_ms = 1e30f;
                for (auto c : cands) {
                    set_shape(c.first, c.second);
                    for (int m : g.members) {
                        BatchInst& D = hdesc[m];
                        D.ty = insts[m].ty;
                        D.tz = insts[m].tz;
                    }
                    HJ_CUDA(ctx, cudaMemcpyAsync(d_insts, hdesc.data(), hdesc.size() * sizeof(BatchInst),
                                                 cudaMemcpyHostToDevice, ctx->stream));
                    build_tiles(insts, g, 0, nullptr);
                    HJ_CUDA(ctx, cudaMemcpyAsync(B + g.off_tiles, g.tiles.data(), g.tiles.size() * sizeof(BatchTile),
                                                 cudaMemcpyHostToDevice, ctx->stream));
                    // stage 1 only writes V1, which the first real step rewrites
                    cudaError_t e = launch_group_stage(ctx, g, d_insts, B, 1, ctx->stream);
                    float ms = 1e30f;
                    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                        cudaEventRecord(e0, ctx->stream);
                        e = launch_group_stage(ctx, g, d_insts, B, 1, ctx->stream);
                        cudaEventRecord(e1, ctx->stream);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        float x = 0.f;
                        if (e == cudaSuccess) cudaEventElapsedTime(&x, e0, e1);
                        ms = std::min(ms, x);
                    }
                    if (e != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return cuda_fail(ctx, e, "batch tuning launch");
                    }
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
            set_shape(best.first, best.second);
            ctx->batch_shape[key] = best;
        }
        for (size_t j = 0; j < insts.size(); ++j) {
            hdesc[j].ty = insts[j].ty;
            hdesc[j].tz = insts[j].tz;
        }
        HJ_CUDA(ctx, cudaMemcpyAsync(d_insts, hdesc.data(), hdesc.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                                     ctx->stream));

        // ---- the step loop
        long long max_steps = 0;
        for (const Inst& in : insts) max_steps = std::max<long long>(max_steps, (long long)in.S.dts.size());
        if (!ctx->capture_stream) HJ_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        long long gstep = 0;
        cudaError_t err = cudaSuccess;
        while (gstep < max_steps && err == cudaSuccess) {
            size_t active_tiles = 0;
            for (Group& g : groups) {
                build_tiles(insts, g, gstep, nullptr);
                active_tiles += g.tiles.size();
                if (!g.tiles.empty()) {
                    err = cudaMemcpyAsync(B + g.off_tiles, g.tiles.data(), g.tiles.size() * sizeof(BatchTile),
                                          cudaMemcpyHostToDevice, ctx->stream);
                    if (err != cudaSuccess) break;
                }
            }
            if (err != cudaSuccess) break;
            // this tile list serves until a quarter of its tiles belong to finished instances
            long long seg_end = max_steps;
            {
                std::vector<long long> ends_sorted;
                for (const Inst& in : insts)
                    if ((long long)in.S.dts.size() > gstep) ends_sorted.push_back((long long)in.S.dts.size());
                std::sort(ends_sorted.begin(), ends_sorted.end());
                ends_sorted.erase(std::unique(ends_sorted.begin(), ends_sorted.end()), ends_sorted.end());
                size_t dead = 0;
                for (long long e : ends_sorted) {
                    if (e >= max_steps) break;
                    for (const Inst& in : insts)
                        if ((long long)in.S.dts.size() == e) {
                            const int D = in.G.ndim;
                            const size_t t = (size_t)((in.G.n[1] + in.ty - 1) / in.ty) *
                                             (D >= 3 ? (in.G.n[D - 1] + in.tz - 1) / in.tz : 1) *
                                             (D == 4 ? in.G.n[2] : 1);
                            dead += t;
                        }
                    if (4 * dead >= active_tiles) {
                        seg_end = e;
                        break;
                    }
                }
            }
            const long long seg = seg_end - gstep;
            const int K = (int)std::min<long long>(seg, kGraphSteps);
            cudaGraphExec_t exec = nullptr;
            if (seg >= 2 * K && K >= 2) {
                // capture K steps on the private stream, replay on the context's stream
                cudaGraph_t graph = nullptr;
                err = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
                for (int k = 0; k < K && err == cudaSuccess; ++k)
                    err = enqueue_step(ctx, groups, d_insts, (int)insts.size(), B, ctx->capture_stream, false);
                cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
                if (err == cudaSuccess) err = e2;
                if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
            }
            long long done = 0;
            if (exec && err == cudaSuccess) {
                for (; done + K <= seg && err == cudaSuccess; done += K) {
                    err = cudaGraphLaunch(exec, ctx->stream);
                    ctx->launches += K * launches_per_step(groups);
                }
            }
            for (; done < seg && err == cudaSuccess; ++done)
                err = enqueue_step(ctx, groups, d_insts, (int)insts.size(), B, ctx->stream, true);
            if (exec) {
                // the exec may still run: it is destroyed after the stream passes this point
                cudaStreamSynchronize(ctx->stream);
                cudaGraphExecDestroy(exec);
            }
            gstep = seg_end;
        }
        if (err != cudaSuccess) return cuda_fail(ctx, err, "batch step loop");

        // ---- results: duplicate slices, host copies, final checks
        HJ_CUDA(ctx, cudaMemsetAsync(slots, 0, insts.size() * 16, ctx->stream));
        for (size_t j = 0; j < insts.size(); ++j) {
            const Inst& in = insts[j];
            const hj_problem* pr = &problems[in.idx];
            const BatchInst& D = hdesc[j];
            const size_t bytes = (size_t)in.N * in.es;
            for (int s = 1; s < pr->n_slices; ++s)
                if (in.S.slice_steps[s] > 0 && in.S.slice_steps[s] == in.S.slice_steps[s - 1])
                    HJ_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(D.out) + (size_t)s * bytes,
                                                 static_cast<char*>(D.out) + (size_t)(s - 1) * bytes, bytes,
                                                 cudaMemcpyDeviceToDevice, ctx->stream));
            int* flag = reinterpret_cast<int*>(slots + 2 * j + 1);
            cudaError_t e = in.dtype == HJ_F64
                                ? launch_nonfinite_f64(reinterpret_cast<const double*>(A + in.off_v), in.N, flag, ctx->stream)
                                : launch_nonfinite_f32(reinterpret_cast<const float*>(A + in.off_v), in.N, flag, ctx->stream);
            ctx->launches += 1;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batch final check");
            if (!out_on_device[in.idx])
                HJ_CUDA(ctx, cudaMemcpyAsync(out_slices[in.idx], D.out, (size_t)pr->n_slices * bytes,
                                             cudaMemcpyDeviceToHost, ctx->stream));
        }
        HJ_CUDA(ctx, cudaMemcpyAsync(hslots.data(), slots, hslots.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        HJ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (size_t j = 0; j < insts.size(); ++j) {
            const Inst& in = insts[j];
            if (hslots[2 * j + 1] & 0xffffffffull)
                return fail(ctx, HJ_ENONFINITE, "problem %d: the solution became non-finite", in.idx);
            const hj_problem* pr = &problems[in.idx];
            if (out_times)
                if (double* ot = out_times[in.idx])
                    for (int s = 0; s < pr->n_slices; ++s) ot[s] = in.S.slice_t[s];
            if (stats) {
                hj_stats& S = stats[in.idx];
                S.steps = (long long)in.S.dts.size();
                S.cell_updates = S.steps * in.N;
                S.step_bound_inv = in.sbi;
                S.t_final = in.S.slice_t[pr->n_slices - 1];
            }
        }
    }
    // ---- instances the batched kernel does not cover
    for (int i : single) {
        hj_stats s1;
        st = hj_solve(ctx, &problems[i], out_slices[i], out_on_device[i], out_times ? out_times[i] : nullptr, &s1);
        if (st) {
            const std::string msg = ctx->last_error;
            return fail(ctx, st, "problem %d: %s", i, msg.c_str());
        }
        if (stats) stats[i] = s1;
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
        for (int i = 0; i < n; ++i) {
            stats[i].elapsed_ms = ms;
            stats[i].kernel_launches = ctx->launches - launches0;
        }
    return HJ_OK;
}
