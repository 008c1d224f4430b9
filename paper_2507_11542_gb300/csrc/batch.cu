// batch.cu -- hj_solve_batch: many independent solves advanced together by
// the Engine (engine.h): every eligible problem takes a slot, all slots are
// activated with one synchronisation, and K-step blocks (CUDA graphs) run
// until every instance has taken all of its steps. Problems the batched row
// kernel does not serve are solved one by one with hj_solve.
#include <chrono>
#include <string>
#include <vector>

#include "ctx.h"
#include "engine.h"

using namespace hj;

namespace {
constexpr int kBlockSteps = 16;

// Releases every slot of the engine (after an error mid-way).
void clear_engine(Engine* eng) {
    for (size_t i = 0; i < eng->slots.size(); ++i)
        if (eng->slots[i].used) eng->drop((int)i);
}
}  // namespace

extern "C" hj_status hj_solve_batch(hj_ctx* ctx, int32_t n, const hj_problem* problems, void* const* out_slices,
                                    const int32_t* out_on_device, double* const* out_times, hj_stats* stats) {
    NvtxRange range("hj_solve_batch");
    if (!ctx) return HJ_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    if (n < 0 || (n > 0 && (!problems || !out_slices || !out_on_device)))
        return fail(ctx, HJ_EINVAL, "batch needs problems, outputs and output placement flags");
    if (n == 0) return HJ_OK;
    for (int i = 0; i < n; ++i) {  // everything is validated before any work
        const hj_problem* pr = &problems[i];
        hj_status st;
        if ((st = check_grid(ctx, &pr->grid)) || (st = check_method(ctx, &pr->grid, &pr->method)) ||
            (st = check_solver_settings(ctx, &pr->method)) || (st = check_slices(ctx, pr->n_slices, pr->slice_times, pr->t0))) {
            const std::string msg = ctx->last_error;
            return fail(ctx, st, "problem %d: %s", i, msg.c_str());
        }
        if (!elem_size(pr->dtype)) return fail(ctx, HJ_EINVAL, "problem %d: unknown dtype", i);
        if (!pr->v0 || !out_slices[i]) return fail(ctx, HJ_EINVAL, "problem %d: NULL v0 or output", i);
    }
    DeviceGuard guard(ctx->device);
    const long long launches0 = ctx->launches;
    std::vector<int> batched, single;
    size_t need = 0;
    for (int i = 0; i < n; ++i) {
        if (Engine::eligible(&problems[i])) {
            batched.push_back(i);
            need += Engine::footprint(&problems[i], out_on_device[i] != 0) + 256;
        } else {
            single.push_back(i);
        }
    }
    hj_status st = HJ_OK;
    if (!batched.empty()) {
        if (!ctx->batch_engine || ctx->batch_engine_bytes < need || ctx->batch_engine_slots < (int)batched.size()) {
            delete ctx->batch_engine;
            ctx->batch_engine = nullptr;
            Engine* e = new Engine();
            if ((st = e->init(ctx, ctx->stream, (int)batched.size(), need))) {
                delete e;
                return st;
            }
            ctx->batch_engine = e;
            ctx->batch_engine_bytes = need;
            ctx->batch_engine_slots = (int)batched.size();
        }
        Engine* eng = ctx->batch_engine;
        for (int i : batched) {
            int slot = -1;
            st = eng->admit(&problems[i], out_slices[i], out_on_device[i] != 0, out_times ? out_times[i] : nullptr,
                            (uint64_t)i, &slot);
            if (st) {
                clear_engine(eng);
                return st == HJ_EBUSY ? fail(ctx, HJ_ENOMEM, "problem %d does not fit the batch arena", i) : st;
            }
        }
        std::vector<int> failed;
        if ((st = eng->activate(&failed))) {
            clear_engine(eng);
            return st;
        }
        if (!failed.empty()) {
            const int idx = (int)eng->slots[failed[0]].tag;
            clear_engine(eng);
            return fail(ctx, HJ_ENONFINITE, "problem %d: v0 holds NaN or Inf", idx);
        }
        while (eng->any_active()) {
            if ((st = eng->run(kBlockSteps))) {
                clear_engine(eng);
                return st;
            }
        }
        std::vector<int> done;
        eng->done_slots(&done);
        if ((st = eng->retire(done))) {
            clear_engine(eng);
            return st;
        }
        for (int si : done) {
            const Slot& S = eng->slots[si];
            if (S.status) return fail(ctx, S.status, "problem %d: the solution became non-finite", (int)S.tag);
            if (stats) stats[S.tag] = S.stats;
        }
    }
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
            stats[i].queued_ms = 0.0;
            stats[i].kernel_launches = ctx->launches - launches0;
        }
    return HJ_OK;
}
