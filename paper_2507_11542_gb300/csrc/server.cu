// server.cu -- hj_server_*: a continuous-batching request loop.
//
// Requests are queued by hj_server_submit (never blocks). An engine thread
// owns a private stream, context and Engine (engine.h) whose arena is the
// server's HBM budget. Each tick it admits queued requests in arrival order
// while a slot is free and the request's footprint fits the arena, activates
// them, advances every in-flight request by a block of RK3 steps (one
// batched launch per stage and group, replayed as a CUDA graph), and retires
// the requests that finished: their grids stay on the device from admission
// to retirement, and requests that arrive while others run join at the next
// tick. Latency is measured from submission to retirement.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.h"
#include "engine.h"

using namespace hj;

namespace {
constexpr int kTickSteps = 8;
using Clock = std::chrono::steady_clock;

struct Request {
    hj_problem prob;
    std::vector<double> times;
    void* out = nullptr;
    int out_on_device = 1;
    double* out_times = nullptr;
    size_t footprint = 0;
    int state = 0;  // 0 queued, 1 on the device, 2 done
    bool cancel = false;
    int slot = -1;
    hj_status status = HJ_OK;
    hj_stats stats{};
    Clock::time_point t_submit;
    Clock::time_point t_admit;  // when it left the queue (valid once state >= 1)
    bool admitted = false;
};
}  // namespace

struct hj_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    hj_ctx* ctx = nullptr;  // private: used only by the engine thread
    Engine eng;
    size_t budget = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    hj_status fatal = HJ_OK;
    std::string fatal_msg;
    uint64_t completed = 0;
    size_t bytes_in_use = 0;
    long long launches = 0;  // the engine's kernel launches, copied under the lock each tick
    std::thread th;
};

namespace {

void finish(hj_server* s, uint64_t ticket, hj_status st) {
    Request& r = s->reqs[ticket];
    r.state = 2;
    r.status = st;
    const Clock::time_point now = Clock::now();
    r.stats.elapsed_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
    r.stats.queued_ms = std::chrono::duration<double, std::milli>((r.admitted ? r.t_admit : now) - r.t_submit).count();
    s->completed += 1;
}

void engine_loop(hj_server* s) {
    cudaSetDevice(s->device);
    std::unordered_map<int, uint64_t> slot_ticket;
    std::vector<int> done, failed;
    for (;;) {
        std::vector<uint64_t> admit, cancel_running;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            for (auto& kv : s->reqs)
                if (kv.second.state == 1 && kv.second.cancel) cancel_running.push_back(kv.first);
            // admission in arrival order while a slot is free and the footprint fits
            int free_slots = 0;
            for (const Slot& sl : s->eng.slots) free_slots += !sl.used;
            size_t free_bytes = s->budget > s->bytes_in_use ? s->budget - s->bytes_in_use : 0;
            while (!s->queue.empty() && free_slots > 0) {
                Request& r = s->reqs[s->queue.front()];
                if (r.footprint + 256 > free_bytes) break;
                free_bytes -= r.footprint + 256;
                free_slots -= 1;
                admit.push_back(s->queue.front());
                s->queue.pop_front();
                r.state = 1;
                r.admitted = true;
                r.t_admit = Clock::now();
            }
            if (admit.empty() && cancel_running.empty() && !s->eng.any_active()) {
                s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        NvtxRange tick_range("server tick");  // admission, activation, steps and retirement of one tick
        hj_status st = HJ_OK;
        // cancellations of requests on the device take effect here, between blocks of steps
        for (uint64_t t : cancel_running) {
            int slot;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                slot = s->reqs[t].slot;
            }
            if (slot >= 0 && (st = s->eng.drop(slot))) break;
            std::lock_guard<std::mutex> lk(s->mu);
            s->bytes_in_use -= s->reqs[t].footprint + 256;
            slot_ticket.erase(slot);
            finish(s, t, HJ_ECANCELLED);
        }
        for (size_t a = 0; a < admit.size() && st == HJ_OK; ++a) {
            Request* r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = &s->reqs[admit[a]];
            }
            int slot = -1;
            hj_status ast = s->eng.admit(&r->prob, r->out, r->out_on_device != 0, r->out_times, admit[a], &slot);
            std::lock_guard<std::mutex> lk(s->mu);
            if (ast == HJ_EBUSY) {  // the arena is fragmented: retry later, keeping arrival order
                for (size_t b = admit.size(); b-- > a;) {
                    s->reqs[admit[b]].state = 0;
                    s->reqs[admit[b]].admitted = false;
                    s->queue.push_front(admit[b]);
                }
                break;
            }
            if (ast) {
                st = ast;
                break;
            }
            r->slot = slot;
            s->bytes_in_use += r->footprint + 256;
            slot_ticket[slot] = admit[a];
        }
        if (st == HJ_OK) st = s->eng.activate(&failed);
        if (st == HJ_OK && !failed.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int sl : failed) {
                const uint64_t t = slot_ticket[sl];
                s->bytes_in_use -= s->reqs[t].footprint + 256;
                slot_ticket.erase(sl);
                finish(s, t, HJ_ENONFINITE);
            }
            s->cv_done.notify_all();
        }
        if (st == HJ_OK && s->eng.any_active()) st = s->eng.run(kTickSteps);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->launches = s->eng.launches;
        }
        if (st == HJ_OK) {
            s->eng.done_slots(&done);
            if (!done.empty()) st = s->eng.retire(done);
            if (st == HJ_OK && !done.empty()) {
                std::lock_guard<std::mutex> lk(s->mu);
                for (int sl : done) {
                    const uint64_t t = slot_ticket[sl];
                    Request& r = s->reqs[t];
                    r.stats = s->eng.slots[sl].stats;
                    s->bytes_in_use -= r.footprint + 256;
                    slot_ticket.erase(sl);
                    finish(s, t, s->eng.slots[sl].status);
                }
                s->cv_done.notify_all();
            }
        }
        if (st != HJ_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->fatal = st;
            s->fatal_msg = hj_ctx_last_error(s->ctx);
            for (auto& kv : s->reqs)
                if (kv.second.state != 2) finish(s, kv.first, st);
            s->queue.clear();
            s->cv_done.notify_all();
            break;
        }
    }
    // shutting down: everything not finished is cancelled
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs)
        if (kv.second.state != 2) finish(s, kv.first, HJ_ECANCELLED);
    s->queue.clear();
    s->cv_done.notify_all();
}

}  // namespace

extern "C" {

hj_status hj_server_create(hj_ctx* ctx, size_t hbm_budget, int32_t max_slots, hj_server** out) {
    if (!ctx || !out || max_slots < 1 || hbm_budget < 4096) return HJ_EINVAL;
    *out = nullptr;
    DeviceGuard guard(ctx->device);
    hj_server* s = new (std::nothrow) hj_server();
    if (!s) return HJ_ENOMEM;
    s->device = ctx->device;
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return fail(ctx, HJ_ECUDA, "server stream");
    }
    hj_status st = hj_ctx_create(ctx->device, s->stream, &s->ctx);
    if (st == HJ_OK) st = s->eng.init(s->ctx, s->stream, max_slots, hbm_budget, /*multirate=*/true);
    if (st != HJ_OK) {
        const std::string msg = s->ctx ? hj_ctx_last_error(s->ctx) : "";
        s->eng.shutdown();
        if (s->ctx) hj_ctx_destroy(s->ctx);
        cudaStreamDestroy(s->stream);
        delete s;
        return fail(ctx, st, "server set-up: %s", msg.c_str());
    }
    s->th = std::thread(engine_loop, s);
    *out = s;
    return HJ_OK;
}

hj_status hj_server_submit(hj_server* s, const hj_problem* p, void* out_slices, int32_t out_on_device,
                           double* out_times, uint64_t* ticket) {
    if (!s || !p || !ticket || !out_slices || !p->v0) return HJ_EINVAL;
    *ticket = 0;
    if (check_grid(nullptr, &p->grid) || check_method(nullptr, &p->grid, &p->method) ||
        check_solver_settings(nullptr, &p->method) || check_slices(nullptr, p->n_slices, p->slice_times, p->t0) ||
        !elem_size(p->dtype))
        return HJ_EINVAL;
    if (!Engine::eligible(p)) return HJ_EINVAL;
    const size_t fp = Engine::footprint(p, out_on_device != 0);
    if (fp + 256 > s->budget) return HJ_ENOMEM;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop || s->fatal) return s->fatal ? s->fatal : HJ_ECANCELLED;
    const uint64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.prob = *p;
    r.times.assign(p->slice_times, p->slice_times + p->n_slices);
    r.prob.slice_times = r.times.data();
    r.out = out_slices;
    r.out_on_device = out_on_device;
    r.out_times = out_times;
    r.footprint = fp;
    r.t_submit = Clock::now();
    s->queue.push_back(t);
    s->cv_work.notify_one();
    *ticket = t;
    return HJ_OK;
}

hj_status hj_server_wait(hj_server* s, uint64_t ticket, int32_t timeout_ms, hj_stats* stats) {
    if (!s) return HJ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HJ_EINVAL;
    auto is_done = [&] { return s->reqs[ticket].state == 2; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, is_done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), is_done)) {
        return HJ_ETIMEOUT;
    }
    Request& r = s->reqs[ticket];
    const hj_status st = r.status;
    if (stats) *stats = r.stats;
    s->reqs.erase(ticket);
    return st;
}

hj_status hj_server_cancel(hj_server* s, uint64_t ticket) {
    if (!s) return HJ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.state == 2) return HJ_EINVAL;
    if (it->second.state == 0) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == ticket) {
                s->queue.erase(q);
                break;
            }
        finish(s, ticket, HJ_ECANCELLED);
        s->cv_done.notify_all();
    } else {
        it->second.cancel = true;
        s->cv_work.notify_one();
    }
    return HJ_OK;
}

hj_status hj_server_counters(hj_server* s, hj_server_info* info) {
    if (!s || !info) return HJ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    info->queued = (int64_t)s->queue.size();
    int64_t running = 0;
    for (const auto& kv : s->reqs) running += kv.second.state == 1;
    info->running = running;
    info->completed = (int64_t)s->completed;
    info->bytes_in_use = (int64_t)s->bytes_in_use;
    info->budget = (int64_t)s->budget;
    info->kernel_launches = s->launches;
    return s->fatal;
}

void hj_server_destroy(hj_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    {
        DeviceGuard guard(s->device);
        cudaStreamSynchronize(s->stream);
        s->eng.shutdown();
        hj_ctx_destroy(s->ctx);
        cudaStreamDestroy(s->stream);
    }
    delete s;
}

}  // extern "C"
