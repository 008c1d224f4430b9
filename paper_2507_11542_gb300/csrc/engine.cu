// engine.cu -- see engine.h.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

namespace hj {

namespace {
constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
int max_block_threads(int dtype) { return rows_max_threads(dtype == HJ_F64); }
bool uses_angles(int dyn) { return dyn == HJ_DYN_AIR3D || dyn == HJ_DYN_DUBINS4D || dyn == HJ_DYN_ROCKETS; }
long long nodes_of(const hj_grid& g) {
    long long n = 1;
    for (int d = 0; d < g.ndim; ++d) n *= g.n[d];
    return n;
}
}  // namespace

// ---------------------------------------------------------------------------
// Arena
// ---------------------------------------------------------------------------
void Arena::reset(unsigned char* base, size_t cap) {
    base_ = base;
    cap_ = cap;
    used_ = 0;
    free_.clear();
    if (cap) free_.push_back({0, cap});
}

bool Arena::alloc(size_t bytes, size_t* off) {
    bytes = align_up(std::max<size_t>(bytes, 1));
    for (size_t i = 0; i < free_.size(); ++i) {
        if (free_[i].second >= bytes) {
            *off = free_[i].first;
            free_[i].first += bytes;
            free_[i].second -= bytes;
            if (free_[i].second == 0) free_.erase(free_.begin() + i);
            used_ += bytes;
            return true;
        }
    }
    return false;
}

void Arena::release(size_t off, size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1));
    used_ -= bytes;
    auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, (size_t)0));
    it = free_.insert(it, {off, bytes});
    // coalesce with the neighbours
    size_t i = it - free_.begin();
    if (i + 1 < free_.size() && free_[i].first + free_[i].second == free_[i + 1].first) {
        free_[i].second += free_[i + 1].second;
        free_.erase(free_.begin() + i + 1);
    }
    if (i > 0 && free_[i - 1].first + free_[i - 1].second == free_[i].first) {
        free_[i - 1].second += free_[i].second;
        free_.erase(free_.begin() + i);
    }
}

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
Engine::~Engine() { shutdown(); }

void Engine::drop_graphs() {
    for (int l = 0; l < kLanes; ++l) {
        if (exec_[l]) cudaGraphExecDestroy(exec_[l]);
        exec_[l] = nullptr;
        exec_K_[l] = 0;
    }
}

void Engine::shutdown() {
    drop_graphs();
    for (int l = 0; l < kLanes; ++l) {
        if (lane_stream_[l]) cudaStreamDestroy(lane_stream_[l]);
        if (lane_ev_[l]) cudaEventDestroy(lane_ev_[l]);
        lane_stream_[l] = nullptr;
        lane_ev_[l] = nullptr;
    }
    if (fork_ev_) cudaEventDestroy(fork_ev_);
    fork_ev_ = nullptr;
    for (Group& g : groups_) cudaFree(g.d_tiles);
    groups_.clear();
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    cap_stream_ = nullptr;
    cudaFree(arena_mem_);
    cudaFree(d_insts_);
    cudaFree(d_words_);
    arena_mem_ = nullptr;
    d_insts_ = nullptr;
    d_words_ = nullptr;
    slots.clear();
}

hj_status Engine::init(hj_ctx* ctx, cudaStream_t stream, int max_slots, size_t arena_bytes, bool multirate) {
    ctx_ = ctx;
    stream_ = stream;
    multirate_ = multirate;
    max_slots_ = std::max(1, max_slots);
    HJ_CUDA(ctx, cudaMalloc(&arena_mem_, std::max<size_t>(arena_bytes, kAlign)));
    arena_.reset(static_cast<unsigned char*>(arena_mem_), std::max<size_t>(arena_bytes, kAlign));
    HJ_CUDA(ctx, cudaMalloc(&d_insts_, sizeof(BatchInst) * max_slots_));
    HJ_CUDA(ctx, cudaMemsetAsync(d_insts_, 0, sizeof(BatchInst) * max_slots_, stream_));
    HJ_CUDA(ctx, cudaMalloc(&d_words_, 16 * (size_t)max_slots_));
    HJ_CUDA(ctx, cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
    if (multirate_) {
        HJ_CUDA(ctx, cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming));
        for (int l = 0; l < kLanes; ++l) {
            HJ_CUDA(ctx, cudaStreamCreateWithFlags(&lane_stream_[l], cudaStreamNonBlocking));
            HJ_CUDA(ctx, cudaEventCreateWithFlags(&lane_ev_[l], cudaEventDisableTiming));
        }
    }
    h_insts_.assign(max_slots_, BatchInst());
    std::memset(h_insts_.data(), 0, sizeof(BatchInst) * h_insts_.size());
    slots.assign(max_slots_, Slot());
    return HJ_OK;
}

bool Engine::eligible(const hj_problem* p) {
    const GridDev G = make_grid(&p->grid, p->method.extrap);
    const bool rk3_node = (p->method.order == 0 || p->method.order == 3) && p->method.alpha_mode == HJ_ALPHA_NODE;
    return rk3_node && default_launch(&p->method) && rows_eligible(G, p->method.scheme, p->method.dynamics, p->dtype) &&
           G.n[0] + 1 <= max_block_threads(p->dtype);
}

// The arena layout of one instance, as offsets from the start of its block:
// V, V1, V2, the angle tables (FP64, FP32), the host-output staging, and the
// slice schedule (ends, end_slice, end_dt). footprint() is its total size.
namespace {
struct SlotLayout {
    size_t v, v1, v2, td, tf, stage, ends, end_slice, end_dt, total;
};
SlotLayout slot_layout(const hj_problem* p, bool out_on_device) {
    const size_t es = elem_size(p->dtype);
    const size_t n = (size_t)nodes_of(p->grid);
    const size_t arr = align_up(n * es);
    SlotLayout L;
    size_t o = 0;
    L.v = o; o += arr;
    L.v1 = o; o += arr;
    L.v2 = o; o += arr;
    L.td = L.tf = L.stage = 0;
    if (uses_angles(p->method.dynamics)) {
        L.td = o; o += align_up(2 * (size_t)p->grid.n[2] * 8);
        L.tf = o; o += align_up(2 * (size_t)p->grid.n[2] * 4);
    }
    if (!out_on_device) {
        L.stage = o;
        o += align_up((size_t)p->n_slices * n * es);
    }
    L.ends = o; o += align_up((size_t)p->n_slices * 8);
    L.end_slice = o; o += align_up((size_t)p->n_slices * 8);
    L.end_dt = o; o += align_up((size_t)p->n_slices * 8);
    L.total = o;
    return L;
}
}  // namespace

size_t Engine::footprint(const hj_problem* p, bool out_on_device) { return slot_layout(p, out_on_device).total; }

int Engine::free_slot() const {
    for (int i = 0; i < max_slots_; ++i)
        if (!slots[i].used) return i;
    return -1;
}

hj_status Engine::admit(const hj_problem* p, void* out, bool out_on_device, double* out_times, uint64_t tag,
                        int* slot_out) {
    const int si = free_slot();
    if (si < 0) return HJ_EBUSY;
    size_t off = 0;
    const size_t bytes = footprint(p, out_on_device);
    if (!arena_.alloc(bytes, &off)) return HJ_EBUSY;
    Slot& S = slots[si];
    S = Slot();
    S.used = true;
    S.prob = *p;
    S.times.assign(p->slice_times, p->slice_times + p->n_slices);
    S.prob.slice_times = S.times.data();
    S.out = out;
    S.out_on_device = out_on_device;
    S.out_times = out_times;
    S.G = make_grid(&p->grid, p->method.extrap);
    S.dtype = p->dtype;
    S.es = elem_size(p->dtype);
    S.N = S.G.total;
    S.angles = uses_angles(p->method.dynamics);
    S.tag = tag;
    S.off = off;
    S.bytes = bytes;
    const SlotLayout L = slot_layout(p, out_on_device);
    S.o_v = off + L.v;
    S.o_v1 = off + L.v1;
    S.o_v2 = off + L.v2;
    if (S.angles) {
        S.o_td = off + L.td;
        S.o_tf = off + L.tf;
    }
    if (!out_on_device) S.o_stage = off + L.stage;
    S.o_ends = off + L.ends;
    S.o_end_slice = off + L.end_slice;
    S.o_end_dt = off + L.end_dt;
    unsigned char* A = arena_.base();
    HJ_CUDA(ctx_, cudaMemcpyAsync(A + S.o_v, p->v0, (size_t)S.N * S.es,
                                  p->v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream_));
    if (S.angles) {
        angle_table(&p->grid, &S.table);
        S.table_f.assign(S.table.begin(), S.table.end());
        HJ_CUDA(ctx_, cudaMemcpyAsync(A + S.o_td, S.table.data(), S.table.size() * 8, cudaMemcpyHostToDevice, stream_));
        HJ_CUDA(ctx_, cudaMemcpyAsync(A + S.o_tf, S.table_f.data(), S.table_f.size() * 4, cudaMemcpyHostToDevice,
                                      stream_));
    }
    unsigned long long* w = d_words_ + 2 * si;
    HJ_CUDA(ctx_, cudaMemsetAsync(w, 0, 16, stream_));
    cudaError_t e = S.dtype == HJ_F64
                        ? launch_nonfinite_f64(reinterpret_cast<const double*>(A + S.o_v), S.N, reinterpret_cast<int*>(w + 1), stream_)
                        : launch_nonfinite_f32(reinterpret_cast<const float*>(A + S.o_v), S.N, reinterpret_cast<int*>(w + 1), stream_);
    if (e == cudaSuccess)
        e = launch_step_bound(S.G, p->method.dynamics, p->method.params,
                              S.angles ? reinterpret_cast<const double*>(A + S.o_td) : nullptr, w, 0, stream_);
    launches += 2;
    ctx_->launches += 2;
    if (e != cudaSuccess) return cuda_fail(ctx_, e, "admission launch");
    pending_.push_back(si);
    *slot_out = si;
    return HJ_OK;
}

hj_status Engine::activate(std::vector<int>* failed) {
    NvtxRange range("activate instances");
    if (failed) failed->clear();
    if (pending_.empty()) return HJ_OK;
    std::vector<unsigned long long> words(2 * (size_t)max_slots_);
    HJ_CUDA(ctx_, cudaMemcpyAsync(words.data(), d_words_, words.size() * 8, cudaMemcpyDeviceToHost, stream_));
    HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
    unsigned char* A = arena_.base();
    std::vector<int> ok;
    for (int si : pending_) {
        Slot& S = slots[si];
        S.table.clear();
        S.table.shrink_to_fit();
        S.table_f.clear();
        S.table_f.shrink_to_fit();
        if (words[2 * si + 1] & 0xffffffffull) {
            S.status = HJ_ENONFINITE;
            if (failed) failed->push_back(si);
            arena_.release(S.off, S.bytes);
            S.used = false;
            continue;
        }
        std::memcpy(&S.sbi, &words[2 * si], sizeof(double));
        plan_schedule(&S.prob.method, S.sbi, S.prob.n_slices, S.prob.slice_times, S.prob.t0, &S.S);
        S.steps_total = (long long)S.S.dts.size();
        S.k_host = 0;
        // distinct positive slice step counts, the slice written there, and that step's dt
        std::vector<long long> ends;
        std::vector<long long> end_slice;
        std::vector<double> end_dt;
        for (int s = 0; s < S.prob.n_slices; ++s) {
            const long long e = S.S.slice_steps[s];
            if (e > 0 && (ends.empty() || ends.back() != e)) {
                ends.push_back(e);
                end_slice.push_back(s);
                end_dt.push_back(S.S.dts[e - 1]);
            }
        }
        double dt_full = std::fmin(S.prob.method.max_step, S.prob.method.cfl * (1.0 / S.sbi));
        // every step that ends no slice must use dt_full (the schedule's only clipped steps end slices)
        {
            size_t j = 0;
            for (long long k = 0; k < S.steps_total; ++k) {
                const bool ends_slice = j < ends.size() && ends[j] == k + 1;
                if (ends_slice) ++j;
                else if (S.S.dts[k] != dt_full) return fail(ctx_, HJ_EINVAL, "schedule step %lld is not the full step", k);
            }
        }
        std::vector<long long> es64(end_slice.begin(), end_slice.end());
        std::vector<int> es32(end_slice.begin(), end_slice.end());
        if (!ends.empty()) {
            HJ_CUDA(ctx_, cudaMemcpyAsync(A + S.o_ends, ends.data(), ends.size() * 8, cudaMemcpyHostToDevice, stream_));
            HJ_CUDA(ctx_, cudaMemcpyAsync(A + S.o_end_slice, es32.data(), es32.size() * 4, cudaMemcpyHostToDevice,
                                          stream_));
            HJ_CUDA(ctx_, cudaMemcpyAsync(A + S.o_end_dt, end_dt.data(), end_dt.size() * 8, cudaMemcpyHostToDevice,
                                          stream_));
        }
        void* outbase = S.out_on_device ? S.out : (void*)(A + S.o_stage);
        for (int s = 0; s < S.prob.n_slices; ++s)  // slices taken before any step hold V0
            if (S.S.slice_steps[s] == 0)
                HJ_CUDA(ctx_, cudaMemcpyAsync(static_cast<char*>(outbase) + (size_t)s * S.N * S.es, A + S.o_v,
                                              (size_t)S.N * S.es, cudaMemcpyDeviceToDevice, stream_));
        BatchInst& D = h_insts_[si];
        std::memset(&D, 0, sizeof D);
        StageParams P = stage_params(ctx_, S.G, &S.prob.method, S.dtype);
        P.trig_d = S.angles ? reinterpret_cast<const double*>(A + S.o_td) : nullptr;
        P.trig_f = S.angles ? reinterpret_cast<const float*>(A + S.o_tf) : nullptr;
        P.mode = kStage;
        D.P = finalize(P);
        D.steps_total = (int)S.steps_total;
        D.k = 0;
        D.brt = S.prob.method.brt;
        D.V = A + S.o_v;
        D.V1 = A + S.o_v1;
        D.V2 = A + S.o_v2;
        D.dt_full = dt_full;
        D.ends = reinterpret_cast<const long long*>(A + S.o_ends);
        D.end_slice = reinterpret_cast<const int*>(A + S.o_end_slice);
        D.end_dt = reinterpret_cast<const double*>(A + S.o_end_dt);
        D.n_ends = (int)ends.size();
        D.out = outbase;
        D.nodes = S.N;
        D.elem = (int)S.es;
        D.cursor = 0;
        D.dt = dt_full;
        D.slice_out = nullptr;
        if (!ends.empty() && ends[0] == 1) {
            D.dt = end_dt[0];
            D.slice_out = static_cast<char*>(outbase) + (size_t)end_slice[0] * S.N * S.es;
            D.cursor = 1;
        }
        D.dt_f = (float)D.dt;
        S.lane = !multirate_ ? 0 : lane_of(S.N);
        D.lane = S.lane;
        // group
        const int dyn = S.prob.method.dynamics;
        const int scheme = S.prob.method.scheme;
        int gi = -1;
        for (size_t k = 0; k < groups_.size(); ++k)
            if (groups_[k].dtype == S.dtype && groups_[k].ndim == S.G.ndim && groups_[k].dyn == dyn &&
                groups_[k].scheme == scheme)
                gi = (int)k;
        if (gi < 0) {
            Group g;
            g.dtype = S.dtype;
            g.ndim = S.G.ndim;
            g.dyn = dyn;
            g.scheme = scheme;
            groups_.push_back(g);
            gi = (int)groups_.size() - 1;
        }
        S.group = gi;
        ok.push_back(si);
    }
    pending_.clear();
    // launch shapes of the groups that gained members
    for (size_t gi = 0; gi < groups_.size(); ++gi) {
        std::vector<int> members, fresh;
        for (int i = 0; i < max_slots_; ++i)
            if (slots[i].used && slots[i].group == (int)gi) members.push_back(i);
        for (int si : ok)
            if (slots[si].group == (int)gi) fresh.push_back(si);
        if (fresh.empty()) continue;
        hj_status st = shape_group(groups_[gi], members, fresh);
        if (st) return st;
        // members already stepping keep their device state; only their tile shape is refreshed
        for (int m : members)
            if (std::find(fresh.begin(), fresh.end(), m) == fresh.end())
                HJ_CUDA(ctx_, cudaMemcpyAsync(reinterpret_cast<char*>(d_insts_ + m) + offsetof(BatchInst, ty),
                                              &h_insts_[m].ty, 2 * sizeof(int), cudaMemcpyHostToDevice, stream_));
    }
    for (int si : ok) {
        h_insts_[si].ty = slots[si].ty;
        h_insts_[si].tz = slots[si].tz;
        HJ_CUDA(ctx_, cudaMemcpyAsync(d_insts_ + si, &h_insts_[si], sizeof(BatchInst), cudaMemcpyHostToDevice, stream_));
        slots[si].active = slots[si].steps_total > 0;
    }
    // the descriptors' host copies must stay alive until the copies run
    HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
    tiles_dirty_ = true;
    return HJ_OK;
}

namespace {
void tile_shape(const Slot& S, int threads, int tz_target, int* ty, int* tz) {
    const int nx = S.G.n[0], ny = S.G.n[1];
    // node rows: the most whose block (rows_block_threads) fits `threads`
    int t = 1;
    while (t < ny && rows_block_threads(nx, t + 1, threads) <= threads) ++t;
    while (t > 1 && rows_smem(nx, t, S.es) > 200 * 1024) --t;
    *ty = t;
    const int D = S.G.ndim;
    *tz = D >= 3 ? std::max(1, std::min(tz_target, S.G.n[D - 1])) : 1;
}
long long tiles_of(const Slot& S) {
    const int D = S.G.ndim;
    return (long long)((S.G.n[1] + S.ty - 1) / S.ty) * (D >= 3 ? (S.G.n[D - 1] + S.tz - 1) / S.tz : 1) *
           (D == 4 ? S.G.n[2] : 1);
}
void append_tiles(const Slot& S, int si, std::vector<BatchTile>* out) {
    const int D = S.G.ndim;
    const int rt = (S.G.n[1] + S.ty - 1) / S.ty;
    const int ns = D >= 3 ? S.G.n[D - 1] : 1;
    const int nch = D >= 3 ? (ns + S.tz - 1) / S.tz : 1;
    const int n2 = D == 4 ? S.G.n[2] : 1;
    for (int c = 0; c < nch; ++c)
        for (int j = 0; j < n2; ++j)
            for (int t = 0; t < rt; ++t) out->push_back(BatchTile{si, t, j, c});
}
}  // namespace

// The group's block size and planes per tile: measured once per (dtype,
// dimension, dynamics, scheme) and context on the members at hand, then reused.
hj_status Engine::shape_group(Group& g, const std::vector<int>& members, const std::vector<int>& fresh) {
    int max_nx = 0;
    for (int m : members) max_nx = std::max(max_nx, slots[m].G.n[0]);
    auto apply = [&](int threads, int tzt) {
        g.threads = threads;
        g.tz_target = tzt;
        g.smem = 0;
        for (int m : members) {
            tile_shape(slots[m], threads, tzt, &slots[m].ty, &slots[m].tz);
            g.smem = std::max(g.smem, rows_smem(slots[m].G.n[0], slots[m].ty, slots[m].es));
            h_insts_[m].ty = slots[m].ty;
            h_insts_[m].tz = slots[m].tz;
        }
    };
    const std::vector<long long> key = {g.dtype, g.ndim, g.dyn, g.scheme};
    auto it = ctx_->batch_shape.find(key);
    if (it != ctx_->batch_shape.end() && it->second.first >= max_nx + 1) {
        apply(it->second.first, it->second.second);
        return HJ_OK;
    }
    std::vector<std::pair<int, int>> cands;
    for (int threads : {256, 512, 1024})
        if (threads <= max_block_threads(g.dtype) && threads >= max_nx + 1)
            for (int tzt : {4, 8, 16, 32}) cands.push_back({threads, tzt});
    if (cands.empty()) cands.push_back({std::min(((max_nx + 1 + 31) / 32) * 32, max_block_threads(g.dtype)), 8});
    std::pair<int, int> best = cands[0];
    if (cands.size() > 1) {
        cudaEvent_t e0, e1;
        HJ_CUDA(ctx_, cudaEventCreate(&e0));
        HJ_CUDA(ctx_, cudaEventCreate(&e1));
        float best_ms = 1e30f;
        cudaError_t e = cudaSuccess;
        for (auto c : cands) {
            // timed on the new members only (their descriptors have not started stepping)
            apply(c.first, c.second);
            for (int m : fresh)
                e = cudaMemcpyAsync(d_insts_ + m, &h_insts_[m], sizeof(BatchInst), cudaMemcpyHostToDevice, stream_);
            g.tiles.clear();
            for (int m : fresh) append_tiles(slots[m], m, &g.tiles);
            if (g.tiles.size() > g.tile_cap) {
                cudaStreamSynchronize(stream_);
                cudaFree(g.d_tiles);
                g.d_tiles = nullptr;
                g.tile_cap = g.tiles.size() * 2;
                e = cudaMalloc(&g.d_tiles, g.tile_cap * sizeof(BatchTile));
                if (e != cudaSuccess) {
                    g.d_tiles = nullptr;
                    g.tile_cap = 0;
                }
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(g.d_tiles, g.tiles.data(), g.tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice,
                                    stream_);
            // stage 1 only writes V1, which the first real step rewrites
            auto launch = [&]() {
                return g.dtype == HJ_F64 ? launch_batch_stage_f64(g.d_tiles, (int)g.tiles.size(), d_insts_, 1, g.ndim,
                                                                  g.dyn, g.scheme, g.threads, g.smem, stream_)
                                         : launch_batch_stage_f32(g.d_tiles, (int)g.tiles.size(), d_insts_, 1, g.ndim,
                                                                  g.dyn, g.scheme, g.threads, g.smem, stream_);
            };
            if (e == cudaSuccess) e = launch();
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, stream_);
                e = launch();
                cudaEventRecord(e1, stream_);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float x = 0.f;
                if (e == cudaSuccess) cudaEventElapsedTime(&x, e0, e1);
                ms = std::min(ms, x);
            }
            launches += 3;
            ctx_->launches += 3;
            if (e != cudaSuccess) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(ctx_, e, "batch launch-shape timing");
    }
    apply(best.first, best.second);
    ctx_->batch_shape[key] = best;
    return HJ_OK;
}

hj_status Engine::rebuild_tiles() {
    bool any_graph = false;
    for (int l = 0; l < kLanes; ++l) any_graph = any_graph || exec_[l] != nullptr;
    if (any_graph) {
        HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
        drop_graphs();
    }
    tiles_total_ = 0;
    for (size_t gi = 0; gi < groups_.size(); ++gi) {
        Group& g = groups_[gi];
        g.tiles.clear();
        // by lane (the tiles of lanes >= l are a suffix), then largest instances
        // first: their many tiles start early, small ones fill the tail
        std::vector<int> order;
        for (int i = 0; i < max_slots_; ++i)
            if (slots[i].used && slots[i].active && slots[i].group == (int)gi) order.push_back(i);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            return slots[a].lane != slots[b].lane ? slots[a].lane < slots[b].lane : slots[a].N > slots[b].N;
        });
        g.smem = 0;
        for (int l = 0; l < kLanes; ++l) g.lane_off[l] = 0;
        for (int i : order) {
            append_tiles(slots[i], i, &g.tiles);
            // tiles of lanes above this instance's start after it
            for (int l = slots[i].lane + 1; l < kLanes; ++l) g.lane_off[l] = g.tiles.size();
            g.smem = std::max(g.smem, rows_smem(slots[i].G.n[0], slots[i].ty, slots[i].es));
        }
        tiles_total_ += (long long)g.tiles.size();
        if (g.tiles.empty()) continue;
        if (g.tiles.size() > g.tile_cap) {
            HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
            cudaFree(g.d_tiles);
            g.d_tiles = nullptr;
            g.tile_cap = g.tiles.size() * 2;
            HJ_CUDA(ctx_, cudaMalloc(&g.d_tiles, g.tile_cap * sizeof(BatchTile)));
        }
        HJ_CUDA(ctx_, cudaMemcpyAsync(g.d_tiles, g.tiles.data(), g.tiles.size() * sizeof(BatchTile),
                                      cudaMemcpyHostToDevice, stream_));
    }
    // the tile vectors must not change while the copies are pending
    HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
    tiles_dirty_ = false;
    return HJ_OK;
}

// One RK3 step of the instances of lane `lane` and above.
cudaError_t Engine::enqueue_step(cudaStream_t s, bool count, int lane, bool exact) {
    for (int stage = 1; stage <= 3; ++stage)
        for (const Group& g : groups_) {
            const size_t off = g.lane_off[lane];
            const size_t end = exact ? lane_end(g, lane) : g.tiles.size();
            if (end <= off) continue;
            const int nt = (int)(end - off);
            cudaError_t e = g.dtype == HJ_F64 ? launch_batch_stage_f64(g.d_tiles + off, nt, d_insts_, stage, g.ndim,
                                                                       g.dyn, g.scheme, g.threads, g.smem, s)
                                              : launch_batch_stage_f32(g.d_tiles + off, nt, d_insts_, stage, g.ndim,
                                                                       g.dyn, g.scheme, g.threads, g.smem, s);
            if (e != cudaSuccess) return e;
            if (count) {
                launches += 1;
                ctx_->launches += 1;
            }
        }
    if (count) {
        launches += 1;
        ctx_->launches += 1;
    }
    return launch_batch_advance(d_insts_, max_slots_, lane, exact ? lane : kLanes - 1, s);
}

long long Engine::dead_tiles() const {
    long long dead = 0;
    for (int i = 0; i < max_slots_; ++i) {
        const Slot& S = slots[i];
        if (S.used && S.active && S.k_host >= S.steps_total) dead += tiles_of(S);
    }
    return dead;
}

bool Engine::any_active() const {
    for (int i = 0; i < max_slots_; ++i)
        if (slots[i].used && slots[i].active && slots[i].k_host < slots[i].steps_total) return true;
    return false;
}

void Engine::done_slots(std::vector<int>* out) const {
    out->clear();
    for (int i = 0; i < max_slots_; ++i) {
        const Slot& S = slots[i];
        if (S.used && (!S.active || S.k_host >= S.steps_total)) out->push_back(i);
    }
}

hj_status Engine::run(int K) {
    NvtxRange range("batched steps");
    if (K <= 0 || !any_active()) return HJ_OK;
    if (tiles_dirty_) {
        hj_status st = rebuild_tiles();
        if (st) return st;
    }
    cudaError_t e = cudaSuccess;
    // Without lanes: K steps of every instance on stream_. With lanes: lane l
    // takes kLaneMult[l] * K steps of its own instances on its own stream,
    // all lanes forked from stream_ and joined back into it.
    if (multirate_) e = cudaEventRecord(fork_ev_, stream_);
    for (int l = 0; l < (multirate_ ? kLanes : 1) && e == cudaSuccess; ++l) {
        bool any = false;
        long long per_step = 1;
        for (const Group& g : groups_)
            if ((multirate_ ? lane_end(g, l) : g.tiles.size()) > g.lane_off[l]) {
                any = true;
                per_step += 3;
            }
        if (!any) continue;
        const int Kl = multirate_ ? kLaneMult[l] * K : K;
        cudaStream_t s = multirate_ ? lane_stream_[l] : stream_;
        if (multirate_) e = cudaStreamWaitEvent(s, fork_ev_, 0);
        if (e == cudaSuccess && Kl >= 2) {
            if (!exec_[l] || exec_K_[l] != Kl) {
                if (exec_[l]) {
                    cudaStreamSynchronize(stream_);
                    cudaGraphExecDestroy(exec_[l]);
                    exec_[l] = nullptr;
                }
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal);
                for (int k = 0; k < Kl && e == cudaSuccess; ++k) e = enqueue_step(cap_stream_, false, l, multirate_);
                cudaError_t e2 = cudaStreamEndCapture(cap_stream_, &graph);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec_[l], graph, 0);
                if (graph) cudaGraphDestroy(graph);
                exec_K_[l] = Kl;
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(exec_[l], s);
            if (e == cudaSuccess) {
                launches += per_step * Kl;
                ctx_->launches += per_step * Kl;
            }
        } else {
            for (int k = 0; k < Kl && e == cudaSuccess; ++k) e = enqueue_step(s, true, l, multirate_);
        }
        if (multirate_ && e == cudaSuccess) e = cudaEventRecord(lane_ev_[l], s);
        if (multirate_ && e == cudaSuccess) e = cudaStreamWaitEvent(stream_, lane_ev_[l], 0);
    }
    if (e != cudaSuccess) return cuda_fail(ctx_, e, "batched step launch");
    for (int i = 0; i < max_slots_; ++i) {
        Slot& S = slots[i];
        if (S.used && S.active) S.k_host = std::min(S.steps_total, S.k_host + (long long)K * kLaneMult[S.lane]);
    }
    // tiles of finished instances idle; rebuild once they are a quarter of the list
    if (4 * dead_tiles() >= tiles_total_ && tiles_total_ > 0) tiles_dirty_ = true;
    return HJ_OK;
}

hj_status Engine::retire(const std::vector<int>& which) {
    if (which.empty()) return HJ_OK;
    unsigned char* A = arena_.base();
    HJ_CUDA(ctx_, cudaMemsetAsync(d_words_, 0, 16 * (size_t)max_slots_, stream_));
    for (int si : which) {
        Slot& S = slots[si];
        const size_t bytes = (size_t)S.N * S.es;
        void* outbase = S.out_on_device ? S.out : (void*)(A + S.o_stage);
        for (int s = 1; s < S.prob.n_slices; ++s)  // repeated slice times repeat the slice
            if (S.S.slice_steps[s] > 0 && S.S.slice_steps[s] == S.S.slice_steps[s - 1])
                HJ_CUDA(ctx_, cudaMemcpyAsync(static_cast<char*>(outbase) + (size_t)s * bytes,
                                              static_cast<char*>(outbase) + (size_t)(s - 1) * bytes, bytes,
                                              cudaMemcpyDeviceToDevice, stream_));
        int* flag = reinterpret_cast<int*>(d_words_ + 2 * si + 1);
        cudaError_t e = S.dtype == HJ_F64
                            ? launch_nonfinite_f64(reinterpret_cast<const double*>(A + S.o_v), S.N, flag, stream_)
                            : launch_nonfinite_f32(reinterpret_cast<const float*>(A + S.o_v), S.N, flag, stream_);
        launches += 1;
        ctx_->launches += 1;
        if (e != cudaSuccess) return cuda_fail(ctx_, e, "final check launch");
        if (!S.out_on_device)
            HJ_CUDA(ctx_, cudaMemcpyAsync(S.out, outbase, (size_t)S.prob.n_slices * bytes, cudaMemcpyDeviceToHost,
                                          stream_));
    }
    std::vector<unsigned long long> words(2 * (size_t)max_slots_);
    HJ_CUDA(ctx_, cudaMemcpyAsync(words.data(), d_words_, words.size() * 8, cudaMemcpyDeviceToHost, stream_));
    HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
    for (int si : which) {
        Slot& S = slots[si];
        S.status = (words[2 * si + 1] & 0xffffffffull) ? HJ_ENONFINITE : HJ_OK;
        if (S.out_times)
            for (int s = 0; s < S.prob.n_slices; ++s) S.out_times[s] = S.S.slice_t[s];
        S.stats.steps = S.steps_total;
        S.stats.cell_updates = S.steps_total * S.N;
        S.stats.step_bound_inv = S.sbi;
        S.stats.t_final = S.S.slice_t.empty() ? 0.0 : S.S.slice_t[S.prob.n_slices - 1];
        arena_.release(S.off, S.bytes);
        S.used = false;
        S.active = false;
    }
    tiles_dirty_ = true;
    return HJ_OK;
}

hj_status Engine::drop(int si) {
    Slot& S = slots[si];
    if (!S.used) return HJ_OK;
    // park the device descriptor: no further steps for this slot
    BatchInst& D = h_insts_[si];
    D.steps_total = 0;
    D.k = 0;
    HJ_CUDA(ctx_, cudaMemcpyAsync(d_insts_ + si, &D, sizeof(BatchInst), cudaMemcpyHostToDevice, stream_));
    HJ_CUDA(ctx_, cudaStreamSynchronize(stream_));
    pending_.erase(std::remove(pending_.begin(), pending_.end(), si), pending_.end());
    arena_.release(S.off, S.bytes);
    S.used = false;
    S.active = false;
    tiles_dirty_ = true;
    return HJ_OK;
}

}  // namespace hj
