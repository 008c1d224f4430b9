// engine.h -- device-resident multi-instance stepping shared by the batched
// solve and the serving loop.
//
// An Engine owns one device arena (first-fit), a table of instance slots with
// their device descriptors (BatchInst), and per-group tile lists. Instances
// are admitted into free slots (arrays uploaded, CFL bound and non-finite
// check launched), activated together (one synchronisation: schedules and
// descriptors), advanced K RK3 steps at a time for all active instances (a
// captured CUDA graph replayed while the tile set is unchanged), and retired
// when their steps are done. Not thread-safe: one thread drives an Engine.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include "ctx.h"

namespace hj {

class Arena {
 public:
    void reset(unsigned char* base, size_t cap);
    bool alloc(size_t bytes, size_t* off);  // 256-byte aligned, first fit
    void release(size_t off, size_t bytes);
    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    unsigned char* base() const { return base_; }

 private:
    unsigned char* base_ = nullptr;
    size_t cap_ = 0, used_ = 0;
    std::vector<std::pair<size_t, size_t>> free_;  // (offset, size), sorted by offset
};

struct Slot {
    bool used = false, active = false;
    hj_problem prob;                 // copy; slice_times points into `times`
    std::vector<double> times;
    void* out = nullptr;
    bool out_on_device = true;
    double* out_times = nullptr;
    GridDev G;
    int dtype = 0;
    size_t es = 0;
    long long N = 0;
    bool angles = false;
    int group = -1;
    int lane = 0;                    // rate class (Engine::init with lanes)
    int ty = 1, tz = 1;
    Schedule S;
    double sbi = 0.0;
    long long steps_total = 0, k_host = 0;
    size_t off = 0, bytes = 0;       // the slot's arena block
    size_t o_v = 0, o_v1 = 0, o_v2 = 0, o_td = 0, o_tf = 0, o_stage = 0, o_ends = 0, o_end_slice = 0, o_end_dt = 0;
    std::vector<double> table;       // host angle tables, alive until activation
    std::vector<float> table_f;
    hj_stats stats{};
    hj_status status = HJ_OK;
    uint64_t tag = 0;                // caller's identifier (problem index or ticket)
};

class Engine {
 public:
    ~Engine();
    // Allocates the arena (arena_bytes), descriptor table and reduction words.
    // With multirate, instances are sorted by size into rate lanes: per K
    // steps of the largest, smaller ones take kLaneMult[lane] * K (a server's
    // small requests do not wait for the pace of its largest ones). The lanes'
    // step blocks run concurrently, each on its own stream.
    hj_status init(hj_ctx* ctx, cudaStream_t stream, int max_slots, size_t arena_bytes, bool multirate = false);
    void shutdown();

    // Whether the batched row kernel serves this problem.
    static bool eligible(const hj_problem* p);
    // Arena bytes one problem needs.
    static size_t footprint(const hj_problem* p, bool out_on_device);

    int free_slot() const;
    // Copies the problem into a free slot and enqueues its upload, CFL bound
    // and non-finite check. HJ_EBUSY: no slot or arena space right now.
    hj_status admit(const hj_problem* p, void* out, bool out_on_device, double* out_times, uint64_t tag,
                    int* slot_out);
    // Activates every admitted slot: one synchronisation, then schedules,
    // launch shapes and descriptors. Slots whose v0 is not finite come back in
    // `failed` with status HJ_ENONFINITE and are released.
    hj_status activate(std::vector<int>* failed);
    // K RK3 steps of every active slot.
    hj_status run(int K);
    bool any_active() const;
    // Active slots whose steps are all enqueued.
    void done_slots(std::vector<int>* out) const;
    // Finishes slots (duplicate slices, host copies, final checks), one
    // synchronisation; fills stats/out_times and releases them.
    hj_status retire(const std::vector<int>& slots);
    // Marks a slot finished now (cancellation) and releases it.
    hj_status drop(int slot);

    std::vector<Slot> slots;
    long long launches = 0;

 private:
    // Multipliers about inversely proportional to size, so that requests of
    // different sizes get similar shares of the GPU per tick (the smallest
    // lane's multiplier is capped: more steps of tiny launches only slow the
    // other lanes down). Chosen by measurement on the served workload.
    static constexpr int kLanes = 5;
    static constexpr int kLaneMult[kLanes] = {1, 2, 4, 8, 8};
    // lane of an instance of N nodes: the first l with N > kLaneNodes[l], else the last
    static constexpr long long kLaneNodes[kLanes - 1] = {1LL << 24, 1LL << 23, 1LL << 22, 1LL << 21};

    struct Group {
        int dtype = 0, ndim = 0, dyn = 0, scheme = HJ_WENO5;
        int threads = 0, tz_target = 8;
        size_t smem = 0;
        std::vector<BatchTile> tiles;     // instances by lane, then by size (largest first)
        size_t lane_off[kLanes] = {};  // first tile of an instance of lane >= l
        BatchTile* d_tiles = nullptr;
        size_t tile_cap = 0;
    };
    hj_status shape_group(Group& g, const std::vector<int>& members, const std::vector<int>& fresh);
    hj_status rebuild_tiles();
    // One RK3 step of the instances of lane `lane` (exact) or of lanes >= lane.
    cudaError_t enqueue_step(cudaStream_t s, bool count, int lane, bool exact);
    size_t lane_end(const Group& g, int lane) const { return lane + 1 < kLanes ? g.lane_off[lane + 1] : g.tiles.size(); }
    static int lane_of(long long nodes) {
        int l = 0;
        while (l < kLanes - 1 && nodes <= kLaneNodes[l]) ++l;
        return l;
    }
    long long dead_tiles() const;

    hj_ctx* ctx_ = nullptr;
    cudaStream_t stream_ = nullptr;
    cudaStream_t cap_stream_ = nullptr;
    int max_slots_ = 0;
    void* arena_mem_ = nullptr;
    Arena arena_;
    BatchInst* d_insts_ = nullptr;
    std::vector<BatchInst> h_insts_;
    unsigned long long* d_words_ = nullptr;  // per slot: CFL accumulator, non-finite flag
    std::vector<Group> groups_;
    bool tiles_dirty_ = true;
    long long tiles_total_ = 0;
    bool multirate_ = false;
    cudaGraphExec_t exec_[kLanes] = {};  // the step blocks of each lane
    int exec_K_[kLanes] = {};
    // multirate: each lane's step block runs on a stream of its own, forked
    // from and joined back into stream_, so that the lanes overlap on the GPU
    cudaStream_t lane_stream_[kLanes] = {};
    cudaEvent_t fork_ev_ = nullptr;
    cudaEvent_t lane_ev_[kLanes] = {};
    void drop_graphs();
    std::vector<int> pending_;
};

}  // namespace hj
