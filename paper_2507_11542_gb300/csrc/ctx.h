// ctx.h -- the library context and the helpers shared by the translation
// units behind the C ABI (hj_api.cu, batch.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/hj.h"
#include "hj_internal.h"

namespace hj {
class Engine;
}

struct hj_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    void* work[2] = {nullptr, nullptr};   // RK stage buffers (V1, V2)
    size_t work_bytes = 0;
    void* state = nullptr;                // the solve's own copy of V
    size_t state_bytes = 0;
    unsigned long long* aux = nullptr;    // [0] step-bound accumulator, [1] non-finite flag
    double* trig_d = nullptr;             // cos/sin tables of the dimension-2 coordinate
    float* trig_f = nullptr;
    size_t trig_cap = 0;
    double trig_key[3] = {0.0, 0.0, 0.0};  // (n, lo, dx) of the uploaded tables
    bool trig_valid = false;
    std::string last_error;
    long long launches = 0;
    int sm_count = 0;
    std::map<std::vector<long long>, hj::RowsCfg> rows_cache;  // tuned launch shapes per grid shape
    void* tune_buf = nullptr;                                 // output scratch of tuning launches
    size_t tune_bytes = 0;
    std::map<std::vector<long long>, std::pair<int, int>> batch_shape;  // (threads, planes per tile) per group kind
    hj::Engine* batch_engine = nullptr;                        // reused by hj_solve_batch
    size_t batch_engine_bytes = 0;
    int batch_engine_slots = 0;
};

namespace hj {

#define HJ_CUDA(ctx, call)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

hj_status fail(hj_ctx* ctx, hj_status st, const char* fmt, ...);
hj_status cuda_fail(hj_ctx* ctx, cudaError_t e, const char* what);
size_t elem_size(int dtype);
hj_status check_grid(hj_ctx* ctx, const hj_grid* g);
hj_status check_method(hj_ctx* ctx, const hj_grid* g, const hj_method* m);
hj_status check_solver_settings(hj_ctx* ctx, const hj_method* m);
hj_status check_slices(hj_ctx* ctx, int n_slices, const double* slice_times, double t0);
GridDev make_grid(const hj_grid* g, int extrap);
// WENO5 epsilon floor along dimension d, in raw-difference units
double weno_floor(const GridDev& g, int dtype, int d);
hj_status ensure(hj_ctx* ctx, void** p, size_t* cap, size_t bytes);
// cos/sin of the dimension-2 coordinate from the host math library: n cosines then n sines
void angle_table(const hj_grid* g, std::vector<double>* out);
hj_status step_bound(hj_ctx* ctx, const hj_grid* g, const hj_method* m, double* out);
hj_status nonfinite(hj_ctx* ctx, const void* v, long long n, int dtype, bool* bad);
// Whether the row-tiled kernel can take a grid (kernel: hj_method.kernel;
// HJ_KERNEL_NODE makes it false).
bool rows_eligible(const GridDev& G, int scheme, int dynamics, int dtype, int kernel = HJ_KERNEL_AUTO);
StageParams stage_params(hj_ctx* ctx, const GridDev& G, const hj_method* m, int dtype);
// Whether a method leaves the launch choices to the library (kernel AUTO, no tile override).
bool default_launch(const hj_method* m);

// The time schedule of one solve (Sec. 5, Listing 6): dt of every RK3 step,
// the number of steps completed at each slice, and the time reached there.
struct Schedule {
    std::vector<double> dts;
    std::vector<long long> slice_steps;
    std::vector<double> slice_t;
};
void plan_schedule(const hj_method* m, double step_bound_inv, int n_slices, const double* slice_times, double t0,
                   Schedule* s);

}  // namespace hj
