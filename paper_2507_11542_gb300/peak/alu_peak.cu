// alu_peak.cu -- measured ceilings of the two pipes the level-set stage is
// bound by: FP32 FFMA and FP64 DFMA throughput of this GPU, for the roofline
// the benchmark reports (an FMA counts two flops). Built as its own library
// (libhj_peak.so); the level-set library does not use it.
//
// Each thread runs kChains independent FMA chains v <- v * a + b, so that the
// pipe, not the latency of one chain, sets the rate; a (slightly below one)
// and b keep the values finite. The sum of the chains is stored only if it
// equals an impossible value, so the work cannot be optimised away and the
// kernel writes nothing.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop(T* sink, int iters, T a, T b) {
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = T(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == T(-1234567.0)) sink[blockIdx.x] = s;
}

template <typename T>
int measure(int device, int blocks_per_sm, int iters, int reps, double* tflops, double* ms_out) {
    if (cudaSetDevice(device) != cudaSuccess) return 1;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
    const int blocks = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 1;
    float best = 1e30f;
    int rc = 0;
    for (int r = 0; r <= reps && rc == 0; ++r) {  // r = 0: warm-up
        cudaEventRecord(e0);
        fma_loop<T><<<blocks, kThreads>>>(nullptr, iters, T(0.9999999), T(1e-7));
        cudaEventRecord(e1);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) rc = 2;
        float ms = 0.f;
        if (rc == 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double fmas = (double)blocks * kThreads * (double)iters * kUnroll * kChains;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    *ms_out = best;
    return 0;
}

}  // namespace

// dtype 1: FP32 (FFMA), 2: FP64 (DFMA). Returns 0 on success, writes the best
// of `reps` timed launches (TFLOP/s and its duration in ms).
extern "C" int hj_alu_peak(int device, int dtype, int reps, double* tflops, double* ms) {
    if (!tflops || !ms || reps < 1) return 1;
    if (dtype == 1) return measure<float>(device, 8, 4096, reps, tflops, ms);
    if (dtype == 2) return measure<double>(device, 8, 64, reps, tflops, ms);
    return 1;
}
