// Test probe: evaluates the library's FP64 reciprocal (rcp_newton in
// weno_iface.cuh, the hardware estimate refined by two Newton-Raphson steps)
// on device arrays, so that a test can hold it against 1/x.
#include <cuda_runtime.h>

#include "weno_iface.cuh"

namespace {
__global__ void rcp_probe_kernel(const double* x, double* r, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = hj::rcp_newton(x[i]);
}
}  // namespace

extern "C" int rcp_probe(const double* x, double* r, long long n) {
    if (n <= 0) return 0;
    rcp_probe_kernel<<<(unsigned)((n + 255) / 256), 256>>>(x, r, n);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
