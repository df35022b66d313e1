// tbpm_fp64_peak: measures the FP64 FMA issue rate of the current GPU, the
// ceiling of the FP64 Clenshaw sweeps (which GB300's narrow FP64 pipe bounds
// before HBM does). A measurement helper of the benchmark, not a step of the
// method.
//
// Every thread runs kChains independent FMA chains (x <- x * a + b) for `iters`
// rounds, so the pipe always has independent work; the grid holds 1024
// threads on every SM. The chains' final values are summed into one store
// that is taken only if the sum is exactly zero (it never is for the inputs
// used), so the compiler keeps every FMA. FP64 operations counted: 2 per FMA.
#include <cmath>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

__global__ void __launch_bounds__(kPeakBlock) dfma_kernel(int iters, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 0.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace tbpm

extern "C" int tbpm_fp64_peak(int device, int iters, int reps, double *tflops, double *ms_per_launch)
{
    using namespace tbpm;
    if (!tflops || iters < 1 || reps < 1 || iters > (1 << 26)) return TBPM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return TBPM_ERR_NO_DEVICE;
    if (device < 0) {
        if (cudaGetDevice(&device) != cudaSuccess) return TBPM_ERR_CUDA;
    }
    if (device >= ndev || cudaSetDevice(device) != cudaSuccess) return TBPM_ERR_ARG;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TBPM_ERR_CUDA;
    const int grid = sms * (1024 / kPeakBlock);
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TBPM_OK;
    float best = 1e30f;
    if (cudaMalloc(&sink, sizeof(double) * grid) != cudaSuccess) return TBPM_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TBPM_ERR_CUDA;
    // a = 1 - 2^-20 and b = 2^-20 keep x near 1 (the fixed point), so no value
    // overflows, underflows or becomes subnormal
    const double a = 1.0 - std::ldexp(1.0, -20), b = std::ldexp(1.0, -20);
    if (!rc) {
        dfma_kernel<<<grid, kPeakBlock>>>(iters, a, b, sink);         // warm-up
        if (cudaDeviceSynchronize() != cudaSuccess) rc = TBPM_ERR_CUDA;
    }
    for (int r = 0; r < reps && !rc; ++r) {
        cudaEventRecord(e0);
        dfma_kernel<<<grid, kPeakBlock>>>(iters, a, b, sink);
        cudaEventRecord(e1);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = TBPM_ERR_CUDA;
            break;
        }
        if (ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    const double flops = 2.0 * kChains * (double)iters * grid * kPeakBlock;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_per_launch) *ms_per_launch = best;
    return TBPM_OK;
}
