// tbpm_fp64_peak: measures the FP64 FMA issue rate of the current GPU, the
// ceiling of the FP64 Clenshaw sweeps (which GB300's narrow FP64 pipe bounds
// before HBM does). A measurement helper of the benchmark, not a step of the
// method.
//
// Every thread runs CH independent FMA chains (x <- x * a + b) for `iters`
// rounds, so the pipe always has independent work. Three launch shapes are
// timed and the fastest is kept: 8 chains with 1024 or 2048 threads per SM,
// and 16 chains with 1024. The chains' final values are summed into one store
// that is taken only if the sum is exactly zero (it never is for the inputs
// used), so the compiler keeps every FMA. FP64 operations counted: 2 per FMA.
#include <cmath>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kPeakBlock = 256;

template <int CH>
__global__ void __launch_bounds__(kPeakBlock) dfma_kernel(int iters, double a, double b, double *sink)
{
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
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
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TBPM_OK;
    double best_tf = 0.0, best_ms = 0.0;
    const int max_grid = sms * (2048 / kPeakBlock);
    if (cudaMalloc(&sink, sizeof(double) * max_grid) != cudaSuccess) return TBPM_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TBPM_ERR_CUDA;
    // a = 1 - 2^-20 and b = 2^-20 keep x near 1 (the fixed point), so no value
    // overflows, underflows or becomes subnormal
    const double a = 1.0 - std::ldexp(1.0, -20), b = std::ldexp(1.0, -20);
    // (chains, threads per SM)
    const int shapes[3][2] = {{8, 1024}, {8, 2048}, {16, 1024}};
    for (int sh = 0; sh < 3 && !rc; ++sh) {
        const int ch = shapes[sh][0], grid = sms * (shapes[sh][1] / kPeakBlock);
        auto launch = [&]() {
            if (ch == 8) dfma_kernel<8><<<grid, kPeakBlock>>>(iters, a, b, sink);
            else dfma_kernel<16><<<grid, kPeakBlock>>>(iters, a, b, sink);
        };
        launch();                                                    // warm-up
        if (cudaDeviceSynchronize() != cudaSuccess) { rc = TBPM_ERR_CUDA; break; }
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(e0);
            launch();
            cudaEventRecord(e1);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = TBPM_ERR_CUDA;
                break;
            }
            const double tf = 2.0 * ch * (double)iters * grid * kPeakBlock / (ms * 1e-3) / 1e12;
            if (tf > best_tf) { best_tf = tf; best_ms = ms; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    *tflops = best_tf;
    if (ms_per_launch) *ms_per_launch = best_ms;
    return TBPM_OK;
}
