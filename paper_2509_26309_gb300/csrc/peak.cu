// tbpm_fp64_peak: measures the FP64 FMA issue rate of the current GPU, the
// ceiling of the FP64 Clenshaw sweeps (which GB300's narrow FP64 pipe bounds
// before HBM does). A measurement helper of the benchmark, not a step of the
// method.
//
// Every thread runs CH independent chains of one FP64 instruction form for
// `iters` rounds, so the pipe always has independent work:
//   form 0: x <- fma(x, a, b), a and b kernel parameters
//   form 1: x <- fma(x, a, b), a and b loaded into registers from memory
//   form 2: x <- x * a          form 3: x <- x + b
// with a = 1 - 2^-20 and b = 2^-20, so that no value overflows, underflows or
// becomes subnormal. Each form runs at two launch shapes (8 chains with 1024
// and 2048 threads per SM) and the fastest launch of all is kept. The chains'
// final values are summed into one store that is taken only if the sum is
// exactly zero (it never is for these inputs), so the compiler keeps every
// instruction. Every FP64 instruction counts as 2 operations (one issue slot
// of the FP64 pipe), as the sweeps' roofline counts them.
#include <cmath>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kPeakBlock = 256;
constexpr int kPeakChains = 8;

template <int FORM>
__global__ void __launch_bounds__(kPeakBlock) fp64_probe_kernel(int iters, double a, double b, const double *ab,
                                                               double *sink)
{
    double x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    double ra = a, rb = b;
    if (FORM == 1) {
        ra = ab[0];
        rb = ab[1];
    }
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) {
            if (FORM == 0) x[c] = fma(x[c], a, b);
            else if (FORM == 1) x[c] = fma(x[c], ra, rb);
            else if (FORM == 2) x[c] = x[c] * ra;
            else x[c] = x[c] + rb;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
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
    // a = 1 - 2^-20 and b = 2^-20 keep every chain near 1
    const double a = 1.0 - std::ldexp(1.0, -20), b = std::ldexp(1.0, -20);
    const double ab_host[2] = {a, b};
    if (cudaMalloc(&sink, sizeof(double) * (max_grid + 2)) != cudaSuccess) return TBPM_ERR_OOM;
    double *ab = sink + max_grid;
    if (cudaMemcpy(ab, ab_host, sizeof(ab_host), cudaMemcpyHostToDevice) != cudaSuccess) rc = TBPM_ERR_CUDA;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = TBPM_ERR_CUDA;
    for (int form = 0; form < 4 && !rc; ++form)
        for (int tps : {1024, 2048}) {
            const int grid = sms * (tps / kPeakBlock);
            auto launch = [&]() {
                if (form == 0) fp64_probe_kernel<0><<<grid, kPeakBlock>>>(iters, a, b, ab, sink);
                else if (form == 1) fp64_probe_kernel<1><<<grid, kPeakBlock>>>(iters, a, b, ab, sink);
                else if (form == 2) fp64_probe_kernel<2><<<grid, kPeakBlock>>>(iters, a, b, ab, sink);
                else fp64_probe_kernel<3><<<grid, kPeakBlock>>>(iters, a, b, ab, sink);
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
                const double tf = 2.0 * kPeakChains * (double)iters * grid * kPeakBlock / (ms * 1e-3) / 1e12;
                if (tf > best_tf) { best_tf = tf; best_ms = ms; }
            }
            if (rc) break;
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    *tflops = best_tf;
    if (ms_per_launch) *ms_per_launch = best_ms;
    return TBPM_OK;
}
