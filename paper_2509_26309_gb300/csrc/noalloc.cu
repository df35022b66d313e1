// tbpm_dos_corr_noalloc: the DOS correlation for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed, pre-planned
// device-memory budget (an embedding host application that owns every
// allocation), a plugin whose host forbids allocation after start-up, or
// code on a path where an allocation could stall or fail at the wrong moment.
// This entry point takes the Hamiltonian, the initial state and the output
// as device buffers the caller already owns, and keeps its own working
// vectors in one file-scope __device__ array of fixed size (kScratchBytes),
// which every GPU that loads the library holds until the process exits. It
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array's host-side name is only a stand-in for the device symbol, so the
// host never passes it to a kernel. The device address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call on each
// device, and again on the first call after that device's context has been
// replaced (cudaDeviceReset reloads the module, and the array may move): the
// cache is keyed by the context's process-unique id. That first call should
// therefore come before any stream capture. Every call waits on its stream for
// the term count (a 4-byte device-to-host read).
//
// The array is per process and per device. All calls of one process on one
// device share it, and it keeps the last call's contents: every call writes
// each scratch element before reading it (the coefficient kernel fills the
// coefficients and K, psi is copied from psi0, each Clenshaw term is written in
// full before it is read, and each step's dot partials are written before they
// are reduced), so nothing has to start at zero. Calls of one process that
// overlap on the GPU (other streams or host threads on the same device) race on
// the array; other processes have their own copy.
#include <cuda.h>      // CUcontext and CUresult only: the two driver calls are reached through the runtime

#include <cmath>
#include <mutex>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int64_t kMaxN = TBPM_NOALLOC_MAX_N;
constexpr int kNblk = 1024;                           // sweep blocks (fixed: deterministic dots)
// layout: coef[kMaxTerms] | K (padded to 16 B) | partials[kNblk] | psi[n] | b0[n] | b1[n]
constexpr size_t kCoefOff = 0;
constexpr size_t kKOff = kCoefOff + sizeof(double2) * kMaxTerms;
constexpr size_t kPartOff = kKOff + 256;
constexpr size_t kPsiOff = kPartOff + sizeof(double2) * kNblk;
constexpr size_t kVecBytes = sizeof(double2) * kMaxN;
constexpr size_t kScratchBytes = kPsiOff + 3 * kVecBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;                    // context the address belongs to (0: none yet)
    void *addr = nullptr;
};
ScratchAddr g_addr[64];                               // device address of g_scratch per device

// Clenshaw sweep on a plain CSR matrix with complex values (the operator is
// scaled in the kernel): y = a psi + beta (s H x) - z, s = 2/rescale. The kinds
// match cheb_sweep.cu: a = c[ia] - c[ib], beta = bscale (* c[ic]).
__global__ void __launch_bounds__(kBlock) csr_sweep(int64_t n, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ col,
                                                    const double2 *__restrict__ val, double s,
                                                    const double2 *__restrict__ x,
                                                    const double2 *psi, double2 *y,
                                                    const double2 *z, const double2 *coef,
                                                    int ia, int ib, int ic, double bscale,
                                                    const double2 *psi0, double2 *partials)
{
    __shared__ double2 red[kBlock / 32];
    const double2 ca = coef[ia];
    const double2 cb = ib >= 0 ? coef[ib] : make_double2(0.0, 0.0);
    const double ar = ca.x - cb.x, ai = ca.y - cb.y;
    double br = bscale, bi = 0.0;
    if (ic >= 0) { br = bscale * coef[ic].x; bi = bscale * coef[ic].y; }
    double dr = 0.0, di = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double hr = 0.0, hi = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            const double2 v = val[p], xv = x[col[p]];
            hr = fma(v.x, xv.x, fma(-v.y, xv.y, hr));
            hi = fma(v.x, xv.y, fma(v.y, xv.x, hi));
        }
        hr *= s; hi *= s;
        const double2 ps = psi[i];
        double yr = ar * ps.x - ai * ps.y + br * hr - bi * hi;
        double yi = ar * ps.y + ai * ps.x + br * hi + bi * hr;
        if (z) { const double2 zz = z[i]; yr -= zz.x; yi -= zz.y; }
        y[i] = make_double2(yr, yi);
        if (psi0) {
            const double2 q = psi0[i];
            dr = fma(q.x, yr, fma(q.y, yi, dr));
            di = fma(q.x, yi, fma(-q.y, yr, di));
        }
    }
    if (psi0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, o);
            di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(dr, di);
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 r = make_double2(0.0, 0.0);
            for (int w = 0; w < kBlock / 32; ++w) { r.x += red[w].x; r.y += red[w].y; }
            partials[blockIdx.x] = r;
        }
    }
}

__global__ void copy_state(int64_t n, const double2 *src, double2 *dst)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// <psi0|psi0> partials (the C(t_0) entry).
__global__ void __launch_bounds__(kBlock) self_dot(int64_t n, const double2 *a, double2 *partials)
{
    __shared__ double2 red[kBlock / 32];
    double dr = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 q = a[i];
        dr = fma(q.x, q.x, fma(q.y, q.y, dr));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dr += __shfl_xor_sync(0xffffffffu, dr, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(dr, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 r = make_double2(0.0, 0.0);
        for (int w = 0; w < kBlock / 32; ++w) r.x += red[w].x;
        partials[blockIdx.x] = r;
    }
}

// Process-unique id of the calling thread's current context (0 if there is
// none yet). The driver's cuCtxGetCurrent and cuCtxGetId are reached through
// the runtime's entry-point query, so the library needs no link to libcuda.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {                    // called under g_mu
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1) return e != cudaSuccess ? e : cudaErrorNotSupported;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !f2) return e != cudaSuccess ? e : cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) return cudaErrorUnknown;
    *id = 0;
    if (c && get_id(c, id) != CUDA_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

// Device address of g_scratch for the current device, looked up (with the
// device current) once per device and context.
cudaError_t scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    if (id == 0 || id != g_addr[dev].ctx_id || !g_addr[dev].addr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);      // also makes the device's context current
        if (e != cudaSuccess) return e;
        if ((e = current_context_id(&id)) != cudaSuccess) return e;
        if (id == 0) return cudaErrorDeviceUninitialized;
        g_addr[dev].ctx_id = id;
        g_addr[dev].addr = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev].addr);
    return cudaSuccess;
}

}  // namespace
}  // namespace tbpm

extern "C" int tbpm_dos_corr_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                     const double *val, double rescale, const double *psi0,
                                     double dt, int n_steps, double *corr, void *stream)
{
    using namespace tbpm;
    if (n < 1 || !row_ptr || !col || !val || !psi0 || !corr || n_steps < 0) return TBPM_ERR_ARG;
    if (!(rescale > 0.0) || !std::isfinite(rescale) || !(dt != 0.0) || !std::isfinite(dt))
        return TBPM_ERR_ARG;
    if (n > kMaxN) return TBPM_ERR_UNSUPPORTED;
    const double x = dt * rescale;
    if (!(std::fabs(x) <= 40.0)) return TBPM_ERR_ARG;
    cudaStream_t s = stream ? (cudaStream_t)stream : cudaStreamLegacy;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return TBPM_ERR_CUDA;
    double2 *coef = reinterpret_cast<double2 *>(base + kCoefOff);
    int *dK = reinterpret_cast<int *>(base + kKOff);
    double2 *part = reinterpret_cast<double2 *>(base + kPartOff);
    double2 *psi = reinterpret_cast<double2 *>(base + kPsiOff);
    double2 *bv[2] = {reinterpret_cast<double2 *>(base + kPsiOff + kVecBytes),
                      reinterpret_cast<double2 *>(base + kPsiOff + 2 * kVecBytes)};
    const double2 *p0 = reinterpret_cast<const double2 *>(psi0);
    const double2 *v = reinterpret_cast<const double2 *>(val);
    double2 *out = reinterpret_cast<double2 *>(corr);

    if (launch_bessel(x, 1e-12, coef, dK, s) != cudaSuccess) return TBPM_ERR_CUDA;
    int K = -1;
    if (cudaMemcpyAsync(&K, dK, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TBPM_ERR_CUDA;
    if (K < 1) return TBPM_ERR_ARG;
    K = K < 3 ? 3 : K;
    int grid = (int)((n + kBlock - 1) / kBlock);
    grid = grid > kNblk ? kNblk : grid;
    const double sc = 2.0 / rescale;
    copy_state<<<grid, kBlock, 0, s>>>(n, p0, psi);
    self_dot<<<grid, kBlock, 0, s>>>(n, p0, part);
    if (launch_reduce(part, 1, 1, grid, nullptr, 0, out, s) != cudaSuccess) return TBPM_ERR_CUDA;
    for (int step = 0; step < n_steps; ++step) {
        // b_{K-2} = c_{K-2} psi + c_{K-1} (2 H~) psi
        csr_sweep<<<grid, kBlock, 0, s>>>(n, row_ptr, col, v, sc, psi, psi, bv[0], nullptr, coef,
                                          K - 2, -1, K - 1, 1.0, nullptr, nullptr);
        if (K >= 4)   // b_{K-3} = (c_{K-3} - c_{K-1}) psi + 2 H~ b_{K-2}
            csr_sweep<<<grid, kBlock, 0, s>>>(n, row_ptr, col, v, sc, bv[0], psi, bv[1], nullptr, coef,
                                              K - 3, K - 1, -1, 1.0, nullptr, nullptr);
        for (int k = K - 4; k >= 1; --k) {   // b_k = c_k psi + 2 H~ b_{k+1} - b_{k+2}
            double2 *yk = bv[(K - 2 - k) & 1];
            csr_sweep<<<grid, kBlock, 0, s>>>(n, row_ptr, col, v, sc, bv[(K - 3 - k) & 1], psi, yk, yk,
                                              coef, k, -1, -1, 1.0, nullptr, nullptr);
        }
        // psi <- (c_0 - [K=3] c_2) psi + H~ b_1 - [K>=4] b_2, with <psi0|psi>
        csr_sweep<<<grid, kBlock, 0, s>>>(n, row_ptr, col, v, sc, bv[(K - 3) & 1], psi, psi,
                                          K >= 4 ? bv[(K - 4) & 1] : nullptr, coef, 0,
                                          K == 3 ? 2 : -1, -1, 0.5, p0, part);
        if (launch_reduce(part, 1, 1, grid, nullptr, step + 1, out, s) != cudaSuccess) return TBPM_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return TBPM_ERR_CUDA;
    return TBPM_OK;
}
