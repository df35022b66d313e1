// DOS post-steps on the GPU: the Hann-windowed transform of the correlation
// function (the analysis step Analyzer.calc_dos of Sec. 3.2.3) and the
// Jackson-kernel KPM density of states (Weisse et al., Rev. Mod. Phys. 78,
// 275 (2006), Eqs. 71 and 81). Both are direct sums, one block per energy,
// with exact twiddles from sincospi/cospi of rational multiples of pi.
#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

// D(E_j) = dt/(2 pi) sum_{m=-N}^{N-1} w_m C(t_m) exp(i E_j t_m),
// E_j t_m = pi (j - N) m / N, w_m = (1 + cos(pi m / N)) / 2, C(-t) = conj C(t).
__global__ void dos_hann_kernel(const double2 *corr, int N, double dt, double *energies,
                                double *dos)
{
    __shared__ double sre[256];
    const int j = blockIdx.x;
    const int64_t twoN = 2 * (int64_t)N;
    double acc = 0.0;
    for (int m = -N + (int)threadIdx.x; m <= N - 1; m += blockDim.x) {
        const int a = m < 0 ? -m : m;
        const double2 c = corr[a];
        const double cr = c.x, ci = m < 0 ? -c.y : c.y;
        const double w = 0.5 * (1.0 + cospi((double)m / (double)N));
        int64_t q = ((int64_t)(j - N) * (int64_t)m) % twoN;
        if (q < 0) q += twoN;
        double sn, cs;
        sincospi((double)q / (double)N, &sn, &cs);
        acc = fma(w, cr * cs - ci * sn, acc);           // real part only
    }
    sre[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sre[threadIdx.x] += sre[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double pi = 3.141592653589793238462643383279502884;
        dos[j] = sre[0] * dt / (2.0 * pi);
        energies[j] = (double)(j - N) * (pi / ((double)N * dt));
    }
}

// rho(x_j) = [g_0 mu_0 + 2 sum_{m>=1} g_m mu_m T_m(x_j)] / (pi sqrt(1 - x_j^2)),
// x_j = cos(pi (j + 1/2) / n_e), T_m(x_j) = cos(pi m (2j + 1) / (2 n_e)),
// g_m = [(M - m + 1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))] / (M + 1).
__global__ void kpm_dos_kernel(const double2 *mu, int M, int n_e, double rescale,
                               double *energies, double *rho)
{
    __shared__ double sre[256];
    const int j = blockIdx.x;
    const double cot1 = cospi(1.0 / (M + 1)) / sinpi(1.0 / (M + 1));
    const int64_t period = 4 * (int64_t)n_e;
    double acc = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double r = (double)m / (double)(M + 1);
        const double g = ((double)(M - m + 1) * cospi(r) + sinpi(r) * cot1) / (double)(M + 1);
        const int64_t q = ((int64_t)m * (2 * (int64_t)j + 1)) % period;
        const double tm = cospi((double)q / (2.0 * (double)n_e));
        acc = fma((m == 0 ? 1.0 : 2.0) * g * mu[m].x, tm, acc);
    }
    sre[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sre[threadIdx.x] += sre[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double pi = 3.141592653589793238462643383279502884;
        const double x = cospi((j + 0.5) / (double)n_e);
        const double sn = sinpi((j + 0.5) / (double)n_e);   // sqrt(1 - x^2), x = cos(theta)
        energies[j] = rescale * x;
        rho[j] = sre[0] / (pi * sn) / rescale;
    }
}

}  // namespace

cudaError_t launch_dos_hann(const double2 *corr, int n_steps, double dt, double *energies,
                            double *dos, cudaStream_t s)
{
    dos_hann_kernel<<<2 * n_steps, 256, 0, s>>>(corr, n_steps, dt, energies, dos);
    return cudaGetLastError();
}

cudaError_t launch_kpm_dos(const double2 *mu, int M, int n_e, double rescale, double *energies,
                           double *rho, cudaStream_t s)
{
    kpm_dos_kernel<<<n_e, 256, 0, s>>>(mu, M, n_e, rescale, energies, rho);
    return cudaGetLastError();
}

}  // namespace tbpm
