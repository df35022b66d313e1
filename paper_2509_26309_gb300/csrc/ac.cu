// AC (optical) conductivity by the current-current correlation of TBPM, one
// of the solver capabilities of Sec. 1 and Sec. 4.2.2, with the current
// operators given as sparse matrices as TBPM solvers take them (Sec. 2.3.4).
// The formulation is the standard TBPM one (hbar = e = 1):
//   C_ab(t) = <phi2(t)| J_a |phi1_b(t)>,  phi2(t) = e^{-iHt} f(H) phi,
//   phi1_b(t) = e^{-iHt} [1 - f(H)] J_b phi,
// f the Fermi-Dirac function applied as a Chebyshev series of H~ whose
// coefficients come from Chebyshev-Gauss quadrature on 2 * kFermiCap nodes.
// This file holds the kernels that are not Chebyshev sweeps: the Fermi
// coefficients, the current-operator product, the fused J_a product + four
// dots per time step, the layout change of the result and the windowed
// transform to Re sigma(w). The sweeps are those of cheb_sweep.cu.
#include "tbpm_internal.cuh"
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

__device__ __forceinline__ double fermi_occ(double beta, double mu, double e)
{
    const double z = beta * (e - mu);
    if (z > 0.0) {
        const double q = exp(-z);
        return q / (1.0 + q);
    }
    return 1.0 / (1.0 + exp(z));
}

// fj[j] = f(rescale * cos(pi (2j + 1) / (2M))), j < M
__global__ void fermi_nodes_kernel(double beta, double mu, double rescale, int M, double *fj)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) fj[j] = fermi_occ(beta, mu, rescale * cospi((double)(2 * j + 1) / (2.0 * (double)M)));
}

// One block per k < kcap: a_k = (2 - delta_k0)/M sum_j fj[j] cos(k (2j+1) pi / (2M)).
// The phase k (2j+1) is reduced modulo 4M in integers, so cospi sees an exact
// argument in [0, 2). fc[k] = a_k, gc[k] = delta_k0 - a_k (the series of 1 - f);
// kmax = 1 + the largest k with |a_k| >= tol.
__global__ void __launch_bounds__(256) fermi_coef_kernel(const double *fj, int M, double tol, double2 *fc,
                                                         double2 *gc, int *kmax)
{
    __shared__ double sm[256];
    const int k = blockIdx.x;
    const int64_t period = 4 * (int64_t)M;
    double s = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const int64_t ph = ((int64_t)k * (2 * j + 1)) % period;
        s = fma(fj[j], cospi((double)ph / (2.0 * (double)M)), s);
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double a = (k == 0 ? 1.0 : 2.0) * sm[0] / (double)M;
        fc[k] = make_double2(a, 0.0);
        gc[k] = make_double2((k == 0 ? 1.0 : 0.0) - a, 0.0);
        if (fabs(a) >= tol) atomicMax(kmax, k + 1);
    }
}

// y = J x for a SELL-32 current operator (complex values, no separate diagonal).
// One warp per 32-row slice, grid-stride.
__global__ void __launch_bounds__(256) jmul_kernel(CurrentOp j, const double2 *__restrict__ vals,
                                                   const double2 *__restrict__ x, double2 *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < j.nslices; s += nw) {
        const int64_t off = j.slice_off[s];
        const int w = (int)((j.slice_off[s + 1] - off) >> 5);
        double ar = 0.0, ai = 0.0;
        for (int q = 0; q < w; ++q) {
            const int64_t e = off + 32 * q + lane;
            const int c = __ldg(j.cols + e);
            const double2 v = __ldg(vals + e);
            const double2 xv = __ldg(x + c);
            ar = fma(v.x, xv.x, fma(-v.y, xv.y, ar));
            ai = fma(v.x, xv.y, fma(v.y, xv.x, ai));
        }
        y[(s << 5) + lane] = make_double2(ar, ai);
    }
}

// Per row i: u_a = (J_a phi2)_i for a = x, y, then conj(u_a) phi1_b[i] for
// (a, b) = xx, xy, yx, yy, accumulated per lane over the warp's slices and
// reduced once per warp into partials[(slot * 4 + q) * W + warp], W = warps
// in the grid (fixed per context). J_a is Hermitian, so sum_i conj(u_a,i)
// phi1_b,i = <phi2|J_a|phi1_b>. IMAG: every value of J_a is i times a real
// number (the current operators of a lattice with real hoppings, i [H, x_a]),
// so each product takes two FP64 FMAs instead of four, with the same result.
template <bool IMAG>
__global__ void __launch_bounds__(kBlockB1) jdot_kernel(CurrentOp j, const double2 *__restrict__ phi2,
                                                        const double2 *__restrict__ p1x,
                                                        const double2 *__restrict__ p1y, double2 *partials,
                                                        int slot)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t s = warp; s < j.nslices; s += nw) {
        const int64_t off = j.slice_off[s];
        const int w = (int)((j.slice_off[s + 1] - off) >> 5);
        double xr = 0.0, xi = 0.0, yr = 0.0, yi = 0.0;
        for (int q = 0; q < w; ++q) {
            const int64_t e = off + 32 * q + lane;
            const int c = __ldg(j.cols + e);
            const double2 vx = __ldg(j.jx + e);
            const double2 vy = __ldg(j.jy + e);
            const double2 p = __ldg(phi2 + c);
            if (IMAG) {
                xr = fma(-vx.y, p.y, xr);
                xi = fma(vx.y, p.x, xi);
                yr = fma(-vy.y, p.y, yr);
                yi = fma(vy.y, p.x, yi);
            } else {
                xr = fma(vx.x, p.x, fma(-vx.y, p.y, xr));
                xi = fma(vx.x, p.y, fma(vx.y, p.x, xi));
                yr = fma(vy.x, p.x, fma(-vy.y, p.y, yr));
                yi = fma(vy.x, p.y, fma(vy.y, p.x, yi));
            }
        }
        const int64_t row = (s << 5) + lane;
        const double2 bx = p1x[row], by = p1y[row];
        // conj(u) b = (ur br + ui bi) + i (ur bi - ui br)
        acc[0] = fma(xr, bx.x, fma(xi, bx.y, acc[0]));
        acc[1] = fma(xr, bx.y, fma(-xi, bx.x, acc[1]));
        acc[2] = fma(xr, by.x, fma(xi, by.y, acc[2]));
        acc[3] = fma(xr, by.y, fma(-xi, by.x, acc[3]));
        acc[4] = fma(yr, bx.x, fma(yi, bx.y, acc[4]));
        acc[5] = fma(yr, bx.y, fma(-yi, bx.x, acc[5]));
        acc[6] = fma(yr, by.x, fma(yi, by.y, acc[6]));
        acc[7] = fma(yr, by.y, fma(-yi, by.x, acc[7]));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            partials[((int64_t)slot * 4 + q) * nw + warp] = make_double2(acc[2 * q], acc[2 * q + 1]);
}

// dst[q * (n + 1) + m] = src[m * 4 + q]
__global__ void ac_transpose_kernel(const double2 *src, int64_t np1, double2 *dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * np1) return;
    const int64_t q = i / np1, m = i - q * np1;
    dst[i] = src[m * 4 + q];
}

// One block per (correlation q, frequency j):
//   sigma[q][j] = (exp(-beta w) - 1)/(w s) sum_{m<N} dt w_m sin(w t_m) 2 Im C_q(t_m),
//   w_m = (1 + cos(pi m / N)) / 2; sigma = 0 at w = 0.
__global__ void __launch_bounds__(256) ac_cond_kernel(const double2 *corr, int N, double dt, double beta,
                                                      double area, const double *omegas, int n_w, double *sigma)
{
    __shared__ double sm[256];
    const int q = blockIdx.x / n_w, jw = blockIdx.x - q * n_w;
    const double w = omegas[jw];
    const double2 *c = corr + (int64_t)q * (N + 1);
    double acc = 0.0;
    if (w != 0.0)
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            const double win = 0.5 * (1.0 + cospi((double)m / (double)N));
            acc = fma(win * sin(w * (double)m * dt), 2.0 * c[m].y, acc);
        }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        sigma[(int64_t)q * n_w + jw] = w == 0.0 ? 0.0 : (exp(-beta * w) - 1.0) / (w * area) * dt * sm[0];
}

}  // namespace

cudaError_t launch_fermi_coeffs(double beta, double mu, double rescale, double tol, int kcap, double *fj,
                                double2 *fc, double2 *gc, int *kmax, cudaStream_t s)
{
    const int M = 2 * kcap;
    cudaError_t e = cudaMemsetAsync(kmax, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    fermi_nodes_kernel<<<(M + 255) / 256, 256, 0, s>>>(beta, mu, rescale, M, fj);
    fermi_coef_kernel<<<kcap, 256, 0, s>>>(fj, M, tol, fc, gc, kmax);
    return cudaGetLastError();
}

cudaError_t launch_jmul(const CurrentOp &j, const double2 *vals, const void *x, void *y, int grid, cudaStream_t s)
{
    jmul_kernel<<<grid, 256, 0, s>>>(j, vals, reinterpret_cast<const double2 *>(x), reinterpret_cast<double2 *>(y));
    return cudaGetLastError();
}

cudaError_t launch_jdot(const CurrentOp &j, const void *phi2, const void *p1x, const void *p1y,
                        double2 *partials, int slot, int grid, cudaStream_t s)
{
    if (j.imag)
        jdot_kernel<true><<<grid, kBlockB1, 0, s>>>(j, reinterpret_cast<const double2 *>(phi2),
                                                    reinterpret_cast<const double2 *>(p1x),
                                                    reinterpret_cast<const double2 *>(p1y), partials, slot);
    else
        jdot_kernel<false><<<grid, kBlockB1, 0, s>>>(j, reinterpret_cast<const double2 *>(phi2),
                                                     reinterpret_cast<const double2 *>(p1x),
                                                     reinterpret_cast<const double2 *>(p1y), partials, slot);
    return cudaGetLastError();
}

cudaError_t launch_ac_transpose(const double2 *src, int64_t np1, double2 *dst, cudaStream_t s)
{
    const int64_t n = 4 * np1;
    ac_transpose_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, np1, dst);
    return cudaGetLastError();
}

cudaError_t launch_ac_cond(const double2 *corr, int n_steps, double dt, double beta, double area,
                           const double *omegas, int n_w, double *sigma, cudaStream_t s)
{
    ac_cond_kernel<<<4 * n_w, 256, 0, s>>>(corr, n_steps, dt, beta, area, omegas, n_w, sigma);
    return cudaGetLastError();
}

}  // namespace tbpm
