// Small kernels around the sweeps: Chebyshev coefficients, dots, deterministic
// reductions, state loading and the KPM moment assembly.
#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

// c_k = (2 - delta_k0) (-i)^k J_k(x) for k < kMaxTerms, and K = the first
// k > |x| with |J_k(x)| < tol (the cutoff of the series; the coefficient
// array of the propagation listings of Sec. 2.2.1).
//
// J_k(|x|) comes from Miller's backward recurrence (J.C.P. Miller 1952; the
// method of Abramowitz & Stegun 9.12, Example 1): start far above the wanted
// orders with J_{m+1} = 0, J_m = tiny, run J_{k-1} = (2k/x) J_k - J_{k+1}
// down to k = 0, and normalise with the identity J_0 + 2 sum_{k>=1} J_{2k} = 1
// (A&S 9.1.46). The recurrence is stable downwards and the normalisation
// removes the arbitrary start value. Whenever the running values exceed 1e200
// they and everything stored so far are scaled by 1e-200. Below |x| = 0.5 the
// power series J_k(x) = sum_m (-1)^m (x/2)^{2m+k} / (m! (m+k)!) (A&S 9.1.10)
// converges in a few terms without cancellation and is used instead, which
// also keeps the recurrence ratio 2k/x bounded. J_k(-x) = (-1)^k J_k(x)
// (A&S 9.1.5).
__global__ void bessel_kernel(double x, double tol, double2 *coef, int *K_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double ax = fabs(x);
    double j[kMaxTerms];
    if (ax < 0.5) {
        const double h = 0.5 * ax, h2 = h * h;
        double lead = 1.0;                               // (x/2)^k / k!
        for (int k = 0; k < kMaxTerms; ++k) {
            if (k > 0) lead *= h / k;
            double term = lead, sum = lead;
            for (int q = 1; q < 30 && term != 0.0; ++q) {
                term *= -h2 / ((double)q * (double)(q + k));
                sum += term;
            }
            j[k] = sum;
        }
    } else {
        int m = kMaxTerms + 30 + 2 * (int)ceil(ax);
        m += (m & 1);                                    // even start order
        double jp1 = 0.0, jk = 1e-300, norm = 0.0;
        for (int k = 0; k < kMaxTerms; ++k) j[k] = 0.0;
        for (int k = m; k >= 1; --k) {
            // jk = J_k, jp1 = J_{k+1}  ->  J_{k-1}
            const double jm1 = (2.0 * k / ax) * jk - jp1;
            if (k < kMaxTerms) j[k] = jk;
            if ((k & 1) == 0) norm += 2.0 * jk;
            jp1 = jk;
            jk = jm1;
            if (fabs(jk) > 1e200) {
                jk *= 1e-200; jp1 *= 1e-200; norm *= 1e-200;
                for (int q = 0; q < kMaxTerms; ++q) j[q] *= 1e-200;
            }
        }
        j[0] = jk;
        norm += jk;
        const double inv = 1.0 / norm;
        for (int k = 0; k < kMaxTerms; ++k) j[k] *= inv;
    }
    int K = -1;
    for (int k = 1; k < kMaxTerms; ++k) {
        if ((double)k > ax && fabs(j[k]) < tol) { K = k; break; }
    }
    for (int k = 0; k < kMaxTerms; ++k) {
        double v = j[k];
        if (x < 0.0 && (k & 1)) v = -v;
        const double f = (k == 0) ? v : 2.0 * v;
        double2 c;
        switch (k & 3) {                                  // (-i)^k
        case 0: c = make_double2(f, 0.0); break;
        case 1: c = make_double2(0.0, -f); break;
        case 2: c = make_double2(-f, 0.0); break;
        default: c = make_double2(0.0, f); break;
        }
        coef[k] = c;
    }
    *K_out = K;
}

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

__device__ __forceinline__ double2 block_sum2(double re, double im, double2 *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sm[w] = make_double2(re, im);
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { r.x += sm[i].x; r.y += sm[i].y; }
    __syncthreads();
    return r;
}

// <a|b> over 32-row slices (grid-stride, one warp per slice at a time).
// per_slice: one fixed-butterfly partial per slice, partials[s] (instances of
// a batch stay apart); otherwise per-lane sums over the warp's slices and one
// partial per warp, partials[warp] (as the single-instance final sweep).
template <typename R>
__global__ void __launch_bounds__(kBlockB1) dot_slices(const void *a_, const void *b_, int64_t nslices,
                                                     double2 *partials, bool per_slice)
{
    typedef typename V2<R>::T V;
    const V *a = reinterpret_cast<const V *>(a_);
    const V *b = reinterpret_cast<const V *>(b_);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double wr = 0.0, wi = 0.0;
    for (int64_t s = warp; s < nslices; s += nwarps) {
        const V p = a[s * 32 + lane], q = b[s * 32 + lane];
        const double pr = p.x, pi = p.y, qr = q.x, qi = q.y;
        if (per_slice) {
            double re = fma(pr, qr, pi * qi), im = fma(pr, qi, -pi * qr);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == 0) partials[s] = make_double2(re, im);
        } else {
            wr = fma(pr, qr, fma(pi, qi, wr));
            wi = fma(pr, qi, fma(-pi, qr, wi));
        }
    }
    if (!per_slice) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wr += __shfl_xor_sync(0xffffffffu, wr, o);
            wi += __shfl_xor_sync(0xffffffffu, wi, o);
        }
        if (lane == 0) partials[warp] = make_double2(wr, wi);
    }
}

// Segmented fixed-order sums of per-slice partials laid out [nslot][nterm][nslices]:
//   out[g * ld + (base + offset + d) * nterm + q] = sum_{s in segment g} P[(d * nterm + q) * nslices + s],
// segment g = [seg_off[g], seg_off[g+1]) (one segment [0, nslices) if seg_off is
// null), base = *counter (0 if null). One block per (d, q, g).
__global__ void __launch_bounds__(256) reduce_seg_kernel(const double2 *partials, int nslot, int nterm,
                                                         int64_t nslices, const int64_t *seg_off,
                                                         int nseg, const int *counter, int offset,
                                                         double2 *out, int64_t ld)
{
    __shared__ double sr[256], si[256];
    const int idx = blockIdx.x;
    const int g = idx % nseg, dq = idx / nseg;
    const int d = dq / nterm, q = dq - d * nterm;
    if (d >= nslot) return;
    const int64_t lo = seg_off ? seg_off[g] : 0, hi = seg_off ? seg_off[g + 1] : nslices;
    const double2 *p = partials + ((int64_t)d * nterm + q) * nslices;
    double re = 0.0, im = 0.0;
    for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) { re += p[s].x; im += p[s].y; }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { sr[threadIdx.x] += sr[threadIdx.x + o]; si[threadIdx.x] += si[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int base = counter ? *counter : 0;
        out[(int64_t)g * ld + (int64_t)(base + offset + d) * nterm + q] = make_double2(sr[0], si[0]);
    }
}

// scale[g] = 1/sqrt(sum_{s in segment g} norm[s].x): one block per segment.
__global__ void __launch_bounds__(256) renorm_seg_kernel(const double2 *norm, int64_t nslices,
                                                         const int64_t *seg_off, double *scale)
{
    __shared__ double sm[256];
    const int g = blockIdx.x;
    const int64_t lo = seg_off ? seg_off[g] : 0, hi = seg_off ? seg_off[g + 1] : nslices;
    double v = 0.0;
    for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) v += norm[s].x;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) scale[g] = sm[0] > 0.0 ? 1.0 / sqrt(sm[0]) : 1.0;
}

// Column `col` of an interleaved [n_pad][B] state buffer, scaled by scale[col]
// (or 1), as FP64 complex [n] (the inverse of load_column).
template <typename R>
__global__ void store_column_kernel(const void *src_, int64_t n, int B, int col, const double *scale,
                                    double2 *dst)
{
    typedef typename V2<R>::T V;
    const V *src = reinterpret_cast<const V *>(src_);
    const double sc = scale ? scale[col] : 1.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const V v = src[i * B + col];
        dst[i] = make_double2(sc * (double)v.x, sc * (double)v.y);
    }
}

// Quasi-eigenstate accumulation after time step m = *counter + delta + 1:
//   Q_e += pre * w_m * exp(i E_e t_m) * psi,  t_m = m h,  w_m = (1 + cos(pi m / N)) / 2,
// Q: FP64 complex [n_e][n_pad]. The phases are formed once per block.
template <typename R>
__global__ void qe_accumulate_kernel(const void *psi_, double2 *Q, const double *energies, int n_e,
                                     int64_t n_pad, const int *counter, int delta, double h, int N,
                                     double pre)
{
    typedef typename V2<R>::T V;
    extern __shared__ double2 ph[];
    const int m = (counter ? *counter : 0) + delta + 1;
    const double w = 0.5 * (1.0 + cospi((double)m / (double)N));
    for (int e = threadIdx.x; e < n_e; e += blockDim.x) {
        double sn, cs;
        sincos(energies[e] * (double)m * h, &sn, &cs);
        ph[e] = make_double2(pre * w * cs, pre * w * sn);
    }
    __syncthreads();
    const V *psi = reinterpret_cast<const V *>(psi_);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
        const V v = psi[i];
        const double vr = (double)v.x, vi = (double)v.y;
        // four energies at a time: their loads issue together (the stores of
        // one energy would otherwise hold back the loads of the next)
        int e = 0;
        for (; e + 4 <= n_e; e += 4) {
            double2 q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = Q[(int64_t)(e + j) * n_pad + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                q[j].x = fma(ph[e + j].x, vr, fma(-ph[e + j].y, vi, q[j].x));
                q[j].y = fma(ph[e + j].x, vi, fma(ph[e + j].y, vr, q[j].y));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) Q[(int64_t)(e + j) * n_pad + i] = q[j];
        }
        for (; e < n_e; ++e) {
            double2 q = Q[(int64_t)e * n_pad + i];
            q.x = fma(ph[e].x, vr, fma(-ph[e].y, vi, q.x));
            q.y = fma(ph[e].x, vi, fma(ph[e].y, vr, q.y));
            Q[(int64_t)e * n_pad + i] = q;
        }
    }
}

// Q_e = pre * psi0 for every energy (the m = 0 term, w_0 = 1).
template <typename R>
__global__ void qe_init_kernel(const void *psi_, double2 *Q, int n_e, int64_t n_pad, double pre)
{
    typedef typename V2<R>::T V;
    const V *psi = reinterpret_cast<const V *>(psi_);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += stride) {
        const V v = psi[i];
        for (int e = 0; e < n_e; ++e) Q[(int64_t)e * n_pad + i] = make_double2(pre * (double)v.x, pre * (double)v.y);
    }
}

// Batch coefficients: zero c_k for k >= max(K_g, 3) of every instance g, so
// that running more terms than an instance needs changes nothing (the
// Clenshaw terms b_k of those orders stay exactly zero).
__global__ void mask_coef_kernel(double2 *coef, const int *K, int ninst)
{
    const int g = blockIdx.x;
    if (g >= ninst) return;
    const int Ke = K[g] < 3 ? 3 : K[g];
    for (int k = threadIdx.x; k < kMaxTerms; k += blockDim.x)
        if (k >= Ke) coef[(int64_t)g * kMaxTerms + k] = make_double2(0.0, 0.0);
}

__global__ void fill_kernel(double *p, int n, double v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// One warp per (slot, term): lane-strided partial sums, then a fixed butterfly.
__global__ void reduce_kernel(const double2 *partials, int nslot, int nterm, int nblk,
                              const int *counter, int offset, double2 *out)
{
    const int wid = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= nslot * nterm) return;
    const int d = wid / nterm, q = wid - d * nterm;
    const double2 *p = partials + ((int64_t)d * nterm + q) * nblk;
    double re = 0.0, im = 0.0;
    for (int b = lane; b < nblk; b += 32) { re += p[b].x; im += p[b].y; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        const int base = counter ? *counter : 0;
        out[(int64_t)(base + offset + d) * nterm + q] = make_double2(re, im);
    }
}

__global__ void advance_kernel(int *counter, int by)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *counter += by;
}

// src: FP64 complex [nstates][n] (state-major); dst: R2 [n_pad][B] for states
// j0 .. j0+B-1, zero for padding rows and for states >= nstates.
template <typename R>
__global__ void load_states_kernel(const double2 *src, int64_t n, int64_t n_pad, int nstates,
                                   int j0, int B, void *dst0_, void *dst1_)
{
    typedef typename V2<R>::T V;
    V *dst0 = reinterpret_cast<V *>(dst0_);
    V *dst1 = reinterpret_cast<V *>(dst1_);
    const int64_t total = n_pad * B;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t row = e / B;
        const int j = (int)(e - row * B) + j0;
        V v;
        if (row < n && j < nstates) {
            const double2 s = src[(int64_t)j * n + row];
            v.x = (R)s.x; v.y = (R)s.y;
        } else {
            v.x = (R)0; v.y = (R)0;
        }
        if (dst0) dst0[e] = v;
        if (dst1) dst1[e] = v;
    }
}

template <typename R>
__global__ void load_column_kernel(const double2 *src, int64_t n, int B, int col, void *dst0_,
                                   void *dst1_)
{
    typedef typename V2<R>::T V;
    V *dst0 = reinterpret_cast<V *>(dst0_);
    V *dst1 = reinterpret_cast<V *>(dst1_);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 s = src[i];
        V v;
        v.x = (R)s.x; v.y = (R)s.y;
        dst0[i * B + col] = v;
        dst1[i * B + col] = v;
    }
}

// 1/||psi_j|| per state from the final sweep's FP64 norm partials (one warp
// per state, fixed order); all ones when there are no partials yet.
__global__ void renorm_kernel(const double2 *norm_partials, int nblk, int B, double *scale)
{
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (j >= B) return;
    if (!norm_partials) {
        if (lane == 0) scale[j] = 1.0;
        return;
    }
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += norm_partials[(int64_t)b * B + j].x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) scale[j] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
}

// dots[q] = (<T_q|T_q>, <T_{q+1}|T_q>), q = 0..; the product identities
//   mu_{2q} = 2<T_q|T_q> - mu_0,  mu_{2q+1} = 2<T_q|T_{q+1}> - mu_1
// with mu_0 = <T_0|T_0> and mu_1 = <T_0|T_1>.
__global__ void kpm_finalize_kernel(const double2 *dots, int M, double2 *mu)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double2 mu0 = dots[0];
    const double2 c01 = dots[1];                          // <T_1|T_0>
    const double2 mu1 = make_double2(c01.x, -c01.y);      // <T_0|T_1>
    double2 r;
    if (m == 0) r = mu0;
    else if (m == 1) r = mu1;
    else if ((m & 1) == 0) {
        const double2 d = dots[(m >> 1) * 2];
        r = make_double2(2.0 * d.x - mu0.x, 2.0 * d.y - mu0.y);
    } else {
        const double2 d = dots[(m >> 1) * 2 + 1];         // <T_{q+1}|T_q>
        r = make_double2(2.0 * d.x - mu1.x, -2.0 * d.y - mu1.y);
    }
    mu[m] = r;
}

}  // namespace

cudaError_t launch_bessel(double x, double tol, double2 *d_coef, int *d_K, cudaStream_t s)
{
    bessel_kernel<<<1, 32, 0, s>>>(x, tol, d_coef, d_K);
    return cudaGetLastError();
}

cudaError_t launch_dot(int precision, const void *a, const void *b, int64_t nslices,
                       double2 *partials, int grid, bool per_slice, cudaStream_t s)
{
    if (precision == TBPM_FP64) dot_slices<double><<<grid, kBlockB1, 0, s>>>(a, b, nslices, partials, per_slice);
    else dot_slices<float><<<grid, kBlockB1, 0, s>>>(a, b, nslices, partials, per_slice);
    return cudaGetLastError();
}

cudaError_t launch_reduce_seg(const double2 *partials, int nslot, int nterm, int64_t nslices,
                              const int64_t *seg_off, int nseg, const int *counter, int offset,
                              double2 *out, int64_t ld, cudaStream_t s)
{
    const int blocks = nslot * nterm * nseg;
    if (blocks <= 0) return cudaSuccess;
    reduce_seg_kernel<<<blocks, 256, 0, s>>>(partials, nslot, nterm, nslices, seg_off, nseg, counter,
                                             offset, out, ld);
    return cudaGetLastError();
}

cudaError_t launch_renorm_seg(const double2 *norm, int64_t nslices, const int64_t *seg_off, int nseg,
                              double *scale, cudaStream_t s)
{
    renorm_seg_kernel<<<nseg, 256, 0, s>>>(norm, nslices, seg_off, scale);
    return cudaGetLastError();
}

cudaError_t launch_store_column(int precision, const void *src, int64_t n, int B, int col,
                                const double *scale, double *dst, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    double2 *d = reinterpret_cast<double2 *>(dst);
    if (precision == TBPM_FP64)
        store_column_kernel<double><<<(int)blocks, 256, 0, s>>>(src, n, B, col, scale, d);
    else
        store_column_kernel<float><<<(int)blocks, 256, 0, s>>>(src, n, B, col, scale, d);
    return cudaGetLastError();
}

cudaError_t launch_qe_accumulate(int precision, const void *psi, double2 *Q, const double *energies, int n_e,
                                 int64_t n_pad, const int *counter, int delta, double h, int N, double pre,
                                 cudaStream_t s)
{
    int64_t blocks = (n_pad + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    const size_t sm = sizeof(double2) * (size_t)n_e;
    if (precision == TBPM_FP64)
        qe_accumulate_kernel<double><<<(int)blocks, 256, sm, s>>>(psi, Q, energies, n_e, n_pad, counter, delta, h, N, pre);
    else
        qe_accumulate_kernel<float><<<(int)blocks, 256, sm, s>>>(psi, Q, energies, n_e, n_pad, counter, delta, h, N, pre);
    return cudaGetLastError();
}

cudaError_t launch_qe_init(int precision, const void *psi, double2 *Q, int n_e, int64_t n_pad, double pre,
                           cudaStream_t s)
{
    int64_t blocks = (n_pad + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (precision == TBPM_FP64) qe_init_kernel<double><<<(int)blocks, 256, 0, s>>>(psi, Q, n_e, n_pad, pre);
    else qe_init_kernel<float><<<(int)blocks, 256, 0, s>>>(psi, Q, n_e, n_pad, pre);
    return cudaGetLastError();
}

cudaError_t launch_mask_coef(double2 *coef, const int *K, int ninst, cudaStream_t s)
{
    mask_coef_kernel<<<ninst, 128, 0, s>>>(coef, K, ninst);
    return cudaGetLastError();
}

cudaError_t launch_fill(double *p, int n, double v, cudaStream_t s)
{
    fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double2 *partials, int nslot, int nterm, int nblk,
                          const int *counter, int offset, double2 *out, cudaStream_t s)
{
    const int warps = nslot * nterm;
    if (warps <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (warps * 32 + threads - 1) / threads;
    reduce_kernel<<<blocks, threads, 0, s>>>(partials, nslot, nterm, nblk, counter, offset, out);
    return cudaGetLastError();
}

cudaError_t launch_advance(int *counter, int by, cudaStream_t s)
{
    advance_kernel<<<1, 32, 0, s>>>(counter, by);
    return cudaGetLastError();
}

cudaError_t launch_load_states(int precision, const double *src, int64_t n, int64_t n_pad,
                               int nstates_src, int j0, int B, void *dst0, void *dst1,
                               cudaStream_t s)
{
    const int64_t total = n_pad * B;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    const double2 *sp = reinterpret_cast<const double2 *>(src);
    if (precision == TBPM_FP64)
        load_states_kernel<double><<<(int)blocks, 256, 0, s>>>(sp, n, n_pad, nstates_src, j0, B, dst0, dst1);
    else
        load_states_kernel<float><<<(int)blocks, 256, 0, s>>>(sp, n, n_pad, nstates_src, j0, B, dst0, dst1);
    return cudaGetLastError();
}

cudaError_t launch_load_column(int precision, const double *src, int64_t n, int B, int col,
                               void *dst0, void *dst1, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    const double2 *sp = reinterpret_cast<const double2 *>(src);
    if (precision == TBPM_FP64)
        load_column_kernel<double><<<(int)blocks, 256, 0, s>>>(sp, n, B, col, dst0, dst1);
    else
        load_column_kernel<float><<<(int)blocks, 256, 0, s>>>(sp, n, B, col, dst0, dst1);
    return cudaGetLastError();
}

cudaError_t launch_renorm(const double2 *norm_partials, int nblk, int B, double *scale,
                          cudaStream_t s)
{
    renorm_kernel<<<1, 32 * B, 0, s>>>(norm_partials, nblk, B, scale);
    return cudaGetLastError();
}

cudaError_t launch_kpm_finalize(const double2 *dots, int M, int states, double2 *mu,
                                cudaStream_t s)
{
    (void)states;
    kpm_finalize_kernel<<<(M + 255) / 256, 256, 0, s>>>(dots, M, mu);
    return cudaGetLastError();
}

}  // namespace tbpm
