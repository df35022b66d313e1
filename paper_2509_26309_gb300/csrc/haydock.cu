// Haydock (Lanczos) recursion for the local density of states, and the
// continued-fraction LDOS (the LDOS capability of the TBPM solver, Sec. 1 and
// the LDOS row of the benchmarks in Sec. 4.2.2; the recursion method of
// Haydock, Heine and Kelly).
//
// From v_0 = psi0/||psi0||, v_{-1} = 0, b_0 = 0, for n = 0, 1, ...:
//   w = H v_n - b_n v_{n-1},  a_n = Re <v_n|w>,  u = w - a_n v_n,
//   b_{n+1} = ||u||,  v_{n+1} = u / b_{n+1}.
// The vectors are kept unnormalised, v_n = s_n u_n, with the scalars s_n, b_n
// on the device, so no pass only rescales: one pass forms w (sparse product
// plus the b_n v_{n-1} term, written over u_{n-1}) with the dot <u_n|w>, one
// elementwise pass forms u_{n+1} = w - a_n s_n u_n in place with ||u_{n+1}||^2,
// and two single-block kernels reduce the per-warp FP64 partials in a fixed
// order and update a_n, b_{n+1}, s_{n+1}. The stored operator is A = 2H/rescale,
// so H x = (rescale/2) A x.
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

// scalars sc[]: 0 s_n (scale of u_n), 1 b_n, 2 s_{n-1}, 3 a_n
template <typename R, int OP, bool REALV>
__global__ void __launch_bounds__(kBlockB1) hay_apply(SweepParams p, const double *sc, double half_rescale)
{
    typedef typename V2<R>::T V;
    const V *__restrict__ x = reinterpret_cast<const V *>(p.x);       // u_n
    V *y = reinterpret_cast<V *>(p.y);                                // in u_{n-1}, out w
    const R *diag = reinterpret_cast<const R *>(p.diag);
    const R ca = (R)(half_rescale * sc[0]);
    const R cb = (R)(sc[1] * sc[2]);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dr = 0.0;
    for (int64_t s = warp; s < p.nslices; s += nwarps) {
        const int64_t row = (s << 5) + lane;
        const V xi = __ldg(x + row);
        const V up = y[row];
        const R d = diag ? ldm<R>(diag + row) : (R)0;
        R ar = d * xi.x, ai = d * xi.y;
        if (OP == OP_SELL) sell_apply<R, REALV>(p, s, lane, x, ar, ai);
        else if (row < p.n) stencil_apply<R, OP>(p, row, x, ar, ai);
        V w;
        w.x = fma(ca, ar, -cb * up.x);
        w.y = fma(ca, ai, -cb * up.y);
        y[row] = w;
        const double xr = (double)xi.x, xim = (double)xi.y, wr = (double)w.x, wi = (double)w.y;
        // Re <u_n|w>: a_n is real (H Hermitian), so the imaginary part, which
        // would cost two more FP64 operations per row, is not formed
        dr = fma(xr, wr, fma(xim, wi, dr));
    }
    dr = warp_sum(dr);
    if (lane == 0) p.partials[warp] = make_double2(dr, 0.0);
}

// u_{n+1} = w - a_n s_n u_n (in place over w) and ||u_{n+1}||^2 per warp.
template <typename R>
__global__ void __launch_bounds__(kBlockB1) hay_update(const void *u_, void *w_, int64_t nslices,
                                                       const double *sc, double2 *partials)
{
    typedef typename V2<R>::T V;
    const V *u = reinterpret_cast<const V *>(u_);
    V *w = reinterpret_cast<V *>(w_);
    const R c = (R)(sc[3] * sc[0]);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double nn = 0.0;
    for (int64_t s = warp; s < nslices; s += nwarps) {
        const int64_t row = (s << 5) + lane;
        const V ui = u[row];
        V wi = w[row];
        wi.x = fma(-c, ui.x, wi.x);
        wi.y = fma(-c, ui.y, wi.y);
        w[row] = wi;
        const double r = (double)wi.x, im = (double)wi.y;
        nn = fma(r, r, fma(im, im, nn));
    }
    nn = warp_sum(nn);
    if (lane == 0) partials[warp] = make_double2(nn, 0.0);
}

// Fixed-order block sum of W complex partials (one block of 256 threads).
__device__ double2 sum_partials(const double2 *p, int64_t W)
{
    __shared__ double sr[256], si[256];
    double re = 0.0, im = 0.0;
    for (int64_t i = threadIdx.x; i < W; i += blockDim.x) { re += p[i].x; im += p[i].y; }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { sr[threadIdx.x] += sr[threadIdx.x + o]; si[threadIdx.x] += si[threadIdx.x + o]; }
        __syncthreads();
    }
    return make_double2(sr[0], si[0]);
}

// s_0 = 1/||psi0||, b_0 = 0, s_{-1} = 0, iteration counter 0.
__global__ void hay_init(const double2 *partials, int64_t W, double *sc, int *counter)
{
    const double2 t = sum_partials(partials, W);
    if (threadIdx.x == 0) {
        sc[0] = t.x > 0.0 ? 1.0 / sqrt(t.x) : 0.0;
        sc[1] = 0.0;
        sc[2] = 0.0;
        sc[3] = 0.0;
        *counter = 0;
    }
}

// a_n = s_n Re <u_n|w>
__global__ void hay_scalar1(const double2 *partials, int64_t W, double *sc, double *a_out,
                            const int *counter)
{
    const double2 t = sum_partials(partials, W);
    if (threadIdx.x == 0) {
        const double a = sc[0] * t.x;
        sc[3] = a;
        a_out[*counter] = a;
    }
}

// b_{n+1} = ||u_{n+1}||; shift the scales; n <- n + 1. A b_{n+1} at rounding
// level, <= 1e-12 (|a_n| + b_n), ends the chain (an invariant subspace): it is
// stored as 0 and the scale 0 keeps every later vector, a and b at 0.
__global__ void hay_scalar2(const double2 *partials, int64_t W, double *sc, double *b_out, int *counter)
{
    const double2 t = sum_partials(partials, W);
    if (threadIdx.x == 0) {
        double b = sqrt(t.x);
        if (b <= 1e-12 * (fabs(sc[3]) + sc[1])) b = 0.0;
        b_out[*counter] = b;
        sc[2] = sc[0];
        sc[0] = b > 0.0 ? 1.0 / b : 0.0;
        sc[1] = b;
        *counter += 1;
    }
}

// rho(E_j) = -Im G(E_j + i eta) / pi, G(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ...)),
// evaluated from the bottom level (b[m] = b_{m+1}); one thread per energy.
__global__ void hay_ldos(const double *a, const double *b, int M, const double *energies, int n_e,
                         double eta, double *ldos)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_e) return;
    const double zr = energies[j], zi = eta;
    double gr = 0.0, gi = 0.0;                              // G_{m+1}
    for (int m = M - 1; m >= 0; --m) {
        const double b2 = (m == M - 1) ? 0.0 : b[m] * b[m];
        const double dr = zr - a[m] - b2 * gr, di = zi - b2 * gi;  // z - a_m - b^2 G_{m+1}
        const double inv = 1.0 / (dr * dr + di * di);
        gr = dr * inv;
        gi = -di * inv;
    }
    const double pi = 3.141592653589793238462643383279502884;
    ldos[j] = -gi / pi;
}

template <typename R, int OP, bool REALV>
cudaError_t apply_t(const SweepParams &p, const double *sc, double hr, int grid, cudaStream_t s)
{
    hay_apply<R, OP, REALV><<<grid, kBlockB1, 0, s>>>(p, sc, hr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hay_apply(const SweepVariant &v, const SweepParams &p, const double *sc,
                             double half_rescale, int grid, cudaStream_t s)
{
    if (v.precision == TBPM_FP64) {
        if (v.op == OP_SELL)
            return v.real_values ? apply_t<double, OP_SELL, true>(p, sc, half_rescale, grid, s)
                                 : apply_t<double, OP_SELL, false>(p, sc, half_rescale, grid, s);
        if (v.op == OP_STENCIL_MONO) return apply_t<double, OP_STENCIL_MONO, true>(p, sc, half_rescale, grid, s);
        return apply_t<double, OP_STENCIL_BI, true>(p, sc, half_rescale, grid, s);
    }
    if (v.op == OP_SELL)
        return v.real_values ? apply_t<float, OP_SELL, true>(p, sc, half_rescale, grid, s)
                             : apply_t<float, OP_SELL, false>(p, sc, half_rescale, grid, s);
    if (v.op == OP_STENCIL_MONO) return apply_t<float, OP_STENCIL_MONO, true>(p, sc, half_rescale, grid, s);
    return apply_t<float, OP_STENCIL_BI, true>(p, sc, half_rescale, grid, s);
}

cudaError_t launch_hay_update(int precision, const void *u, void *w, int64_t nslices, const double *sc,
                              double2 *partials, int grid, cudaStream_t s)
{
    if (precision == TBPM_FP64) hay_update<double><<<grid, kBlockB1, 0, s>>>(u, w, nslices, sc, partials);
    else hay_update<float><<<grid, kBlockB1, 0, s>>>(u, w, nslices, sc, partials);
    return cudaGetLastError();
}

cudaError_t launch_hay_scalar(int which, const double2 *partials, int64_t W, double *sc, double *out,
                              int *counter, cudaStream_t s)
{
    if (which == 0) hay_init<<<1, 256, 0, s>>>(partials, W, sc, counter);
    else if (which == 1) hay_scalar1<<<1, 256, 0, s>>>(partials, W, sc, out, counter);
    else hay_scalar2<<<1, 256, 0, s>>>(partials, W, sc, out, counter);
    return cudaGetLastError();
}

cudaError_t launch_hay_ldos(const double *a, const double *b, int M, const double *energies, int n_e,
                            double eta, double *ldos, cudaStream_t s)
{
    hay_ldos<<<(n_e + 127) / 128, 128, 0, s>>>(a, b, M, energies, n_e, eta, ldos);
    return cudaGetLastError();
}

}  // namespace tbpm
