// Haydock (Lanczos) recursion for the local density of states, and the
// continued-fraction LDOS (the LDOS capability of the TBPM solver, Sec. 1 and
// the LDOS row of the benchmarks in Sec. 4.2.2; the recursion method of
// Haydock, Heine and Kelly).
//
// From v_0 = psi0/||psi0||, v_{-1} = 0, b_0 = 0, for n = 0, 1, ...:
//   w = H v_n - b_n v_{n-1},  a_n = Re <v_n|w>,  u = w - a_n v_n,
//   b_{n+1} = ||u||,  v_{n+1} = u / b_{n+1}.
// The vectors are kept unnormalised, v_n = s_n u_n, with the scalars on the
// device, so no pass only rescales, and every scale sits in a scalar: with
// H = (rescale/2) A (the stored operator is A = 2H/rescale) and h = rescale/2,
//   w = h s_n wt,  wt = A u_n - rho_n u_{n-1},  rho_n = b_n s_{n-1} / (h s_n),
//   a_n = h s_n^2 Re <u_n|wt>,
//   u_{n+1} = wt - (a_n / h) u_n,  so that  b_{n+1} = h s_n ||u_{n+1}||,
//   s_{n+1} = 1 / ||u_{n+1}||,  rho_{n+1} = s_n^2 ||u_{n+1}||^2.
// One pass forms wt over u_{n-1} (the sparse product plus one scaled vector:
// 10 FP64 operations per row, 2 more for Re <u_n|wt>), one elementwise pass
// forms u_{n+1} in place with ||u_{n+1}||^2.
// Each pass sums its dot per block in a fixed order; the last block of the grid
// to finish (found by a ticket counter, nothing waits) adds the per-block sums
// in a fixed order, so the total does not depend on which block is last, and
// updates a_n, or b_{n+1} and the scalars. Two launches per level, both
// programmatic dependent launches.
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

// Sum of one value per thread over the block, in a fixed order; the result is
// valid in thread 0.
__device__ double block_total(double v)
{
    __shared__ double ws[kBlockB1 / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kBlockB1 / 32; ++i) t += ws[i];
    return t;
}

// Stores the block's sum (thread 0's `mine`) in part[blockIdx.x] and takes a
// ticket. The block that takes the last ticket returns true in all its threads,
// with the sum of part[0 .. gridDim.x) in thread 0's `total` (each thread loads
// its strided share at once, then the fixed-order block sum: the same order
// whichever block is last), and resets the ticket for the next launch. No
// block waits for another: the others return false at once. Every thread of
// the block must call it.
__device__ bool last_block_total(double mine, double *part, unsigned *ticket, double &total)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = mine;
        __threadfence();                                // the partial before the ticket
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();                                    // every other block's partial is visible
    double t = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) t += __ldcg(part + i);
    total = block_total(t);
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// scalars sc[]: 0 s_n (scale of u_n), 1 b_n, 2 s_{n-1}, 3 a_n, 4 rho_n,
// 5 h s_n^2, 6 a_n / h. Once the chain has ended (s_n = +0, see hay_update) the
// product pass writes zeros: wt would otherwise grow as A^k times the residual.
// a_n -> sc[3], sc[6] and a_out[*counter]
template <typename R, int OP, bool REALV>
__global__ void __launch_bounds__(kBlockB1) hay_apply(SweepParams p, double *sc, double half_rescale,
                                                      double *part, unsigned *ticket, double *a_out,
                                                      const int *counter)
{
    pdl_wait_release();
    typedef typename V2<R>::T V;
    const V *__restrict__ x = reinterpret_cast<const V *>(p.x);       // u_n
    V *y = reinterpret_cast<V *>(p.y);                                // in u_{n-1}, out wt
    const R *diag = reinterpret_cast<const R *>(p.diag);
    const bool ended = __double_as_longlong(sc[0]) == 0;            // s_n == +0
    const R rho = (R)sc[4];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dr = 0.0;
    for (int64_t s = warp; s < p.nslices && !ended; s += nwarps) {
        const int64_t row = (s << 5) + lane;
        const V xi = __ldg(x + row);
        const V up = y[row];
        const R d = diag ? ldm<R>(diag + row) : (R)0;
        R ar = fma(d, xi.x, -rho * up.x), ai = fma(d, xi.y, -rho * up.y);
        if (OP == OP_SELL) sell_apply<R, REALV>(p, s, lane, x, ar, ai);
        else if (row < p.n) stencil_apply<R, OP>(p, row, x, ar, ai);
        V w;
        w.x = ar;
        w.y = ai;
        y[row] = w;
        const double xr = (double)xi.x, xim = (double)xi.y, wr = (double)w.x, wi = (double)w.y;
        // Re <u_n|wt>: a_n is real (H Hermitian), so the imaginary part, which
        // would cost two more FP64 operations per row, is not formed
        dr = fma(xr, wr, fma(xim, wi, dr));
    }
    if (ended) {
        V zero;
        zero.x = (R)0;
        zero.y = (R)0;
        for (int64_t s = warp; s < p.nslices; s += nwarps) y[(s << 5) + lane] = zero;
    }
    double t;
    if (last_block_total(block_total(dr), part, ticket, t) && threadIdx.x == 0) {
        const double a = ended ? 0.0 : sc[5] * t;
        sc[3] = a;
        sc[6] = a / half_rescale;
        a_out[*counter] = a;
    }
}

// u_{n+1} = wt - (a_n / h) u_n (in place over wt) and ||u_{n+1}||^2; the last
// block forms b_{n+1} = h s_n ||u_{n+1}|| (to b_out[*counter]), the next
// scalars, and advances the counter. A b_{n+1} at the rounding level of the
// vectors' precision, <= tol (|a_n| + b_n) with tol = 1e-12 in FP64 and 1e-6
// in FP32, ends the chain (an invariant subspace): it is stored as 0, and
// s = +0 keeps every later vector, a and b at 0.
template <typename R>
__global__ void __launch_bounds__(kBlockB1) hay_update(const void *u_, void *w_, int64_t nslices, double *sc,
                                                       double half_rescale, double *part, unsigned *ticket,
                                                       double *b_out, int *counter)
{
    pdl_wait_release();
    typedef typename V2<R>::T V;
    const V *u = reinterpret_cast<const V *>(u_);
    V *w = reinterpret_cast<V *>(w_);
    const R c = (R)sc[6];
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
    double t;
    if (last_block_total(block_total(nn), part, ticket, t) && threadIdx.x == 0) {
        const double sn = sc[0];
        double b = half_rescale * sn * sqrt(t);
        const double tol = sizeof(R) == 4 ? 1e-6 : 1e-12;
        if (b <= tol * (fabs(sc[3]) + sc[1])) b = 0.0;
        b_out[*counter] = b;
        sc[2] = sn;
        sc[1] = b;
        if (b > 0.0) {
            sc[0] = 1.0 / sqrt(t);
            sc[4] = sn * sn * t;
            sc[5] = half_rescale / t;
        } else {
            sc[0] = 0.0;
            sc[4] = 0.0;
            sc[5] = 0.0;
        }
        *counter += 1;
    }
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

// s_0 = 1/||psi0||, b_0 = 0, s_{-1} = 0, rho_0 = 0, h s_0^2; iteration
// counter and ticket 0.
__global__ void hay_init(const double2 *partials, int64_t W, double *sc, double half_rescale, int *counter)
{
    const double2 t = sum_partials(partials, W);
    if (threadIdx.x == 0) {
        const bool ok = t.x > 0.0;
        sc[0] = ok ? 1.0 / sqrt(t.x) : 0.0;
        sc[1] = 0.0;
        sc[2] = 0.0;
        sc[3] = 0.0;
        sc[4] = 0.0;
        sc[5] = ok ? half_rescale / t.x : 0.0;
        sc[6] = 0.0;
        counter[0] = 0;
        counter[1] = 0;
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
cudaError_t apply_t(const SweepParams &p, double *sc, double hr, double *part, unsigned *ticket, double *a_out,
                    const int *counter, int grid, bool pdl, cudaStream_t s)
{
    return launch_pdl(hay_apply<R, OP, REALV>, grid, kBlockB1, pdl, s, p, sc, hr, part, ticket, a_out, counter);
}

}  // namespace

cudaError_t launch_hay_apply(const SweepVariant &v, const SweepParams &p, double *sc, double half_rescale,
                             double *part, unsigned *ticket, double *a_out, const int *counter, int grid,
                             cudaStream_t s)
{
    const bool pdl = v.pdl;
    if (v.precision == TBPM_FP64) {
        if (v.op == OP_SELL)
            return v.real_values
                       ? apply_t<double, OP_SELL, true>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s)
                       : apply_t<double, OP_SELL, false>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s);
        if (v.op == OP_STENCIL_MONO)
            return apply_t<double, OP_STENCIL_MONO, true>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s);
        return apply_t<double, OP_STENCIL_BI, true>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s);
    }
    if (v.op == OP_SELL)
        return v.real_values
                   ? apply_t<float, OP_SELL, true>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s)
                   : apply_t<float, OP_SELL, false>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s);
    if (v.op == OP_STENCIL_MONO)
        return apply_t<float, OP_STENCIL_MONO, true>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s);
    return apply_t<float, OP_STENCIL_BI, true>(p, sc, half_rescale, part, ticket, a_out, counter, grid, pdl, s);
}

cudaError_t launch_hay_update(const SweepVariant &v, const void *u, void *w, int64_t nslices, double *sc,
                              double half_rescale, double *part, unsigned *ticket, double *b_out, int *counter,
                              int grid, cudaStream_t s)
{
    if (v.precision == TBPM_FP64)
        return launch_pdl(hay_update<double>, grid, kBlockB1, v.pdl, s, u, w, nslices, sc, half_rescale, part,
                          ticket, b_out, counter);
    return launch_pdl(hay_update<float>, grid, kBlockB1, v.pdl, s, u, w, nslices, sc, half_rescale, part, ticket,
                      b_out, counter);
}

// Grids of the two passes, whole waves of their own resident blocks: the
// product pass holds more registers than the Clenshaw sweeps (up to 64 in FP64
// against 40), so the sweep grid would leave a partial second wave.
template <typename K>
static int per_sm(K kern)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kBlockB1, 0) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return n < 1 ? 1 : n;
}

template <typename R>
static int apply_per_sm(const SweepVariant &v)
{
    if (v.op == OP_STENCIL_MONO) return per_sm(hay_apply<R, OP_STENCIL_MONO, true>);
    if (v.op == OP_STENCIL_BI) return per_sm(hay_apply<R, OP_STENCIL_BI, true>);
    return v.real_values ? per_sm(hay_apply<R, OP_SELL, true>) : per_sm(hay_apply<R, OP_SELL, false>);
}

void hay_grids(const SweepVariant &v, int num_sms, int *apply_grid, int *update_grid)
{
    const bool f64 = v.precision == TBPM_FP64;
    *apply_grid = (f64 ? apply_per_sm<double>(v) : apply_per_sm<float>(v)) * num_sms;
    *update_grid = (f64 ? per_sm(hay_update<double>) : per_sm(hay_update<float>)) * num_sms;
}

cudaError_t launch_hay_init(const double2 *partials, int64_t W, double *sc, double half_rescale, int *counter,
                            cudaStream_t s)
{
    hay_init<<<1, 256, 0, s>>>(partials, W, sc, half_rescale, counter);
    return cudaGetLastError();
}

cudaError_t launch_hay_ldos(const double *a, const double *b, int M, const double *energies, int n_e,
                            double eta, double *ldos, cudaStream_t s)
{
    hay_ldos<<<(n_e + 127) / 128, 128, 0, s>>>(a, b, M, energies, n_e, eta, ldos);
    return cudaGetLastError();
}

}  // namespace tbpm
