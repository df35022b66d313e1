// Fused Chebyshev sweeps: sparse (or stencil) product, three-term recurrence,
// series accumulation and the correlation dot, one HBM pass per term.
//
// The series of one time step (Sec. 2.2.1, the propagation listings),
//   psi(t+dt) = sum_{k<K} c_k T_k(H~) psi,   c_k = (2 - delta_k0)(-i)^k J_k(dt*rescale),
// is summed here by Clenshaw's backward recurrence instead of the forward
// recurrence of the listings. With b_K = b_{K+1} = 0,
//   b_k = c_k psi + 2 H~ b_{k+1} - b_{k+2}      (k = K-1 .. 1),
//   psi(t+dt) = c_0 psi + H~ b_1 - b_2.
// Both forms make K-1 sparse products per step. The backward form keeps no
// running sum vector: each sweep reads psi, gathers b_{k+1}, and overwrites
// b_{k+2} with b_k in place, 4 vector streams per row instead of the 5 of the
// forward form (T_{k-1}, T_{k-2} -> T_k, out read and written). As in the
// paper's C++ form, the imaginary factors stay in the coefficients, so the
// sparse product is real-scalar: c_k is real for even k and imaginary for odd
// k, and each sweep multiplies psi by a purely real or purely imaginary number.
//
// The stored operator is pre-scaled at create time to A = 2 H / rescale, so a
// sweep forms acc = A x and
//   FIRST  (k = K-2): y = c_{K-2} psi + c_{K-1} A psi
//   SECOND (k = K-3): y = (c_{K-3} - c_{K-1}) psi + A b_{K-2}
//   MID    (k < K-3): y = c_k psi + A b_{k+1} - b_{k+2}           (y aliases b_{k+2})
//   FINAL  (k = 0)  : y = (c_0 - [K=3] c_2) psi + A b_1 / 2 - [K>=4] b_2   (y aliases psi)
// and the final sweep also accumulates <psi0|y> into per-block partials.
// The KPM sweep (Sec. 1) is T_{m+1} = A T_m - T_{m-1} with the two dots that
// the doubling identities need.
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

enum BMode { B_ONE = 0, B_REAL = 1, B_IMAG = 2 };

// Coefficients of one sweep: a on psi (real, or imaginary if AIMAG), beta on A x.
// For a batch of instances, coefficients and the renormalisation scale are
// those of the slice's instance.
// Only the FP64 operations a sweep needs are issued (each one costs every
// thread of the grid a slot of GB300's narrow FP64 pipe): the difference for
// the second sweep, the scale only when renormalising, bscale only when not 1.
template <typename R, int BM, bool AIMAG>
__device__ __forceinline__ void sweep_coeffs(const SweepParams &p, int inst, R &a, R &beta)
{
    const double2 *c = p.coef + (int64_t)inst * kMaxTerms;
    const double2 ca = c[p.ia];
    double av = AIMAG ? ca.y : ca.x;
    if (p.ib >= 0) av -= AIMAG ? c[p.ib].y : c[p.ib].x;
    // renormalisation folds 1/||psi|| into the coefficients that multiply psi
    // (in the first sweep also into beta, whose operand is psi itself)
    if (p.scale) av *= p.scale[inst];
    a = (R)av;
    beta = (R)p.bscale;
    if (BM != B_ONE && p.ic >= 0) {
        double bv = BM == B_REAL ? c[p.ic].x : c[p.ic].y;
        if (p.bscale != 1.0) bv *= p.bscale;
        if (p.scale) bv *= p.scale[inst];
        beta = (R)bv;
    }
}

// One Clenshaw sweep for a single state per row (B = 1). A warp owns one
// 32-row slice at a time (grid-stride over slices).
// The final sweep accumulates <psi0|y> (and ||y||^2 when renormalising) per
// lane in FP64 across the warp's slices and reduces once per warp, at the end,
// into partials[delta * W + warp] (W = warps in the grid, fixed per context):
// FP64 is GB300's scarce pipe, and a butterfly per slice would cost as many FP64
// instructions as the sparse product. For a batch of instances (MULTI) the
// coefficients are those of each slice's instance and the partials are stored
// per slice, partials[delta * nslices + slice], so that instances stay apart.
template <typename R, int OP, bool REALV, int BM, bool AIMAG, bool HASZ, bool FINAL, bool MULTI>
__global__ void __launch_bounds__(kBlockB1) sweep_b1(SweepParams p)
{
    typedef typename V2<R>::T V;
    pdl_wait_release();
    R a, beta;
    sweep_coeffs<R, BM, AIMAG>(p, 0, a, beta);

    const V *__restrict__ x = reinterpret_cast<const V *>(p.x);
    const V *psi = reinterpret_cast<const V *>(p.psi);
    const V *z = reinterpret_cast<const V *>(p.z);
    V *y = reinterpret_cast<V *>(p.y);
    const V *psi0 = reinterpret_cast<const V *>(p.psi0);
    const R *diag = reinterpret_cast<const R *>(p.diag);

    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dr = 0.0, di = 0.0, nn = 0.0;
    F2Sum fr, fi, fn;                   // FP32 data: the same sums on the FP32 pipe
    constexpr bool kF32 = sizeof(R) == 4;

    int cur_inst = 0;                   // instance whose coefficients a, beta hold
    for (int64_t s = warp; s < p.nslices; s += nwarps) {
        if (MULTI) {                    // instances span many slices: recompute on a change only
            const int g = __ldg(p.slice_inst + s);
            if (g != cur_inst) {
                sweep_coeffs<R, BM, AIMAG>(p, g, a, beta);
                cur_inst = g;
            }
        }
        const int64_t row = (s << 5) + lane;
        const V ps = psi[row];
        // t = a psi - z  (a real: a*psi; a imaginary: i*a*psi), one FMA per part
        R tr, ti;
        if (HASZ) {
            const V zz = z[row];
            if (AIMAG) { tr = fma(-a, ps.y, -zz.x); ti = fma(a, ps.x, -zz.y); }
            else { tr = fma(a, ps.x, -zz.x); ti = fma(a, ps.y, -zz.y); }
        } else {
            if (AIMAG) { tr = -a * ps.y; ti = a * ps.x; } else { tr = a * ps.x; ti = a * ps.y; }
        }
        const V xi = __ldg(x + row);
        const R d = diag ? ldm<R>(diag + row) : (R)0;
        R ar, ai;
        if (BM == B_ONE) { ar = fma(d, xi.x, tr); ai = fma(d, xi.y, ti); }
        else { ar = d * xi.x; ai = d * xi.y; }
        if (OP == OP_SELL) sell_apply<R, REALV>(p, s, lane, x, ar, ai);
        else if (row < p.n) stencil_apply<R, OP>(p, row, x, ar, ai);
        V out;
        if (BM == B_ONE) { out.x = ar; out.y = ai; }
        else if (BM == B_REAL) { out.x = fma(beta, ar, tr); out.y = fma(beta, ai, ti); }
        else { out.x = fma(-beta, ai, tr); out.y = fma(beta, ar, ti); }
        y[row] = out;
        if (FINAL && kF32 && !MULTI) {
            const V q = psi0[row];
            fr.add_dot((float)q.x, (float)out.x, (float)q.y, (float)out.y);
            fi.add_dot((float)q.x, (float)out.y, -(float)q.y, (float)out.x);
            if (p.norm_partials) fn.add_dot((float)out.x, (float)out.x, (float)out.y, (float)out.y);
        } else if (FINAL) {
            const V q = psi0[row];
            const double qr = (double)q.x, qi = (double)q.y;
            const double orr = (double)out.x, oi = (double)out.y;
            if (MULTI) {
                const double sr = warp_sum(fma(qr, orr, qi * oi));
                const double si = warp_sum(fma(qr, oi, -qi * orr));
                if (lane == 0) p.partials[(int64_t)p.delta * p.nslices + s] = make_double2(sr, si);
                if (p.norm_partials) {
                    const double sn = warp_sum(fma(orr, orr, oi * oi));
                    if (lane == 0) p.norm_partials[(int64_t)p.delta * p.nslices + s] = make_double2(sn, 0.0);
                }
            } else {
                dr = fma(qr, orr, fma(qi, oi, dr));
                di = fma(qr, oi, fma(-qi, orr, di));
                if (p.norm_partials) nn = fma(orr, orr, fma(oi, oi, nn));
            }
        }
    }
    if (FINAL && !MULTI && kF32) {
        // FP32 data: the block's sums in FP32 pairs, one conversion per value; the
        // block's first warp slot holds them, its other warp slots zero
        F2Sum a[3] = {fr, fi, fn};
        double v[3];
        block_sum_f2<3>(a, v);
        if (lane == 0) {
            const bool lead = (threadIdx.x >> 5) == 0;
            p.partials[(int64_t)p.delta * nwarps + warp] = lead ? make_double2(v[0], v[1]) : make_double2(0.0, 0.0);
            if (p.norm_partials)
                p.norm_partials[(int64_t)p.delta * nwarps + warp] = make_double2(lead ? v[2] : 0.0, 0.0);
        }
    } else if (FINAL && !MULTI) {
        dr = warp_sum(dr);
        di = warp_sum(di);
        if (lane == 0) p.partials[(int64_t)p.delta * nwarps + warp] = make_double2(dr, di);
        if (p.norm_partials) {
            nn = warp_sum(nn);
            if (lane == 0) p.norm_partials[(int64_t)p.delta * nwarps + warp] = make_double2(nn, 0.0);
        }
    }
}

// KPM sweep for B = 1: y = scale * (A x) - [!first] y. Per lane FP64 sums of
// <x|x> and Re <y|x> over the warp's slices, reduced once per warp into
// partials[(2 delta + 0/1) * W + warp]. With x = T_m psi0 and y = T_{m+1} psi0,
// <y|x> = <psi0|T_{m+1}(H~) T_m(H~)|psi0> is real for Hermitian H (a real
// polynomial of H~ between the same state), so its imaginary part is stored
// as zero instead of costing two more FP64 operations per row.
template <typename R, int OP, bool REALV, bool FIRST>
__global__ void __launch_bounds__(kBlockB1, sizeof(R) == 4 ? 3 : 2) kpm_b1(KpmParams p)
{
    typedef typename V2<R>::T V;
    pdl_wait_release();
    SweepParams sp;                     // operator fields for the shared helpers
    sp.n = p.n; sp.nslices = p.nslices; sp.slice_off = p.slice_off; sp.cols = p.cols; sp.vals = p.vals;
    sp.diag = p.diag; sp.l1 = p.l1; sp.l2 = p.l2; sp.t = p.t; sp.t_perp = p.t_perp;
    const V *__restrict__ x = reinterpret_cast<const V *>(p.x);
    V *y = reinterpret_cast<V *>(p.y);
    const R *diag = reinterpret_cast<const R *>(p.diag);
    const R sc = (R)p.scale;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double nn = 0.0, cr = 0.0;
    F2Sum fn, fr;                       // FP32 data: the same sums on the FP32 pipe
    for (int64_t s = warp; s < p.nslices; s += nwarps) {
        const int64_t row = (s << 5) + lane;
        const V xi = __ldg(x + row);
        const R d = diag ? __ldg(diag + row) : (R)0;
        R ar, ai;
        V out;
        if (FIRST) {
            ar = d * xi.x; ai = d * xi.y;
            if (OP == OP_SELL) sell_apply<R, REALV>(sp, s, lane, x, ar, ai);
            else if (row < p.n) stencil_apply<R, OP>(sp, row, x, ar, ai);
            out.x = sc * ar; out.y = sc * ai;
        } else {
            const V zz = y[row];
            ar = fma(d, xi.x, -zz.x); ai = fma(d, xi.y, -zz.y);
            if (OP == OP_SELL) sell_apply<R, REALV>(sp, s, lane, x, ar, ai);
            else if (row < p.n) stencil_apply<R, OP>(sp, row, x, ar, ai);
            out.x = ar; out.y = ai;
        }
        y[row] = out;
        if (sizeof(R) == 4) {
            fn.add_dot((float)xi.x, (float)xi.x, (float)xi.y, (float)xi.y);
            fr.add_dot((float)out.x, (float)xi.x, (float)out.y, (float)xi.y);
        } else {
            const double xr = (double)xi.x, xim = (double)xi.y;
            const double orr = (double)out.x, oi = (double)out.y;
            nn = fma(xr, xr, fma(xim, xim, nn));
            cr = fma(orr, xr, fma(oi, xim, cr));        // Re sum conj(y) x
        }
    }
    if (sizeof(R) == 4) {
        // the block's sums in FP32 pairs, one conversion per value, in the block's
        // first warp slot (its other warp slots zero)
        F2Sum a[2] = {fn, fr};
        double v[2];
        block_sum_f2<2>(a, v);
        if (lane == 0) {
            const bool lead = (threadIdx.x >> 5) == 0;
            p.partials[((int64_t)p.delta * 2) * nwarps + warp] = make_double2(lead ? v[0] : 0.0, 0.0);
            p.partials[((int64_t)p.delta * 2 + 1) * nwarps + warp] = make_double2(lead ? v[1] : 0.0, 0.0);
        }
        return;
    }
    nn = warp_sum(nn);
    cr = warp_sum(cr);
    if (lane == 0) {
        p.partials[((int64_t)p.delta * 2) * nwarps + warp] = make_double2(nn, 0.0);
        p.partials[((int64_t)p.delta * 2 + 1) * nwarps + warp] = make_double2(cr, 0.0);
    }
}

template <typename R, int OP, bool REALV, bool MULTI>
cudaError_t sweep_dispatch(SweepKind kind, bool a_imag, bool has_z, const SweepParams &p,
                           int grid, bool pdl, cudaStream_t s)
{
    switch (kind) {
    case SW_FIRST:
        return a_imag ? launch_pdl(sweep_b1<R, OP, REALV, B_REAL, true, false, false, MULTI>, grid, kBlockB1, pdl, s, p)
                      : launch_pdl(sweep_b1<R, OP, REALV, B_IMAG, false, false, false, MULTI>, grid, kBlockB1, pdl, s, p);
    case SW_SECOND:
        return a_imag ? launch_pdl(sweep_b1<R, OP, REALV, B_ONE, true, false, false, MULTI>, grid, kBlockB1, pdl, s, p)
                      : launch_pdl(sweep_b1<R, OP, REALV, B_ONE, false, false, false, MULTI>, grid, kBlockB1, pdl, s, p);
    case SW_MID:
        return a_imag ? launch_pdl(sweep_b1<R, OP, REALV, B_ONE, true, true, false, MULTI>, grid, kBlockB1, pdl, s, p)
                      : launch_pdl(sweep_b1<R, OP, REALV, B_ONE, false, true, false, MULTI>, grid, kBlockB1, pdl, s, p);
    case SW_FINAL:
        return has_z ? launch_pdl(sweep_b1<R, OP, REALV, B_REAL, false, true, true, MULTI>, grid, kBlockB1, pdl, s, p)
                     : launch_pdl(sweep_b1<R, OP, REALV, B_REAL, false, false, true, MULTI>, grid, kBlockB1, pdl, s, p);
    }
    return cudaErrorInvalidValue;
}

template <typename R, int OP, bool REALV>
cudaError_t kpm_dispatch(const KpmParams &p, int grid, bool pdl, cudaStream_t s)
{
    return p.first ? launch_pdl(kpm_b1<R, OP, REALV, true>, grid, kBlockB1, pdl, s, p)
                   : launch_pdl(kpm_b1<R, OP, REALV, false>, grid, kBlockB1, pdl, s, p);
}

}  // namespace

cudaError_t launch_sweep(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                         const SweepParams &p, int grid, cudaStream_t s)
{
    if (v.states != 1) return cudaErrorInvalidValue;
    const bool multi = p.slice_inst != nullptr;        // batches of instances: SELL only
    if (multi && v.op != OP_SELL) return cudaErrorInvalidValue;
    if (v.precision == TBPM_FP64) {
        if (v.op == OP_SELL) {
            if (multi)
                return v.real_values ? sweep_dispatch<double, OP_SELL, true, true>(kind, a_imag, has_z, p, grid, v.pdl, s)
                                     : sweep_dispatch<double, OP_SELL, false, true>(kind, a_imag, has_z, p, grid, v.pdl, s);
            return v.real_values ? sweep_dispatch<double, OP_SELL, true, false>(kind, a_imag, has_z, p, grid, v.pdl, s)
                                 : sweep_dispatch<double, OP_SELL, false, false>(kind, a_imag, has_z, p, grid, v.pdl, s);
        }
        if (v.op == OP_STENCIL_MONO)
            return sweep_dispatch<double, OP_STENCIL_MONO, true, false>(kind, a_imag, has_z, p, grid, v.pdl, s);
        return sweep_dispatch<double, OP_STENCIL_BI, true, false>(kind, a_imag, has_z, p, grid, v.pdl, s);
    }
    if (v.op == OP_SELL) {
        if (multi)
            return v.real_values ? sweep_dispatch<float, OP_SELL, true, true>(kind, a_imag, has_z, p, grid, v.pdl, s)
                                 : sweep_dispatch<float, OP_SELL, false, true>(kind, a_imag, has_z, p, grid, v.pdl, s);
        return v.real_values ? sweep_dispatch<float, OP_SELL, true, false>(kind, a_imag, has_z, p, grid, v.pdl, s)
                             : sweep_dispatch<float, OP_SELL, false, false>(kind, a_imag, has_z, p, grid, v.pdl, s);
    }
    if (v.op == OP_STENCIL_MONO)
        return sweep_dispatch<float, OP_STENCIL_MONO, true, false>(kind, a_imag, has_z, p, grid, v.pdl, s);
    return sweep_dispatch<float, OP_STENCIL_BI, true, false>(kind, a_imag, has_z, p, grid, v.pdl, s);
}

cudaError_t launch_kpm(const SweepVariant &v, const KpmParams &p, int grid, cudaStream_t s)
{
    if (v.states != 1) return cudaErrorInvalidValue;
    if (v.precision == TBPM_FP64) {
        if (v.op == OP_SELL)
            return v.real_values ? kpm_dispatch<double, OP_SELL, true>(p, grid, v.pdl, s)
                                 : kpm_dispatch<double, OP_SELL, false>(p, grid, v.pdl, s);
        if (v.op == OP_STENCIL_MONO) return kpm_dispatch<double, OP_STENCIL_MONO, true>(p, grid, v.pdl, s);
        return kpm_dispatch<double, OP_STENCIL_BI, true>(p, grid, v.pdl, s);
    }
    if (v.op == OP_SELL)
        return v.real_values ? kpm_dispatch<float, OP_SELL, true>(p, grid, v.pdl, s)
                             : kpm_dispatch<float, OP_SELL, false>(p, grid, v.pdl, s);
    if (v.op == OP_STENCIL_MONO) return kpm_dispatch<float, OP_STENCIL_MONO, true>(p, grid, v.pdl, s);
    return kpm_dispatch<float, OP_STENCIL_BI, true>(p, grid, v.pdl, s);
}

// Grid of the KPM kernel: its own occupancy (it holds the dot sums in more
// registers than the Clenshaw sweeps), whole waves of resident blocks.
template <typename R>
static int kpm_occupancy(int op, int *per_sm)
{
    cudaError_t e;
    if (op == OP_STENCIL_MONO)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kpm_b1<R, OP_STENCIL_MONO, true, false>, kBlockB1, 0);
    else if (op == OP_STENCIL_BI)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kpm_b1<R, OP_STENCIL_BI, true, false>, kBlockB1, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kpm_b1<R, OP_SELL, true, false>, kBlockB1, 0);
    return e == cudaSuccess ? 0 : 1;
}

int kpm_grid(const SweepVariant &v, int num_sms)
{
    int per_sm = 0;
    const int bad = v.precision == TBPM_FP64 ? kpm_occupancy<double>(v.op, &per_sm)
                                             : kpm_occupancy<float>(v.op, &per_sm);
    if (bad || per_sm < 1) per_sm = 2;
    return per_sm * num_sms;
}

// Grid of the single-state sweeps: whole waves of the middle sweep of this
// operator (the stencil kernels hold more registers than the SELL ones).
template <typename R>
static int middle_sweep_occupancy(int op, int *per_sm)
{
    cudaError_t e;
    if (op == OP_STENCIL_MONO)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            per_sm, sweep_b1<R, OP_STENCIL_MONO, true, B_ONE, false, true, false, false>, kBlockB1, 0);
    else if (op == OP_STENCIL_BI)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            per_sm, sweep_b1<R, OP_STENCIL_BI, true, B_ONE, false, true, false, false>, kBlockB1, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            per_sm, sweep_b1<R, OP_SELL, true, B_ONE, false, true, false, false>, kBlockB1, 0);
    return e == cudaSuccess ? 0 : 1;
}

int sweep_grid(const SweepVariant &v, int num_sms)
{
    int per_sm = 0;
    const int bad = v.precision == TBPM_FP64 ? middle_sweep_occupancy<double>(v.op, &per_sm)
                                             : middle_sweep_occupancy<float>(v.op, &per_sm);
    if (bad || per_sm < 1) per_sm = 4;
    return per_sm * num_sms;
}

}  // namespace tbpm
