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
#include "sweep_b1.cuh"

namespace tbpm {
namespace {

// KPM sweep for B = 1: y = scale * (A x) - [!first] y. Per lane FP64 sums of
// <x|x> and Re <y|x> over the warp's slices, reduced once per warp into
// partials[(2 delta + 0/1) * W + warp]. With x = T_m psi0 and y = T_{m+1} psi0,
// <y|x> = <psi0|T_{m+1}(H~) T_m(H~)|psi0> is real for Hermitian H (a real
// polynomial of H~ between the same state), so its imaginary part is stored
// as zero instead of costing two more FP64 operations per row.
template <typename R, int OP, int VM, bool FIRST>
__global__ void __launch_bounds__(kBlockB1, sizeof(R) == 4 ? 3 : 2) kpm_b1(KpmParams p)
{
    typedef typename V2<R>::T V;
    pdl_wait_release();
    SweepParams sp;                     // operator fields for the shared helpers
    sp.n = p.n; sp.nslices = p.nslices; sp.slice_off = p.slice_off; sp.cols = p.cols; sp.vals = p.vals;
    sp.diag = p.diag; sp.l1 = p.l1; sp.l2 = p.l2; sp.t = p.t; sp.t_perp = p.t_perp;
    sp.cdelta = p.cdelta; sp.vidx = p.vidx; sp.vtab = p.vtab; sp.rowpack = p.rowpack; sp.npad = p.npad;
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
            if (OP == OP_SELL) sell_apply<R, VM>(sp, s, lane, x, ar, ai);
            else if (row < p.n) stencil_apply<R, OP>(sp, row, x, ar, ai);
            out.x = sc * ar; out.y = sc * ai;
        } else {
            const V zz = y[row];
            ar = fma(d, xi.x, -zz.x); ai = fma(d, xi.y, -zz.y);
            if (OP == OP_SELL) sell_apply<R, VM>(sp, s, lane, x, ar, ai);
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

template <typename R, int OP, int VM>
cudaError_t kpm_dispatch(const KpmParams &p, int grid, bool pdl, cudaStream_t s)
{
    return p.first ? launch_pdl(kpm_b1<R, OP, VM, true>, grid, kBlockB1, pdl, s, p)
                   : launch_pdl(kpm_b1<R, OP, VM, false>, grid, kBlockB1, pdl, s, p);
}

}  // namespace

// The default shape (one slice per warp iteration, up to 512 threads per
// block) of every operator.
static cudaError_t launch_sweep_default(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                                 const SweepParams &p, int grid, cudaStream_t s)
{
    const bool multi = p.slice_inst != nullptr;        // batches of instances: SELL only
    const int b = v.block;
    if (multi && v.op != OP_SELL) return cudaErrorInvalidValue;
    if (v.precision == TBPM_FP64) {
        if (v.op == OP_SELL) return sell_shape_launch<1, kBlockB1>(v, kind, a_imag, has_z, p, grid, s);
        if (v.op == OP_STENCIL_MONO)
            return sweep_dispatch<double, OP_STENCIL_MONO, true, false, 1, kBlockB1>(kind, a_imag, has_z, p, grid, b, v.pdl, s);
        return sweep_dispatch<double, OP_STENCIL_BI, true, false, 1, kBlockB1>(kind, a_imag, has_z, p, grid, b, v.pdl, s);
    }
    if (v.op == OP_SELL) return sell_shape_launch<1, kBlockB1>(v, kind, a_imag, has_z, p, grid, s);
    if (v.op == OP_STENCIL_MONO)
        return sweep_dispatch<float, OP_STENCIL_MONO, true, false, 1, kBlockB1>(kind, a_imag, has_z, p, grid, b, v.pdl, s);
    return sweep_dispatch<float, OP_STENCIL_BI, true, false, 1, kBlockB1>(kind, a_imag, has_z, p, grid, b, v.pdl, s);
}

bool sweep_shape_built(const SweepVariant &v)
{
    if (v.block < 32 || (v.block & 31) != 0) return false;
    if (v.spw == 1 && v.block <= kBlockB1) return true;
    if (v.op != OP_SELL) return false;
    return (v.spw == 1 && v.block == 1024) || ((v.spw == 2 || v.spw == 4) && v.block <= kBlockB1);
}

cudaError_t launch_sweep(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                         const SweepParams &p, int grid, cudaStream_t s)
{
    if (v.states != 1 || !sweep_shape_built(v)) return cudaErrorInvalidValue;
    if (p.slice_inst != nullptr && v.op != OP_SELL) return cudaErrorInvalidValue;
    if (v.spw == 1 && v.block <= kBlockB1) return launch_sweep_default(v, kind, a_imag, has_z, p, grid, s);
    if (v.spw == 1) return launch_sell_s1_b1024(v, kind, a_imag, has_z, p, grid, s);
    if (v.spw == 2) return launch_sell_s2_b512(v, kind, a_imag, has_z, p, grid, s);
    return launch_sell_s4_b512(v, kind, a_imag, has_z, p, grid, s);
}

int sweep_shape_occupancy(const SweepVariant &v, bool multi, int kind)
{
    if (!sweep_shape_built(v)) return 0;
    if (v.spw == 1 && v.block <= kBlockB1) {
        if (v.op == OP_SELL) return sell_shape_occupancy<1, kBlockB1>(v, multi, kind);
        if (v.precision == TBPM_FP64)
            return v.op == OP_STENCIL_MONO ? sweep_occupancy_of<double, OP_STENCIL_MONO, true, false, 1, kBlockB1>(v.block, kind)
                                           : sweep_occupancy_of<double, OP_STENCIL_BI, true, false, 1, kBlockB1>(v.block, kind);
        return v.op == OP_STENCIL_MONO ? sweep_occupancy_of<float, OP_STENCIL_MONO, true, false, 1, kBlockB1>(v.block, kind)
                                       : sweep_occupancy_of<float, OP_STENCIL_BI, true, false, 1, kBlockB1>(v.block, kind);
    }
    if (v.spw == 1) return occupancy_sell_s1_b1024(v, multi, kind);
    if (v.spw == 2) return occupancy_sell_s2_b512(v, multi, kind);
    return occupancy_sell_s4_b512(v, multi, kind);
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
        return v.packed == 2 ? kpm_dispatch<float, OP_SELL, VM_ROWS>(p, grid, v.pdl, s)
               : v.packed == 1 ? kpm_dispatch<float, OP_SELL, VM_PACKED>(p, grid, v.pdl, s)
               : v.real_values ? kpm_dispatch<float, OP_SELL, true>(p, grid, v.pdl, s)
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
// operator at the default shape (the stencil kernels hold more registers than
// the SELL ones).
int sweep_grid(const SweepVariant &v, int num_sms)
{
    SweepVariant d = v;
    d.block = kBlockB1;
    d.spw = 1;
    int per_sm = sweep_shape_occupancy(d, false);
    if (per_sm < 1) per_sm = 4;
    return per_sm * num_sms;
}

}  // namespace tbpm
