// The single-state Clenshaw sweep kernel (B = 1), templated on its launch
// shape so that the autotuner can pick the block width and the number of
// 32-row slices a warp works on at once. cheb_sweep.cu instantiates the
// default shape (one slice per warp iteration, blocks of up to 512 threads)
// for every operator; cheb_sweep_s*.cu instantiate the other shapes for
// the stored-matrix (SELL) operator. The recurrence each sweep kind computes is
// described in cheb_sweep.cu.
#pragma once

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

// G slices of uniform SELL width N: every column and value load of the G rows
// is issued first, then every gather, then the FMAs of each row in entry
// order (the same order as sell_apply, so results do not depend on G).
template <typename R, int VM, int N, int G>
__device__ __forceinline__ void sell_group(const SweepParams &p, const int64_t (&off)[G], int64_t s0, int lane,
                                           const typename V2<R>::T *__restrict__ x, R (&ar)[G], R (&ai)[G])
{
    typedef typename V2<R>::T V;
    SellEntry<R, VM> e[G][N];
#pragma unroll
    for (int q = 0; q < G; ++q) {
        SellRow<R, VM> rr;
        rr.init(p, off[q], lane, ((s0 + q) << 5) + lane);
#pragma unroll
        for (int j = 0; j < N; ++j) rr.load(e[q][j], j);
    }
    V xv[G][N];
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
        for (int j = 0; j < N; ++j) xv[q][j] = __ldg(x + e[q][j].c);
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
        for (int j = 0; j < N; ++j) e[q][j].apply(xv[q][j], ar[q], ai[q]);
}

// One Clenshaw sweep for a single state per row (B = 1). A warp owns SPW
// consecutive 32-row slices at a time (grid-stride over groups of SPW slices);
// for SPW > 1 (stored matrix only) every load of a group is issued before its
// arithmetic, so that a warp keeps SPW times as many loads in flight. LB is
// the largest block width the kernel is compiled for (its launch bound).
// The final sweep accumulates <psi0|y> (and ||y||^2 when renormalising) per
// lane in FP64 across the warp's slices and reduces once per warp, at the end,
// into partials[delta * W + warp] (W = warps in the grid, fixed per context):
// FP64 is GB300's scarce pipe, and a butterfly per slice would cost as many FP64
// instructions as the sparse product. For a batch of instances (MULTI) the
// coefficients are those of each slice's instance and the partials are stored
// per slice, partials[delta * nslices + slice], so that instances stay apart:
// a warp sums its consecutive visits to one instance's slices per lane and
// writes the run's sum to the slot of the run's first slice (zeros to the
// others), one butterfly per run instead of one per slice.
// Each row's arithmetic is the same for every shape; only the grouping of the
// dot partials follows the grid. NORM (final sweeps when renormalising) adds the
// sum of |y|^2: a compile-time choice, since a run-time test on norm_partials
// let the compiler form the two FP64 FMAs of every row unconditionally.
template <typename R, int OP, int VM, int BM, bool AIMAG, bool HASZ, bool FINAL, bool MULTI, int SPW, int LB,
          bool NORM = false>
__global__ void __launch_bounds__(LB) sweep_b1(SweepParams p)
{
    typedef typename V2<R>::T V;
    static_assert(SPW == 1 || OP == OP_SELL, "slice groups are built for the stored matrix");
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
    // batch final sweep: the warp's dot sums run over consecutive visits to
    // slices of one instance; the run's sum goes to the slot of its first
    // slice, and every other visited slice's slot gets zero
    int64_t run_slot = -1;
    int run_inst = -1;
    auto flush_run = [&]() {
        const double sr = warp_sum(dr), si = warp_sum(di);
        if (lane == 0) p.partials[(int64_t)p.delta * p.nslices + run_slot] = make_double2(sr, si);
        if constexpr (NORM) {
            const double sn = warp_sum(nn);
            if (lane == 0) p.norm_partials[(int64_t)p.delta * p.nslices + run_slot] = make_double2(sn, 0.0);
        }
        dr = di = nn = 0.0;
        run_slot = -1;
    };
    // t = a psi - z of row `row` (a real: a*psi; a imaginary: i*a*psi), one FMA per part
    auto first_terms = [&](const V &ps, const V &zz, R &tr, R &ti) {
        if (HASZ) {
            if (AIMAG) { tr = fma(-a, ps.y, -zz.x); ti = fma(a, ps.x, -zz.y); }
            else { tr = fma(a, ps.x, -zz.x); ti = fma(a, ps.y, -zz.y); }
        } else {
            if (AIMAG) { tr = -a * ps.y; ti = a * ps.x; } else { tr = a * ps.x; ti = a * ps.y; }
        }
    };
    // y = beta (A x) + t, the dot terms, and the store
    auto finish = [&](int64_t s, int64_t row, int inst, R ar, R ai, R tr, R ti) {
        V out;
        if (BM == B_ONE) { out.x = ar; out.y = ai; }
        else if (BM == B_REAL) { out.x = fma(beta, ar, tr); out.y = fma(beta, ai, ti); }
        else { out.x = fma(-beta, ai, tr); out.y = fma(beta, ar, ti); }
        y[row] = out;
        if (FINAL && kF32 && !MULTI) {
            const V q = psi0[row];
            fr.add_dot((float)q.x, (float)out.x, (float)q.y, (float)out.y);
            fi.add_dot((float)q.x, (float)out.y, -(float)q.y, (float)out.x);
            if constexpr (NORM) fn.add_dot((float)out.x, (float)out.x, (float)out.y, (float)out.y);
        } else if (FINAL) {
            const V q = psi0[row];
            const double qr = (double)q.x, qi = (double)q.y;
            const double orr = (double)out.x, oi = (double)out.y;
            if (MULTI) {
                if (run_slot >= 0 && inst != run_inst) flush_run();
                if (run_slot < 0) {
                    run_slot = s;
                    run_inst = inst;
                } else if (lane == 0) {
                    p.partials[(int64_t)p.delta * p.nslices + s] = make_double2(0.0, 0.0);
                    if constexpr (NORM) p.norm_partials[(int64_t)p.delta * p.nslices + s] = make_double2(0.0, 0.0);
                }
            }
            dr = fma(qr, orr, fma(qi, oi, dr));
            di = fma(qr, oi, fma(-qi, orr, di));
            if constexpr (NORM) nn = fma(orr, orr, fma(oi, oi, nn));
        }
    };
    // one slice on its own (every operator; the tail of a group)
    auto one_slice = [&](int64_t s) {
        if (MULTI) {                    // instances span many slices: recompute on a change only
            const int g = __ldg(p.slice_inst + s);
            if (g != cur_inst) {
                sweep_coeffs<R, BM, AIMAG>(p, g, a, beta);
                cur_inst = g;
            }
        }
        const int64_t row = (s << 5) + lane;
        const V ps = psi[row];
        V zz = V();
        if (HASZ) zz = z[row];
        R tr, ti;
        first_terms(ps, zz, tr, ti);
        const V xi = __ldg(x + row);
        const R d = diag ? ldm<R>(diag + row) : (R)0;
        R ar, ai;
        if (BM == B_ONE) { ar = fma(d, xi.x, tr); ai = fma(d, xi.y, ti); }
        else { ar = d * xi.x; ai = d * xi.y; }
        if (OP == OP_SELL) sell_apply<R, VM>(p, s, lane, x, ar, ai);
        else if (row < p.n) stencil_apply<R, OP>(p, row, x, ar, ai);
        finish(s, row, cur_inst, ar, ai, tr, ti);
    };

    if constexpr (SPW == 1) {
        for (int64_t s = warp; s < p.nslices; s += nwarps) one_slice(s);
    } else {
    for (int64_t s0 = warp * SPW; s0 < p.nslices; s0 += nwarps * SPW) {
        if (s0 + SPW > p.nslices) {     // ragged last group
            for (int q = 0; q < SPW && s0 + q < p.nslices; ++q) one_slice(s0 + q);
            continue;
        }
        // a full group of SPW slices: the row operands and slice extents first
        int64_t off[SPW] = {};
        int w0 = 3;
        bool same = true;
        if constexpr (VM != VM_ROWS) {      // VM_ROWS: every slice has width 3
            w0 = 0;
            int64_t lo = ldm<R>(p.slice_off + s0);
#pragma unroll
            for (int q = 0; q < SPW; ++q) {
                const int64_t hi = ldm<R>(p.slice_off + s0 + q + 1);
                const int w = (int)((hi - lo) >> 5);
                off[q] = lo;
                if (q == 0) w0 = w;
                same = same && (w == w0);
                lo = hi;
            }
        }
        if (!same || (w0 != 3 && w0 != 4)) {   // mixed or other widths: slice by slice
#pragma unroll
            for (int q = 0; q < SPW; ++q) one_slice(s0 + q);
            continue;
        }
        V ps[SPW], zz[SPW], xi[SPW];
        R d[SPW];
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
            const int64_t row = ((s0 + q) << 5) + lane;
            ps[q] = psi[row];
            zz[q] = HASZ ? z[row] : V();
            xi[q] = __ldg(x + row);
            d[q] = diag ? ldm<R>(diag + row) : (R)0;
        }
        R ar[SPW], ai[SPW], tr[SPW], ti[SPW], aq[SPW], bq[SPW];
        int gq[SPW];
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
            if (MULTI) {
                const int g = __ldg(p.slice_inst + s0 + q);
                if (g != cur_inst) {
                    sweep_coeffs<R, BM, AIMAG>(p, g, a, beta);
                    cur_inst = g;
                }
            }
            aq[q] = a;
            bq[q] = beta;
            gq[q] = cur_inst;
            first_terms(ps[q], zz[q], tr[q], ti[q]);
            if (BM == B_ONE) { ar[q] = fma(d[q], xi[q].x, tr[q]); ai[q] = fma(d[q], xi[q].y, ti[q]); }
            else { ar[q] = d[q] * xi[q].x; ai[q] = d[q] * xi[q].y; }
        }
        if (w0 == 3) sell_group<R, VM, 3, SPW>(p, off, s0, lane, x, ar, ai);
        else sell_group<R, VM, 4, SPW>(p, off, s0, lane, x, ar, ai);
#pragma unroll
        for (int q = 0; q < SPW; ++q) {
            a = aq[q];
            beta = bq[q];
            finish(s0 + q, ((s0 + q) << 5) + lane, gq[q], ar[q], ai[q], tr[q], ti[q]);
        }
    }
    }
    if (FINAL && MULTI) {
        if (run_slot >= 0) flush_run();
    } else if (FINAL && kF32) {
        // FP32 data: the block's sums in FP32 pairs, one conversion per value; the
        // block's first warp slot holds them, its other warp slots zero
        F2Sum sums[3] = {fr, fi, fn};
        double v[3];
        block_sum_f2<3>(sums, v);
        if (lane == 0) {
            const bool lead = (threadIdx.x >> 5) == 0;
            p.partials[(int64_t)p.delta * nwarps + warp] = lead ? make_double2(v[0], v[1]) : make_double2(0.0, 0.0);
            if constexpr (NORM)
                p.norm_partials[(int64_t)p.delta * nwarps + warp] = make_double2(lead ? v[2] : 0.0, 0.0);
        }
    } else if (FINAL) {
        dr = warp_sum(dr);
        di = warp_sum(di);
        if (lane == 0) p.partials[(int64_t)p.delta * nwarps + warp] = make_double2(dr, di);
        if constexpr (NORM) {
            nn = warp_sum(nn);
            if (lane == 0) p.norm_partials[(int64_t)p.delta * nwarps + warp] = make_double2(nn, 0.0);
        }
    }
}

// Launches one sweep kind of one operator variant at shape (SPW, LB) with
// `block` threads per block (block <= LB, a multiple of 32).
template <typename R, int OP, int VM, bool MULTI, int SPW, int LB>
cudaError_t sweep_dispatch(SweepKind kind, bool a_imag, bool has_z, const SweepParams &p,
                           int grid, int block, bool pdl, cudaStream_t s)
{
    switch (kind) {
    case SW_FIRST:
        return a_imag ? launch_pdl(sweep_b1<R, OP, VM, B_REAL, true, false, false, MULTI, SPW, LB>, grid, block, pdl, s, p)
                      : launch_pdl(sweep_b1<R, OP, VM, B_IMAG, false, false, false, MULTI, SPW, LB>, grid, block, pdl, s, p);
    case SW_SECOND:
        return a_imag ? launch_pdl(sweep_b1<R, OP, VM, B_ONE, true, false, false, MULTI, SPW, LB>, grid, block, pdl, s, p)
                      : launch_pdl(sweep_b1<R, OP, VM, B_ONE, false, false, false, MULTI, SPW, LB>, grid, block, pdl, s, p);
    case SW_MID:
        return a_imag ? launch_pdl(sweep_b1<R, OP, VM, B_ONE, true, true, false, MULTI, SPW, LB>, grid, block, pdl, s, p)
                      : launch_pdl(sweep_b1<R, OP, VM, B_ONE, false, true, false, MULTI, SPW, LB>, grid, block, pdl, s, p);
    case SW_FINAL:
        // the sum of |y|^2 is formed only when renormalising (norm_partials set)
        if (p.norm_partials)
            return has_z ? launch_pdl(sweep_b1<R, OP, VM, B_REAL, false, true, true, MULTI, SPW, LB, true>, grid, block, pdl, s, p)
                         : launch_pdl(sweep_b1<R, OP, VM, B_REAL, false, false, true, MULTI, SPW, LB, true>, grid, block, pdl, s, p);
        return has_z ? launch_pdl(sweep_b1<R, OP, VM, B_REAL, false, true, true, MULTI, SPW, LB>, grid, block, pdl, s, p)
                     : launch_pdl(sweep_b1<R, OP, VM, B_REAL, false, false, true, MULTI, SPW, LB>, grid, block, pdl, s, p);
    }
    return cudaErrorInvalidValue;
}

// Resident blocks per SM of one sweep kind at this shape (the fewest over the
// kind's forms: c_k real or imaginary; the final sweep with b_2, the form of
// every final sweep but K = 3's; SW_FINAL_NORM: the same with the norm).
template <typename R, int OP, int VM, bool MULTI, int SPW, int LB>
int sweep_occupancy_of(int block, int kind = SW_MID)
{
    auto occ = [block](auto kernel) {
        int per_sm = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) == cudaSuccess ? per_sm : 0;
    };
    switch (kind) {
    case SW_FIRST:
        return std::min(occ(sweep_b1<R, OP, VM, B_REAL, true, false, false, MULTI, SPW, LB>),
                        occ(sweep_b1<R, OP, VM, B_IMAG, false, false, false, MULTI, SPW, LB>));
    case SW_SECOND:
        return std::min(occ(sweep_b1<R, OP, VM, B_ONE, true, false, false, MULTI, SPW, LB>),
                        occ(sweep_b1<R, OP, VM, B_ONE, false, false, false, MULTI, SPW, LB>));
    case SW_FINAL:
        return occ(sweep_b1<R, OP, VM, B_REAL, false, true, true, MULTI, SPW, LB>);
    case SW_FINAL_NORM:
        return occ(sweep_b1<R, OP, VM, B_REAL, false, true, true, MULTI, SPW, LB, true>);
    default:
        return occ(sweep_b1<R, OP, VM, B_ONE, false, true, false, MULTI, SPW, LB>);
    }
}

// The stored-matrix sweeps of one shape, for every precision, value kind and
// single or batched instance: one function per shape, defined by the
// translation unit that instantiates it.
template <int SPW, int LB>
cudaError_t sell_shape_launch(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                              const SweepParams &p, int grid, cudaStream_t s)
{
    const bool multi = p.slice_inst != nullptr;
    if (v.precision == TBPM_FP64) {
        if (multi)
            return v.real_values ? sweep_dispatch<double, OP_SELL, true, true, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s)
                                 : sweep_dispatch<double, OP_SELL, false, true, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s);
        return v.real_values ? sweep_dispatch<double, OP_SELL, true, false, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s)
                             : sweep_dispatch<double, OP_SELL, false, false, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s);
    }
    if (multi)
        return v.real_values ? sweep_dispatch<float, OP_SELL, true, true, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s)
                             : sweep_dispatch<float, OP_SELL, false, true, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s);
    if (v.packed == 2)      // the packed forms: FP32 real values of a single instance
        return sweep_dispatch<float, OP_SELL, VM_ROWS, false, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s);
    if (v.packed == 1)
        return sweep_dispatch<float, OP_SELL, VM_PACKED, false, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s);
    return v.real_values ? sweep_dispatch<float, OP_SELL, true, false, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s)
                         : sweep_dispatch<float, OP_SELL, false, false, SPW, LB>(kind, a_imag, has_z, p, grid, v.block, v.pdl, s);
}

template <int SPW, int LB>
int sell_shape_occupancy(const SweepVariant &v, bool multi, int kind)
{
    if (v.precision == TBPM_FP64) {
        if (multi)
            return v.real_values ? sweep_occupancy_of<double, OP_SELL, true, true, SPW, LB>(v.block, kind)
                                 : sweep_occupancy_of<double, OP_SELL, false, true, SPW, LB>(v.block, kind);
        return v.real_values ? sweep_occupancy_of<double, OP_SELL, true, false, SPW, LB>(v.block, kind)
                             : sweep_occupancy_of<double, OP_SELL, false, false, SPW, LB>(v.block, kind);
    }
    if (multi)
        return v.real_values ? sweep_occupancy_of<float, OP_SELL, true, true, SPW, LB>(v.block, kind)
                             : sweep_occupancy_of<float, OP_SELL, false, true, SPW, LB>(v.block, kind);
    if (v.packed == 2) return sweep_occupancy_of<float, OP_SELL, VM_ROWS, false, SPW, LB>(v.block, kind);
    if (v.packed == 1) return sweep_occupancy_of<float, OP_SELL, VM_PACKED, false, SPW, LB>(v.block, kind);
    return v.real_values ? sweep_occupancy_of<float, OP_SELL, true, false, SPW, LB>(v.block, kind)
                         : sweep_occupancy_of<float, OP_SELL, false, false, SPW, LB>(v.block, kind);
}

}  // namespace
}  // namespace tbpm
