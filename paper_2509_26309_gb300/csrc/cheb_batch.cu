// Batched Clenshaw sweeps: 16 states advance together, FP32 vectors (complex64)
// and hoppings, FP64 coefficients and dot accumulation.
//
// The random initial states of the trace estimate are independent (the paper
// distributes them over MPI ranks, Sec. 2.4.2); here they share one pass over
// the operator. Vectors are interleaved [row][16] complex64, so one row of one
// vector is one 128-byte line: the product of a row reads each matrix entry
// once for all 16 states and gathers one line per neighbour. A block of 256
// threads covers one 32-row slice: 8 threads per row, 2 states (one float4)
// per thread. The sweep kinds and the Clenshaw update are those of
// cheb_sweep.cu (y = a psi + beta A x - z, with A = 2 H / rescale stored).
#include "tbpm_internal.cuh"
#include "sweep_ops.cuh"

#include <algorithm>

namespace tbpm {
namespace {

constexpr int kB = 16;                  // states per row
constexpr int kLanesPerRow = kB / 2;    // float4 = 2 complex64 per thread
constexpr int kRowsPerBlock = kBlock / kLanesPerRow;   // 32 = one slice

enum BMode { B_ONE = 0, B_REAL = 1, B_IMAG = 2 };

struct C2 { float r0, i0, r1, i1; };

__device__ __forceinline__ C2 ld4(const float2 *base, int64_t row, int pair)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(base + row * kB) + pair);
    return C2{v.x, v.y, v.z, v.w};
}

__device__ __forceinline__ C2 ld4_plain(const float2 *base, int64_t row, int pair)
{
    const float4 v = *(reinterpret_cast<const float4 *>(base + row * kB) + pair);
    return C2{v.x, v.y, v.z, v.w};
}

__device__ __forceinline__ void st4(float2 *base, int64_t row, int pair, const C2 &c)
{
    *(reinterpret_cast<float4 *>(base + row * kB) + pair) = make_float4(c.r0, c.i0, c.r1, c.i1);
}

__device__ __forceinline__ void fma4(float v, const C2 &x, C2 &acc)
{
    acc.r0 = fmaf(v, x.r0, acc.r0); acc.i0 = fmaf(v, x.i0, acc.i0);
    acc.r1 = fmaf(v, x.r1, acc.r1); acc.i1 = fmaf(v, x.i1, acc.i1);
}

// acc += A_offdiag x for one row (SELL or lattice stencil).
template <int OP, bool REALV>
__device__ __forceinline__ void apply_row(const SweepParams &p, int64_t s, int r_in_slice,
                                          int64_t row, int pair, const float2 *__restrict__ x,
                                          C2 &acc)
{
    if (OP == OP_SELL) {
        const int64_t off = __ldg(p.slice_off + s);
        const int w = (int)((__ldg(p.slice_off + s + 1) - off) >> 5);
        const int32_t *cp = p.cols + off + r_in_slice;
        if (REALV && (w == 3 || w == 4)) {
            // monolayer / bilayer rows: every column and value load first, then
            // the gathers, then the FMAs (one dependent round trip, not one per pair)
            const float *vp = reinterpret_cast<const float *>(p.vals) + off + r_in_slice;
            int c[4];
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < w) { c[j] = __ldg(cp + 32 * j); v[j] = __ldg(vp + 32 * j); }
            C2 xv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < w) xv[j] = ld4(x, c[j], pair);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < w) fma4(v[j], xv[j], acc);
        } else if (REALV) {
            const float *vp = reinterpret_cast<const float *>(p.vals) + off + r_in_slice;
            int j = 0;
            for (; j + 2 <= w; j += 2) {
                const int c0 = __ldg(cp + 32 * j), c1 = __ldg(cp + 32 * (j + 1));
                const float v0 = __ldg(vp + 32 * j), v1 = __ldg(vp + 32 * (j + 1));
                const C2 x0 = ld4(x, c0, pair), x1 = ld4(x, c1, pair);
                fma4(v0, x0, acc);
                fma4(v1, x1, acc);
            }
            if (j < w) {
                const int c0 = __ldg(cp + 32 * j);
                const float v0 = __ldg(vp + 32 * j);
                fma4(v0, ld4(x, c0, pair), acc);
            }
        } else {
            const float2 *vp = reinterpret_cast<const float2 *>(p.vals) + off + r_in_slice;
            for (int j = 0; j < w; ++j) {
                const int c0 = __ldg(cp + 32 * j);
                const float2 v = __ldg(vp + 32 * j);
                const C2 xx = ld4(x, c0, pair);
                acc.r0 = fmaf(v.x, xx.r0, fmaf(-v.y, xx.i0, acc.r0));
                acc.i0 = fmaf(v.x, xx.i0, fmaf(v.y, xx.r0, acc.i0));
                acc.r1 = fmaf(v.x, xx.r1, fmaf(-v.y, xx.i1, acc.r1));
                acc.i1 = fmaf(v.x, xx.i1, fmaf(v.y, xx.r1, acc.i1));
            }
        }
    } else {
        if (row >= p.n) return;
        // orbital counts are below 2^31: 32-bit index arithmetic
        const unsigned per = (OP == OP_STENCIL_MONO) ? 2u : 4u;
        const unsigned r = (unsigned)row, L1 = (unsigned)p.l1, L2 = (unsigned)p.l2;
        const unsigned cell = r / per;
        const unsigned o = r - cell * per;
        const unsigned m1 = cell / L2;
        const unsigned m2 = cell - m1 * L2;
        const unsigned base_o = o & 2u;
        unsigned n0, n1, n2;
        if ((o & 1u) == 0) {
            const unsigned mm1 = (m1 == 0) ? L1 - 1 : m1 - 1;
            const unsigned mm2 = (m2 == 0) ? L2 - 1 : m2 - 1;
            n0 = cell * per + base_o + 1;
            n1 = (mm1 * L2 + m2) * per + base_o + 1;
            n2 = (m1 * L2 + mm2) * per + base_o + 1;
        } else {
            const unsigned pm1 = (m1 == L1 - 1) ? 0 : m1 + 1;
            const unsigned pm2 = (m2 == L2 - 1) ? 0 : m2 + 1;
            n0 = cell * per + base_o;
            n1 = (pm1 * L2 + m2) * per + base_o;
            n2 = (m1 * L2 + pm2) * per + base_o;
        }
        const C2 x0 = ld4(x, n0, pair), x1 = ld4(x, n1, pair), x2 = ld4(x, n2, pair);
        const float t = (float)p.t;
        acc.r0 = fmaf(t, x0.r0 + x1.r0 + x2.r0, acc.r0);
        acc.i0 = fmaf(t, x0.i0 + x1.i0 + x2.i0, acc.i0);
        acc.r1 = fmaf(t, x0.r1 + x1.r1 + x2.r1, acc.r1);
        acc.i1 = fmaf(t, x0.i1 + x1.i1 + x2.i1, acc.i1);
        if (OP == OP_STENCIL_BI && (o == 0 || o == 3))
            fma4((float)p.t_perp, ld4(x, o == 0 ? cell * 4 + 3 : cell * 4, pair), acc);
    }
}

// Block sums of per-thread (state 2*pair, state 2*pair+1) complex pairs, in a
// fixed order: butterfly over the 4 rows of a warp, then warps in order.
// out[j] (j < 16) receives the block's sum for state j.
__device__ __forceinline__ void block_pairs(double ar, double ai, double br, double bi,
                                            double (*red)[kLanesPerRow][4], double2 *out)
{
#pragma unroll
    for (int o = kLanesPerRow; o < 32; o <<= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
        br += __shfl_xor_sync(0xffffffffu, br, o);
        bi += __shfl_xor_sync(0xffffffffu, bi, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kLanesPerRow) {
        red[w][lane][0] = ar; red[w][lane][1] = ai;
        red[w][lane][2] = br; red[w][lane][3] = bi;
    }
    __syncthreads();
    if (threadIdx.x < kB) {
        const int j = threadIdx.x, pr = j >> 1, h = (j & 1) * 2;
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) { sr += red[q][pr][h]; si += red[q][pr][h + 1]; }
        out[j] = make_double2(sr, si);
    }
    __syncthreads();
}

template <int OP, bool REALV, int BM, bool AIMAG, bool HASZ, bool FINAL>
__global__ void __launch_bounds__(kBlock) sweep_b16(SweepParams p)
{
    __shared__ double red[kBlock / 32][kLanesPerRow][4];
    const double2 ca = p.coef[p.ia];
    const double2 cb = p.ib >= 0 ? p.coef[p.ib] : make_double2(0.0, 0.0);
    const double araw = AIMAG ? (ca.y - cb.y) : (ca.x - cb.x);
    double braw = p.bscale;
    if (BM == B_REAL && p.ic >= 0) braw = p.bscale * p.coef[p.ic].x;
    if (BM == B_IMAG && p.ic >= 0) braw = p.bscale * p.coef[p.ic].y;

    const float2 *__restrict__ x = reinterpret_cast<const float2 *>(p.x);
    const float2 *psi = reinterpret_cast<const float2 *>(p.psi);
    const float2 *z = reinterpret_cast<const float2 *>(p.z);
    float2 *y = reinterpret_cast<float2 *>(p.y);
    const float2 *psi0 = reinterpret_cast<const float2 *>(p.psi0);
    const float *diag = reinterpret_cast<const float *>(p.diag);

    const int r_in = threadIdx.x / kLanesPerRow;       // row within the slice
    const int pair = threadIdx.x % kLanesPerRow;       // states 2*pair, 2*pair+1
    // renormalisation: 1/||psi_j|| folded into the coefficients on psi
    const double sc0 = p.scale ? p.scale[2 * pair] : 1.0;
    const double sc1 = p.scale ? p.scale[2 * pair + 1] : 1.0;
    const float a0 = (float)(sc0 * araw), a1 = (float)(sc1 * araw);
    const float beta0 = (float)(BM == B_ONE ? braw : sc0 * braw);
    const float beta1 = (float)(BM == B_ONE ? braw : sc1 * braw);
    double d0r = 0.0, d0i = 0.0, d1r = 0.0, d1i = 0.0, n0 = 0.0, n1 = 0.0;
    F2Sum f0r, f0i, f1r, f1i, g0, g1;   // the dots, summed on the FP32 pipe

    for (int64_t s = blockIdx.x; s < p.nslices; s += gridDim.x) {
        const int64_t row = s * 32 + r_in;
        const C2 ps = ld4_plain(psi, row, pair);
        C2 t;
        if (AIMAG) { t = C2{-a0 * ps.i0, a0 * ps.r0, -a1 * ps.i1, a1 * ps.r1}; }
        else { t = C2{a0 * ps.r0, a0 * ps.i0, a1 * ps.r1, a1 * ps.i1}; }
        if (HASZ) {
            const C2 zz = ld4_plain(z, row, pair);
            t.r0 -= zz.r0; t.i0 -= zz.i0; t.r1 -= zz.r1; t.i1 -= zz.i1;
        }
        const float d = diag ? __ldg(diag + row) : 0.0f;
        const C2 xi = ld4(x, row, pair);
        C2 acc;
        if (BM == B_ONE) { acc = t; fma4(d, xi, acc); }
        else { acc = C2{d * xi.r0, d * xi.i0, d * xi.r1, d * xi.i1}; }
        apply_row<OP, REALV>(p, s, r_in, row, pair, x, acc);
        C2 out;
        if (BM == B_ONE) out = acc;
        else if (BM == B_REAL)
            out = C2{fmaf(beta0, acc.r0, t.r0), fmaf(beta0, acc.i0, t.i0),
                     fmaf(beta1, acc.r1, t.r1), fmaf(beta1, acc.i1, t.i1)};
        else
            out = C2{fmaf(-beta0, acc.i0, t.r0), fmaf(beta0, acc.r0, t.i0),
                     fmaf(-beta1, acc.i1, t.r1), fmaf(beta1, acc.r1, t.i1)};
        st4(y, row, pair, out);
        if (FINAL) {
            const C2 q = ld4_plain(psi0, row, pair);
            f0r.add_dot(q.r0, out.r0, q.i0, out.i0);
            f0i.add_dot(q.r0, out.i0, -q.i0, out.r0);
            f1r.add_dot(q.r1, out.r1, q.i1, out.i1);
            f1i.add_dot(q.r1, out.i1, -q.i1, out.r1);
            if (p.norm_partials) {
                g0.add_dot(out.r0, out.r0, out.i0, out.i0);
                g1.add_dot(out.r1, out.r1, out.i1, out.i1);
            }
        }
    }
    if (FINAL) {
        d0r = f0r.value(); d0i = f0i.value(); d1r = f1r.value(); d1i = f1i.value();
        n0 = g0.value(); n1 = g1.value();
        block_pairs(d0r, d0i, d1r, d1i, red, p.partials + ((int64_t)p.delta * p.nblk + blockIdx.x) * kB);
        if (p.norm_partials)
            block_pairs(n0, 0.0, n1, 0.0, red,
                        p.norm_partials + ((int64_t)p.delta * p.nblk + blockIdx.x) * kB);
    }
}

template <int OP, bool REALV>
cudaError_t dispatch(SweepKind kind, bool a_imag, bool has_z, const SweepParams &p, int grid,
                     cudaStream_t s)
{
    switch (kind) {
    case SW_FIRST:
        if (a_imag) sweep_b16<OP, REALV, B_REAL, true, false, false><<<grid, kBlock, 0, s>>>(p);
        else sweep_b16<OP, REALV, B_IMAG, false, false, false><<<grid, kBlock, 0, s>>>(p);
        break;
    case SW_SECOND:
        if (a_imag) sweep_b16<OP, REALV, B_ONE, true, false, false><<<grid, kBlock, 0, s>>>(p);
        else sweep_b16<OP, REALV, B_ONE, false, false, false><<<grid, kBlock, 0, s>>>(p);
        break;
    case SW_MID:
        if (a_imag) sweep_b16<OP, REALV, B_ONE, true, true, false><<<grid, kBlock, 0, s>>>(p);
        else sweep_b16<OP, REALV, B_ONE, false, true, false><<<grid, kBlock, 0, s>>>(p);
        break;
    case SW_FINAL:
        if (has_z) sweep_b16<OP, REALV, B_REAL, false, true, true><<<grid, kBlock, 0, s>>>(p);
        else sweep_b16<OP, REALV, B_REAL, false, false, true><<<grid, kBlock, 0, s>>>(p);
        break;
    }
    return cudaGetLastError();
}

// Batched dot <a_j|b_j> for the 16 interleaved states: [nblk][16] partials.
__global__ void __launch_bounds__(kBlock) dot_b16(const float2 *a, const float2 *b, int64_t nslices,
                                                  double2 *partials)
{
    __shared__ double red[kBlock / 32][kLanesPerRow][4];
    const int r_in = threadIdx.x / kLanesPerRow, pair = threadIdx.x % kLanesPerRow;
    double d0r = 0.0, d0i = 0.0, d1r = 0.0, d1i = 0.0;
    for (int64_t s = blockIdx.x; s < nslices; s += gridDim.x) {
        const int64_t row = s * 32 + r_in;
        const C2 q = ld4_plain(a, row, pair), v = ld4_plain(b, row, pair);
        d0r = fma((double)q.r0, (double)v.r0, fma((double)q.i0, (double)v.i0, d0r));
        d0i = fma((double)q.r0, (double)v.i0, fma(-(double)q.i0, (double)v.r0, d0i));
        d1r = fma((double)q.r1, (double)v.r1, fma((double)q.i1, (double)v.i1, d1r));
        d1i = fma((double)q.r1, (double)v.i1, fma(-(double)q.i1, (double)v.r1, d1i));
    }
#pragma unroll
    for (int o = kLanesPerRow; o < 32; o <<= 1) {
        d0r += __shfl_xor_sync(0xffffffffu, d0r, o);
        d0i += __shfl_xor_sync(0xffffffffu, d0i, o);
        d1r += __shfl_xor_sync(0xffffffffu, d1r, o);
        d1i += __shfl_xor_sync(0xffffffffu, d1i, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < kLanesPerRow) {
        red[w][lane][0] = d0r; red[w][lane][1] = d0i;
        red[w][lane][2] = d1r; red[w][lane][3] = d1i;
    }
    __syncthreads();
    if (threadIdx.x < kB) {
        const int j = threadIdx.x, pr = j >> 1, h = (j & 1) * 2;
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) { sr += red[q][pr][h]; si += red[q][pr][h + 1]; }
        partials[(int64_t)blockIdx.x * kB + j] = make_double2(sr, si);
    }
}

// out[j * ld + base + offset + d] = sum_b partials[((d * nblk) + b) * 16 + j]:
// one warp per (slot, state), fixed order.
__global__ void reduce_b16(const double2 *partials, int nslot, int nblk, const int *counter,
                           int offset, double2 *out, int64_t ld)
{
    const int wid = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= nslot * kB) return;
    const int d = wid / kB, j = wid - d * kB;
    double re = 0.0, im = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = partials[((int64_t)d * nblk + b) * kB + j];
        re += v.x; im += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        const int base = counter ? *counter : 0;
        out[(int64_t)j * ld + base + offset + d] = make_double2(re, im);
    }
}

}  // namespace

cudaError_t launch_sweep_b16(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                             const SweepParams &p, int grid, cudaStream_t s)
{
    if (v.precision != TBPM_FP32 || v.states != kB) return cudaErrorInvalidValue;
    if (v.op == OP_SELL)
        return v.real_values ? dispatch<OP_SELL, true>(kind, a_imag, has_z, p, grid, s)
                             : dispatch<OP_SELL, false>(kind, a_imag, has_z, p, grid, s);
    if (v.op == OP_STENCIL_MONO) return dispatch<OP_STENCIL_MONO, true>(kind, a_imag, has_z, p, grid, s);
    return dispatch<OP_STENCIL_BI, true>(kind, a_imag, has_z, p, grid, s);
}

cudaError_t launch_dot_b16(const void *a, const void *b, int64_t nslices, double2 *partials,
                           int grid, cudaStream_t s)
{
    dot_b16<<<grid, kBlock, 0, s>>>(reinterpret_cast<const float2 *>(a),
                                    reinterpret_cast<const float2 *>(b), nslices, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_b16(const double2 *partials, int nslot, int nblk, const int *counter,
                              int offset, double2 *out, int64_t ld, cudaStream_t s)
{
    const int warps = nslot * kB;
    if (warps <= 0) return cudaSuccess;
    reduce_b16<<<(warps * 32 + 255) / 256, 256, 0, s>>>(partials, nslot, nblk, counter, offset, out, ld);
    return cudaGetLastError();
}

int sweep_grid_b16(int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, sweep_b16<OP_SELL, true, B_ONE, false, true, false>, kBlock, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 4;
    return per_sm * num_sms;
}

// The final sweep holds more registers (the FP64 dots of 16 states) than the
// others: one wave of its own occupancy for this operator, at most `grid`.
int sweep_grid_b16_final(const SweepVariant &v, int num_sms, int grid)
{
    int per_sm = 0;
    cudaError_t e;
    if (v.op == OP_SELL)
        e = v.real_values ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &per_sm, sweep_b16<OP_SELL, true, B_REAL, false, true, true>, kBlock, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &per_sm, sweep_b16<OP_SELL, false, B_REAL, false, true, true>, kBlock, 0);
    else if (v.op == OP_STENCIL_MONO)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, sweep_b16<OP_STENCIL_MONO, true, B_REAL, false, true, true>, kBlock, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, sweep_b16<OP_STENCIL_BI, true, B_REAL, false, true, true>, kBlock, 0);
    if (e != cudaSuccess || per_sm < 1) return grid;
    return std::min(grid, per_sm * num_sms);
}

}  // namespace tbpm
