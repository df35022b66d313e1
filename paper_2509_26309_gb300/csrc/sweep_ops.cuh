// Device helpers shared by the sweep kernels: the per-row sparse (SELL) and
// stencil products A x and a fixed-order warp sum.
#pragma once

#include "tbpm_internal.cuh"

namespace tbpm {
namespace ops {

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

// Matrix streams are read once per sweep. For FP32 they are loaded with the
// streaming (evict-first) cache operator so that they do not push the vectors,
// which the next sweep reads again, out of L2; the FP64 sweeps are bound by the
// FP64 pipe and keep the default policy.
template <typename R, typename T>
__device__ __forceinline__ T ldm(const T *p)
{
    if (sizeof(R) == 4) return __ldcs(p);
    return __ldg(p);
}

// How a SELL operator's entries are stored (the VM template argument):
// VM_COMPLEX and VM_REAL: int32 columns and complex or real values; VM_PACKED
// (real values, FP32): for each entry a 16-bit column offset from its row,
// taken modulo the padded row count, and an 8-bit index into a table of at
// most 256 distinct values (3 B per entry instead of 8 for lattice-like
// matrices, whose neighbours sit at a few fixed offsets and whose hoppings take
// a few values). VM_ROWS (real values, FP32, every slice of width 3, at most
// 32 values): one 64-bit word per row holding the row's three 16-bit column
// offsets (bits 0-47) and three 5-bit value indices (bits 48-62), so that a row
// costs one load and no slice extents are read. The entries, and so the
// products, are the same in every form.
enum ValueMode { VM_COMPLEX = 0, VM_REAL = 1, VM_PACKED = 2, VM_ROWS = 3 };

// One stored entry: acc += v x[c] (real v) or v x[c] (complex v).
template <typename R, int VM>
struct SellEntry {
    typedef typename V2<R>::T V;
    int c;
    R v;
    __device__ __forceinline__ void apply(const V &xv, R &ar, R &ai) const
    {
        ar = fma(v, xv.x, ar);
        ai = fma(v, xv.y, ai);
    }
};
template <typename R>
struct SellEntry<R, VM_COMPLEX> {
    typedef typename V2<R>::T V;
    int c;
    V v;
    __device__ __forceinline__ void apply(const V &xv, R &ar, R &ai) const
    {
        ar = fma(v.x, xv.x, fma(-v.y, xv.y, ar));
        ai = fma(v.x, xv.y, fma(v.y, xv.x, ai));
    }
};

// The entries of one lane's row in a slice starting at entry `off`: entry j at
// off + 32 j + lane.
template <typename R, int VM>
struct SellRow {
    typedef typename V2<R>::T V;
    const int32_t *cp;
    const void *vp;
    __device__ __forceinline__ void init(const SweepParams &p, int64_t off, int lane, int64_t)
    {
        cp = p.cols + off + lane;
        vp = VM == VM_REAL ? (const void *)(reinterpret_cast<const R *>(p.vals) + off + lane)
                           : (const void *)(reinterpret_cast<const V *>(p.vals) + off + lane);
    }
    __device__ __forceinline__ void load(SellEntry<R, VM> &e, int j) const
    {
        e.c = ldm<R>(cp + 32 * (int64_t)j);
        if constexpr (VM == VM_REAL) e.v = ldm<R>(reinterpret_cast<const R *>(vp) + 32 * (int64_t)j);
        else e.v = ldm<R>(reinterpret_cast<const V *>(vp) + 32 * (int64_t)j);
    }
};
template <typename R>
struct SellRow<R, VM_PACKED> {
    const int16_t *dp;
    const uint8_t *ip;
    const R *tab;
    int row, npad;
    __device__ __forceinline__ void init(const SweepParams &p, int64_t off, int lane, int64_t r)
    {
        dp = p.cdelta + off + lane;
        ip = p.vidx + off + lane;
        tab = reinterpret_cast<const R *>(p.vtab);
        row = (int)r;
        npad = (int)p.npad;
    }
    __device__ __forceinline__ void load(SellEntry<R, VM_PACKED> &e, int j) const
    {
        int c = row + (int)ldm<R>(dp + 32 * (int64_t)j);
        c = c < 0 ? c + npad : c;
        e.c = c >= npad ? c - npad : c;
        e.v = __ldg(tab + ldm<R>(ip + 32 * (int64_t)j));
    }
};

template <typename R>
struct SellRow<R, VM_ROWS> {
    uint64_t word;
    const R *tab;
    int row, npad;
    __device__ __forceinline__ void init(const SweepParams &p, int64_t, int, int64_t r)
    {
        word = ldm<R>(p.rowpack + r);
        tab = reinterpret_cast<const R *>(p.vtab);
        row = (int)r;
        npad = (int)p.npad;
    }
    __device__ __forceinline__ void load(SellEntry<R, VM_ROWS> &e, int j) const
    {
        int c = row + (int)(int16_t)(uint16_t)(word >> (16 * j));
        c = c < 0 ? c + npad : c;
        e.c = c >= npad ? c - npad : c;
        e.v = __ldg(tab + (int)((word >> (48 + 5 * j)) & 31u));
    }
};

// N entries j0 .. j0+N-1 of the lane's row: all loads first, then the FMAs.
template <typename R, int VM, int N>
__device__ __forceinline__ void sell_entries(const SellRow<R, VM> &rr, int j0,
                                             const typename V2<R>::T *__restrict__ x, R &ar, R &ai)
{
    typedef typename V2<R>::T V;
    SellEntry<R, VM> e[N];
#pragma unroll
    for (int q = 0; q < N; ++q) rr.load(e[q], j0 + q);
    V xv[N];
#pragma unroll
    for (int q = 0; q < N; ++q) xv[q] = __ldg(x + e[q].c);
#pragma unroll
    for (int q = 0; q < N; ++q) e[q].apply(xv[q], ar, ai);
}

// acc = A x for row `row` of a SELL slice, accumulated onto (ar, ai).
// The slice width w is uniform across the warp. Widths 3 and 4 (monolayer and
// AB-bilayer rows with the diagonal stored apart) run as straight-line code;
// other widths as groups of 4 and a plain remainder loop. No code path issues
// instructions for entries past w: a predicated-off FP64 instruction still
// takes its slot in GB300's narrow FP64 pipe.
template <typename R, int VM>
__device__ __forceinline__ void sell_apply(const SweepParams &p, int64_t s, int lane,
                                           const typename V2<R>::T *__restrict__ x,
                                           R &ar, R &ai)
{
    if constexpr (VM == VM_ROWS) {          // every slice has width 3: no extents to read
        SellRow<R, VM_ROWS> rr;
        rr.init(p, 0, lane, (s << 5) + lane);
        sell_entries<R, VM_ROWS, 3>(rr, 0, x, ar, ai);
        return;
    }
    const int64_t off = ldm<R>(p.slice_off + s);
    const int w = (int)((ldm<R>(p.slice_off + s + 1) - off) >> 5);
    SellRow<R, VM> rr;
    rr.init(p, off, lane, (s << 5) + lane);
    if (w == 3) {
        sell_entries<R, VM, 3>(rr, 0, x, ar, ai);
    } else if (w == 4) {
        sell_entries<R, VM, 4>(rr, 0, x, ar, ai);
    } else {
        int j = 0;
        for (; j + 4 <= w; j += 4) sell_entries<R, VM, 4>(rr, j, x, ar, ai);
#pragma unroll 1
        for (; j < w; ++j) sell_entries<R, VM, 1>(rr, j, x, ar, ai);
    }
}

// acc = A x - (on-site part excluded) for a periodic lattice row, onto (ar, ai).
// Monolayer, row = 2 cell + s, cell = m1 L2 + m2:
//   A(m) couples to B(m), B(m - a1), B(m - a2); B(m) to A(m), A(m + a1), A(m + a2).
// Bilayer, row = 4 cell + o (o = A1, B1, A2, B2): each layer as above, plus the
// dimer bond A1(m) - B2(m).
template <typename R, int OP>
__device__ __forceinline__ void stencil_apply(const SweepParams &p, int64_t row,
                                              const typename V2<R>::T *__restrict__ x,
                                              R &ar, R &ai)
{
    typedef typename V2<R>::T V;
    // orbital counts are below 2^31, so the index arithmetic is 32-bit
    const unsigned per = (OP == OP_STENCIL_MONO) ? 2u : 4u;
    const unsigned r = (unsigned)row, L1 = (unsigned)p.l1, L2 = (unsigned)p.l2;
    const unsigned cell = r / per;
    const unsigned o = r - cell * per;
    const unsigned m1 = cell / L2;
    const unsigned m2 = cell - m1 * L2;
    const unsigned base_o = o & 2u;                     // orbital of A in this layer
    unsigned n0, n1, n2;                                // the three in-layer neighbours
    if ((o & 1u) == 0) {                                // A: B(m), B(m-a1), B(m-a2)
        const unsigned mm1 = (m1 == 0) ? L1 - 1 : m1 - 1;
        const unsigned mm2 = (m2 == 0) ? L2 - 1 : m2 - 1;
        n0 = cell * per + base_o + 1;
        n1 = (mm1 * L2 + m2) * per + base_o + 1;
        n2 = (m1 * L2 + mm2) * per + base_o + 1;
    } else {                                            // B: A(m), A(m+a1), A(m+a2)
        const unsigned pm1 = (m1 == L1 - 1) ? 0 : m1 + 1;
        const unsigned pm2 = (m2 == L2 - 1) ? 0 : m2 + 1;
        n0 = cell * per + base_o;
        n1 = (pm1 * L2 + m2) * per + base_o;
        n2 = (m1 * L2 + pm2) * per + base_o;
    }
    const V x0 = __ldg(x + n0), x1 = __ldg(x + n1), x2 = __ldg(x + n2);
    const R t = (R)p.t;
    ar = fma(t, x0.x + x1.x + x2.x, ar);
    ai = fma(t, x0.y + x1.y + x2.y, ai);
    if (OP == OP_STENCIL_BI && (o == 0 || o == 3)) {
        const V xd = __ldg(x + (o == 0 ? cell * 4 + 3 : cell * 4));
        const R tp = (R)p.t_perp;
        ar = fma(tp, xd.x, ar);
        ai = fma(tp, xd.y, ai);
    }
}

// Long sums of FP32 terms at about twice FP32's precision, on the FP32 pipe:
// GB300 issues FP64 at a small fraction of its FP32 rate, so the FP32 kernels
// do not convert every element to FP64 for their dots. Each term (one
// component of a complex product, a1 b1 + a2 b2, formed by one FMA in FP32 as
// the FP32 data it comes from) is added to the running (hi, lo) pair by Knuth's
// two-sum, so the summation itself loses nothing; the pair is converted to
// FP64 once, when the partial leaves the thread. The _rn intrinsics keep the
// compiler from contracting or reordering the two-sum.
struct F2Sum {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        const float s = __fadd_rn(hi, v);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    // += a1 b1 + a2 b2
    __device__ __forceinline__ void add_dot(float a1, float b1, float a2, float b2) { add(fmaf(a1, b1, a2 * b2)); }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Warp sum of a two-sum pair in FP32 (a butterfly of two-sums); lane 0 holds
// the warp's result.
__device__ __forceinline__ void warp_sum_f2(F2Sum &a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, a.hi, o);
        const float l = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a.add(h);
        a.lo = __fadd_rn(a.lo, l);
    }
}

// Block sum of NV two-sum pairs for blocks of up to 1024 threads, in FP32 up
// to one FP64 conversion per value; the results are valid in thread 0. Every
// thread of the block calls it.
template <int NV>
__device__ __forceinline__ void block_sum_f2(F2Sum (&a)[NV], double (&out)[NV])
{
    __shared__ float2 sm[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        warp_sum_f2(a[v]);
        if (lane == 0) sm[v][w] = make_float2(a[v].hi, a[v].lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            F2Sum t;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                t.add(sm[v][i].x);
                t.lo = __fadd_rn(t.lo, sm[v][i].y);
            }
            out[v] = t.value();
        }
    }
}

// Warp-wide sum in a fixed butterfly order; every lane gets the result.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace ops
using namespace ops;
}  // namespace tbpm
