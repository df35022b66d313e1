// Temporal blocking of the Clenshaw sweeps on the matrix-free monolayer
// graphene lattice (FP32 vectors, one state).
//
// Each Chebyshev term needs only the nearest neighbours of the previous term
// (the hopping convention of Sec. 3.2.1: A(m) couples to B(m), B(m - a1),
// B(m - a2)), so several consecutive sweeps of one time step can run on a
// tile of the lattice held on chip, with a halo that the sweeps eat into: HBM
// then carries each term's vectors once per block of kTbS sweeps instead of
// once per sweep. This is the per-term HBM floor the sparse product of
// Sec. 2.2.1 sits on, broken for the structured lattice only.
//
// Layout on chip. A tile region is kTbW1 rows (m1) by 32 cells (m2). Lane l of
// every warp owns cell m2 = o2 + l; warp w owns kTbR consecutive rows. Each
// thread keeps both orbitals (A, B) of its cells in registers: psi, the
// on-site energies, b_{k+1} and b_{k+2}. The neighbours B(m - a2) and
// A(m + a2) are one lane away (warp shuffles), B(m - a1) and A(m + a1) one row
// away (the thread's own registers, or, across a warp boundary, a row that
// each warp publishes in shared memory once per sweep). Lanes at the region's
// left and right edges and rows at its top and bottom read stand-in values:
// those cells are halo.
//
// A block of S sweeps loads psi(t_n), b_{k+1}, b_{k+2} and the on-site
// energies for its region (cp.async into a per-thread staging area while the
// previous tile computes), runs the S sweeps, and stores the interior of its
// last two b's (or, for the block holding the final sweep, psi(t_{n+1}) and
// the <psi0|psi> partials). A-sites lose valid cells on the low side of each
// axis in odd sweeps and on the high side in even ones, B-sites the reverse,
// so after S sweeps both sublattices are valid ceil(S/2) cells inside the
// region: kTbH = ceil(kTbS/2). Blocks read one pair of global b buffers and
// write another, and the final block writes psi(t_{n+1}) to a second state
// buffer: halo loads of other tiles never race with stores.
#include "tbpm_internal.cuh"
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

constexpr int kTbH = (kTbS + 1) / 2;            // halo cells per side
constexpr int kTbWarps = kTbThreads / 32;
constexpr int kTbR = 3;                         // rows per warp
constexpr int kTbW1 = kTbWarps * kTbR;          // region rows (m1)
constexpr int kTbW2 = 32;                       // region cells along m2 (one per lane)
constexpr int kTbT1 = kTbW1 - 2 * kTbH;         // interior rows
constexpr int kTbT2 = kTbW2 - 2 * kTbH;         // interior cells along m2

// Shared memory: the staging area (per thread and row: psi, b_{k+1}, b_{k+2}
// as float4 = (A, B), on-site as float2), then the boundary rows each warp
// publishes per sweep (its first row's A, its last row's B), double-buffered.
constexpr size_t kTbStageBytes = (size_t)kTbThreads * kTbR * (3 * sizeof(float4) + sizeof(float2));
constexpr size_t kTbExchBytes = (size_t)2 * 2 * kTbWarps * 32 * sizeof(float2);
constexpr size_t kTbSmem = kTbStageBytes + kTbExchBytes;
static_assert(kTbSmem <= 227 * 1024, "shared memory per block");

// m mod L for m in [-L, 2L) by one compare (the usual case: regions no larger
// than the lattice), by a division otherwise.
__device__ __forceinline__ int wrap(int m, int L)
{
    if (m < 0) m += L;
    else if (m >= L) m -= L;
    if ((unsigned)m >= (unsigned)L) {
        m %= L;
        if (m < 0) m += L;
    }
    return m;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// This thread's staging slots (row r at [r * kTbThreads]).
struct Stage {
    float4 *ps, *bx, *bz;
    float2 *on;
};

// The cells (row o1 + r0 + r, column o2 + lane) of a tile, as the index of
// their A orbital in float4 units (A and B of a cell are one float4).
__device__ __forceinline__ int cell_index(const TbParams &p, int m1, int m2) { return m1 * p.L2 + m2; }

__device__ __forceinline__ void prefetch_tile(const TbParams &p, const Stage &st, int tile, int r0, int lane,
                                              bool first)
{
    const int t1 = tile / p.tiles2, t2 = tile - t1 * p.tiles2;
    const int o1 = t1 * kTbT1 - kTbH, o2 = t2 * kTbT2 - kTbH;
    const int m2 = wrap(o2 + lane, p.L2);
    const float4 *psi = reinterpret_cast<const float4 *>(p.psi);
    const float4 *bx = reinterpret_cast<const float4 *>(p.bx);
    const float4 *bz = reinterpret_cast<const float4 *>(p.bz);
    const float2 *on = reinterpret_cast<const float2 *>(p.onsite);
#pragma unroll
    for (int r = 0; r < kTbR; ++r) {
        const int c = cell_index(p, wrap(o1 + r0 + r, p.L1), m2);
        const int slot = r * kTbThreads;
        cp_async16(st.ps + slot, psi + c);
        if (p.onsite) cp_async8(st.on + slot, on + c);
        else st.on[slot] = make_float2(0.0f, 0.0f);
        if (!first) {
            cp_async16(st.bx + slot, bx + c);
            cp_async16(st.bz + slot, bz + c);
        }
    }
    cp_async_commit();
}

// One sweep over this thread's kTbR cells. x holds b_{k+1} (A and B of each
// row), z holds b_{k+2} on entry and the new b_k on exit. up is the B value of
// the row above this warp's first row, dn the A value of the row below its
// last row. FORM 0: a middle sweep with c_k real (out = a psi - z + A x);
// FORM 1: c_k imaginary (i a psi); FORM 2: the general form
//   out = alpha psi - hz z + beta (d x + t sum of the neighbours).
template <int FORM>
__device__ __forceinline__ void tb_rows(const float2 (&pa)[kTbR], const float2 (&pb)[kTbR],
                                        const float2 (&oa)[kTbR], const float2 (&x)[2 * kTbR],
                                        float2 (&z)[2 * kTbR], float2 up, float2 dn, float t, const float *c)
{
#pragma unroll
    for (int r = 0; r < kTbR; ++r) {
        const float2 xa = x[2 * r], xb = x[2 * r + 1];
        // A(m): B(m), B(m - a1) (row above), B(m - a2) (lane to the left)
        const float2 b1 = r > 0 ? x[2 * r - 1] : up;
        float2 b2;
        b2.x = __shfl_up_sync(0xffffffffu, xb.x, 1);
        b2.y = __shfl_up_sync(0xffffffffu, xb.y, 1);
        // B(m): A(m), A(m + a1) (row below), A(m + a2) (lane to the right)
        const float2 a1 = r < kTbR - 1 ? x[2 * r + 2] : dn;
        float2 a2;
        a2.x = __shfl_down_sync(0xffffffffu, xa.x, 1);
        a2.y = __shfl_down_sync(0xffffffffu, xa.y, 1);
        const float sar = xb.x + b1.x + b2.x, sai = xb.y + b1.y + b2.y;   // neighbours of A
        const float sbr = xa.x + a1.x + a2.x, sbi = xa.y + a1.y + a2.y;   // neighbours of B
        const float2 za = z[2 * r], zb = z[2 * r + 1];
        float2 na, nb;
        if (FORM == 0) {
            na.x = fmaf(t, sar, fmaf(oa[r].x, xa.x, fmaf(c[0], pa[r].x, -za.x)));
            na.y = fmaf(t, sai, fmaf(oa[r].x, xa.y, fmaf(c[0], pa[r].y, -za.y)));
            nb.x = fmaf(t, sbr, fmaf(oa[r].y, xb.x, fmaf(c[0], pb[r].x, -zb.x)));
            nb.y = fmaf(t, sbi, fmaf(oa[r].y, xb.y, fmaf(c[0], pb[r].y, -zb.y)));
        } else if (FORM == 1) {
            na.x = fmaf(t, sar, fmaf(oa[r].x, xa.x, fmaf(-c[1], pa[r].y, -za.x)));
            na.y = fmaf(t, sai, fmaf(oa[r].x, xa.y, fmaf(c[1], pa[r].x, -za.y)));
            nb.x = fmaf(t, sbr, fmaf(oa[r].y, xb.x, fmaf(-c[1], pb[r].y, -zb.x)));
            nb.y = fmaf(t, sbi, fmaf(oa[r].y, xb.y, fmaf(c[1], pb[r].x, -zb.y)));
        } else {
            float tr = fmaf(-c[4], za.x, fmaf(c[0], pa[r].x, -c[1] * pa[r].y));
            float ti = fmaf(-c[4], za.y, fmaf(c[0], pa[r].y, c[1] * pa[r].x));
            float hr = fmaf(t, sar, oa[r].x * xa.x), hi = fmaf(t, sai, oa[r].x * xa.y);
            na.x = fmaf(c[2], hr, fmaf(-c[3], hi, tr));
            na.y = fmaf(c[2], hi, fmaf(c[3], hr, ti));
            tr = fmaf(-c[4], zb.x, fmaf(c[0], pb[r].x, -c[1] * pb[r].y));
            ti = fmaf(-c[4], zb.y, fmaf(c[0], pb[r].y, c[1] * pb[r].x));
            hr = fmaf(t, sbr, oa[r].y * xb.x);
            hi = fmaf(t, sbi, oa[r].y * xb.y);
            nb.x = fmaf(c[2], hr, fmaf(-c[3], hi, tr));
            nb.y = fmaf(c[2], hi, fmaf(c[3], hr, ti));
        }
        z[2 * r] = na;
        z[2 * r + 1] = nb;
    }
}

__global__ void __launch_bounds__(kTbThreads, 1) tb_block_kernel(TbParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // FP32 coefficients of this launch's sweeps: alpha (re, im), beta (re, im), hz.
    // Formed once per block from the FP64 series: on GB300 an FP64 operation costs
    // as much issue time as a few dozen FP32 ones, so no thread repeats this per tile.
    __shared__ float cf[kTbS][5];
    __shared__ int cform[kTbS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Stage st;
    {
        float4 *base = reinterpret_cast<float4 *>(smem) + threadIdx.x;
        st.ps = base;
        st.bx = base + kTbR * kTbThreads;
        st.bz = base + 2 * kTbR * kTbThreads;
        st.on = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(smem) + 3 * kTbR * kTbThreads) + threadIdx.x;
    }
    // exch[buf][0][w][lane]: first-row A of warp w; exch[buf][1][w][lane]: last-row B
    float2 *exch = reinterpret_cast<float2 *>(smem + kTbStageBytes);
    const int r0 = warp * kTbR;                   // this warp's first region row
    const int K = p.K;
    const bool first = p.j0 == 0;
    const bool final = p.j0 + p.S == K - 1;
    const int ntiles = p.tiles1 * p.tiles2;
    const float t = p.t;

    if ((int)threadIdx.x < p.S) {
        // sweep j of FIRST, SECOND, MID..., FINAL in one form:
        //   out = alpha psi - hz z + beta (d x + t sum of the three neighbours)
        // with alpha, beta complex scalars (real or imaginary by parity) and hz in {0, 1}
        const int j = p.j0 + threadIdx.x;
        const bool is_first = j == 0;
        const bool is_final = j == K - 2;
        const bool is_second = !is_first && !is_final && j == 1;
        const int k = is_final ? 0 : K - 2 - j;
        const double2 ca = p.coef[k];
        double2 cb = make_double2(0.0, 0.0);
        if (is_second || (is_final && K == 3)) cb = p.coef[is_second ? K - 1 : 2];
        const float av = (float)((k & 1) ? (ca.y - cb.y) : (ca.x - cb.x));
        float br = 1.0f, bi = 0.0f;
        if (is_first) {
            const double2 cc = p.coef[K - 1];
            if ((K - 1) & 1) { br = 0.0f; bi = (float)cc.y; } else { br = (float)cc.x; }
        } else if (is_final) {
            br = 0.5f;
        }
        cf[threadIdx.x][0] = (k & 1) ? 0.0f : av;
        cf[threadIdx.x][1] = (k & 1) ? av : 0.0f;
        cf[threadIdx.x][2] = br;
        cf[threadIdx.x][3] = bi;
        cf[threadIdx.x][4] = (!is_first && !is_second && !(is_final && K == 3)) ? 1.0f : 0.0f;
        cform[threadIdx.x] = (is_first || is_second || is_final) ? 2 : (k & 1);
    }
    // <psi0|psi> of this thread's interior cells, all tiles, on the FP32 pipe
    F2Sum sr, si;

    float2 pa[kTbR], pb[kTbR], oa[kTbR], xo[2 * kTbR], zo[2 * kTbR];
    // sweeps run so far by this block: the exchange buffer alternates with it
    // (across tiles too), so a buffer is rewritten only two barriers after its reads
    int nsweep = 0;
    if ((int)blockIdx.x < ntiles) prefetch_tile(p, st, blockIdx.x, r0, lane, first);
    __syncthreads();                               // the coefficient table
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t1 = tile / p.tiles2, t2 = tile - t1 * p.tiles2;
        const int o1 = t1 * kTbT1 - kTbH, o2 = t2 * kTbT2 - kTbH;
        cp_async_wait_all();                      // this thread's own staging slots
#pragma unroll
        for (int r = 0; r < kTbR; ++r) {
            const int slot = r * kTbThreads;
            const float4 ps = st.ps[slot];
            pa[r] = make_float2(ps.x, ps.y);
            pb[r] = make_float2(ps.z, ps.w);
            oa[r] = st.on[slot];
            if (!first) {
                const float4 bx = st.bx[slot], bz = st.bz[slot];
                xo[2 * r] = make_float2(bx.x, bx.y);
                xo[2 * r + 1] = make_float2(bx.z, bx.w);
                zo[2 * r] = make_float2(bz.x, bz.y);
                zo[2 * r + 1] = make_float2(bz.z, bz.w);
            } else {                              // the first sweep's operand is psi
                xo[2 * r] = pa[r];
                xo[2 * r + 1] = pb[r];
                zo[2 * r] = make_float2(0.0f, 0.0f);
                zo[2 * r + 1] = make_float2(0.0f, 0.0f);
            }
        }
        // the staging slots are free again: fetch the next tile during the sweeps
        if (tile + (int)gridDim.x < ntiles) prefetch_tile(p, st, tile + gridDim.x, r0, lane, first);
        // the register arrays trade roles each sweep: even sweeps read b_{k+1} from
        // xo and overwrite zo with b_k, odd sweeps the reverse
        for (int q = 0; q < p.S; ++q) {
            const float *c = cf[q];
            const int form = cform[q];
            float2 *ex = exch + (nsweep++ & 1) * 2 * kTbWarps * 32;
            const float2 *x = (q & 1) ? zo : xo;
            ex[warp * 32 + lane] = x[0];                              // first row, A
            ex[(kTbWarps + warp) * 32 + lane] = x[2 * kTbR - 1];      // last row, B
            __syncthreads();
            const float2 up = warp > 0 ? ex[(kTbWarps + warp - 1) * 32 + lane] : x[1];
            const float2 dn = warp < kTbWarps - 1 ? ex[(warp + 1) * 32 + lane] : x[2 * kTbR - 2];
            if ((q & 1) == 0) {
                if (form == 0) tb_rows<0>(pa, pb, oa, xo, zo, up, dn, t, c);
                else if (form == 1) tb_rows<1>(pa, pb, oa, xo, zo, up, dn, t, c);
                else tb_rows<2>(pa, pb, oa, xo, zo, up, dn, t, c);
            } else {
                if (form == 0) tb_rows<0>(pa, pb, oa, zo, xo, up, dn, t, c);
                else if (form == 1) tb_rows<1>(pa, pb, oa, zo, xo, up, dn, t, c);
                else tb_rows<2>(pa, pb, oa, zo, xo, up, dn, t, c);
            }
        }
        // newest b (or psi(t_{n+1})) in zo after an odd number of sweeps, else in xo
        const bool odd = (p.S & 1) != 0;
        const int m2 = o2 + lane;
        const bool col_in = lane >= kTbH && lane < kTbH + kTbT2 && m2 < p.L2;
#pragma unroll
        for (int r = 0; r < kTbR; ++r) {
            const int c1 = r0 + r;
            const int m1 = o1 + c1;
            if (!col_in || c1 < kTbH || c1 >= kTbH + kTbT1 || m1 >= p.L1) continue;
            const int c = cell_index(p, m1, m2);
            const float2 na = odd ? zo[2 * r] : xo[2 * r], nb = odd ? zo[2 * r + 1] : xo[2 * r + 1];
            const float4 yn = make_float4(na.x, na.y, nb.x, nb.y);
            if (final) {
                __stcs(reinterpret_cast<float4 *>(p.psi_out) + c, yn);
                const float4 q0 = __ldcs(reinterpret_cast<const float4 *>(p.psi0) + c);
                // conj(q0) y = (q0.x y.x + q0.y y.y) + i (q0.x y.y - q0.y y.x), products exact
                sr.add_prod(q0.x, yn.x); sr.add_prod(q0.y, yn.y);
                si.add_prod(q0.x, yn.y); si.add_prod(-q0.y, yn.x);
                sr.add_prod(q0.z, yn.z); sr.add_prod(q0.w, yn.w);
                si.add_prod(q0.z, yn.w); si.add_prod(-q0.w, yn.z);
            } else {
                const float2 pa2 = odd ? xo[2 * r] : zo[2 * r], pb2 = odd ? xo[2 * r + 1] : zo[2 * r + 1];
                __stcs(reinterpret_cast<float4 *>(p.ox) + c, yn);
                __stcs(reinterpret_cast<float4 *>(p.oz) + c, make_float4(pa2.x, pa2.y, pb2.x, pb2.y));
            }
        }
    }
    if (final) {
        const double dr = warp_sum(sr.value());
        const double di = warp_sum(si.value());
        if (lane == 0)
            p.partials[(int64_t)p.delta * gridDim.x * kTbWarps + blockIdx.x * kTbWarps + warp] =
                make_double2(dr, di);
    }
}

}  // namespace

size_t tb_smem_bytes() { return kTbSmem; }
int tb_tiles(int64_t l1, int64_t l2, int *tiles1, int *tiles2)
{
    *tiles1 = (int)((l1 + kTbT1 - 1) / kTbT1);
    *tiles2 = (int)((l2 + kTbT2 - 1) / kTbT2);
    return *tiles1 * *tiles2;
}

cudaError_t tb_prepare()
{
    return cudaFuncSetAttribute(tb_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTbSmem);
}

cudaError_t launch_tb_block(const TbParams &p, int grid, cudaStream_t s)
{
    tb_block_kernel<<<grid, kTbThreads, kTbSmem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace tbpm
