// Temporal blocking of the Clenshaw sweeps on the matrix-free monolayer
// graphene lattice (FP32 vectors, one state).
//
// Each Chebyshev term needs only the nearest neighbours of the previous term
// (the hopping convention of Sec. 3.2.1: A(m) couples to B(m), B(m - a1),
// B(m - a2)), so several consecutive sweeps of one time step can run on a
// tile of the lattice held in shared memory, with a halo that the sweeps eat
// into: HBM then carries each term's vectors once per block of kTbS sweeps
// instead of once per sweep. This is the per-term HBM floor the sparse
// product of Sec. 2.2.1 sits on, broken for the structured lattice only.
//
// A block of S sweeps loads psi(t_n), b_{k+1}, b_{k+2} and the on-site
// energies for a region of kTbW1 x kTbW2 cells (interior plus kTbH cells of
// halo on every side, periodic wrap), runs the S sweeps on chip (each thread
// holds its cells in registers; shared memory carries b_{k+1} to the
// neighbours), and
// stores the interior of its last two b's (or, for the block holding the
// final sweep, psi(t_{n+1}) and the <psi0|psi> partials). A-sites lose valid
// cells on the low side of each axis in odd sweeps and on the high side in
// even ones, B-sites the reverse, so after S sweeps both sublattices are
// valid ceil(S/2) cells inside the region: kTbH = ceil(kTbS/2).
// Blocks read one pair of global b buffers and write another, and the final
// block writes psi(t_{n+1}) to a second state buffer: halo loads of other
// tiles never race with stores.
#include "tbpm_internal.cuh"
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

constexpr int kTbH = (kTbS + 1) / 2;            // halo cells per side
constexpr int kTbW2 = 64;                       // region cells along m2 (4 groups of 16)
constexpr int kTbW1 = 40;                       // region cells along m1
constexpr int kTbT1 = kTbW1 - 2 * kTbH;         // interior cells along m1
constexpr int kTbT2 = kTbW2 - 2 * kTbH;         // interior cells along m2
constexpr int kTbPlane = kTbW1 * kTbW2;         // cells of one sublattice plane
constexpr int kTbWarps = kTbThreads / 32;
constexpr int kTbItems = kTbW1 * (kTbW2 / 16) / kTbWarps;   // 32-orbital work items per warp
static_assert(kTbW1 * (kTbW2 / 16) % kTbWarps == 0, "whole work items per warp");

// Shared memory: the current and the next b (float2 planes [s][c1][c2]),
// then a per-thread staging area into which the next tile's psi, b_{k+1},
// b_{k+2} and on-site energies arrive by cp.async while the current tile's
// sweeps run. Each thread keeps its own cells' values in registers during the
// sweeps; shared memory only publishes b_{k+1} to the neighbours.
constexpr size_t kTbXBytes = (size_t)2 * 2 * kTbPlane * sizeof(float2);
constexpr size_t kTbStageBytes = (size_t)kTbThreads * kTbItems * (3 * sizeof(float2) + sizeof(float));
constexpr size_t kTbSmem = kTbXBytes + kTbStageBytes;
static_assert(kTbSmem <= 227 * 1024, "shared memory per block");

// m mod L for m in [-L, 2L) by one compare (the usual case: tiles no larger
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

__device__ __forceinline__ void cp_async(void *dst, const void *src, int bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Staging slots of item r for this thread: psi, b_{k+1}, b_{k+2} (float2) and on-site (float).
struct Stage {
    float2 *ps, *bx, *bz;
    float *on;
};

__device__ __forceinline__ void prefetch_tile(const TbParams &p, const Stage &st, int tile, int warp, int sl, int cl,
                                              bool first)
{
    const int t1 = tile / p.tiles2, t2 = tile - t1 * p.tiles2;
    const int o1 = t1 * kTbT1 - kTbH, o2 = t2 * kTbT2 - kTbH;
#pragma unroll
    for (int r = 0; r < kTbItems; ++r) {
        const int it = warp + kTbWarps * r;
        const int c1 = it >> 2, c2 = ((it & 3) << 4) + cl;
        const int row = 2 * (wrap(o1 + c1, p.L1) * p.L2 + wrap(o2 + c2, p.L2)) + sl;
        const int slot = r * kTbThreads;
        cp_async(st.ps + slot, p.psi + row, 8);
        if (p.onsite) cp_async(st.on + slot, p.onsite + row, 4);
        else st.on[slot] = 0.0f;
        if (!first) {
            cp_async(st.bx + slot, p.bx + row, 8);
            cp_async(st.bz + slot, p.bz + row, 8);
        }
    }
    cp_async_commit();
}

// One sweep over this thread's kTbItems cells. x holds each cell's b_{k+1}
// (own value; the neighbours' come from shared memory xb), z its b_{k+2} on
// entry and the new b_k on exit (written to yb as well). FORM 0: a middle
// sweep with c_k real (out = a psi - z + A x); FORM 1: c_k imaginary
// (i a psi); FORM 2: the general form
//   out = alpha psi - hz z + beta (d x + t sum of the neighbours).
template <int FORM>
__device__ __forceinline__ void tb_items(const float2 *xb, float2 *yb, int own0, int oth0, int d1, int d2,
                                         const float2 (&ps)[kTbItems], const float (&on)[kTbItems],
                                         const float2 (&x)[kTbItems], float2 (&z)[kTbItems], float t,
                                         const float *c)
{
#pragma unroll
    for (int r = 0; r < kTbItems; ++r) {
        const int oth = oth0 + 16 * kTbWarps * r;
        const float2 x0 = xb[oth], x1 = xb[oth + d1], x2 = xb[oth + d2];
        const float2 xi = x[r], pv = ps[r], zz = z[r];
        const float sr = x0.x + x1.x + x2.x, si = x0.y + x1.y + x2.y;
        float2 out;
        if (FORM == 0) {
            out.x = fmaf(t, sr, fmaf(on[r], xi.x, fmaf(c[0], pv.x, -zz.x)));
            out.y = fmaf(t, si, fmaf(on[r], xi.y, fmaf(c[0], pv.y, -zz.y)));
        } else if (FORM == 1) {
            out.x = fmaf(t, sr, fmaf(on[r], xi.x, fmaf(-c[1], pv.y, -zz.x)));
            out.y = fmaf(t, si, fmaf(on[r], xi.y, fmaf(c[1], pv.x, -zz.y)));
        } else {
            const float tr = fmaf(-c[4], zz.x, fmaf(c[0], pv.x, -c[1] * pv.y));
            const float ti = fmaf(-c[4], zz.y, fmaf(c[0], pv.y, c[1] * pv.x));
            const float hr = fmaf(t, sr, on[r] * xi.x);
            const float hi = fmaf(t, si, on[r] * xi.y);
            out.x = fmaf(c[2], hr, fmaf(-c[3], hi, tr));
            out.y = fmaf(c[2], hi, fmaf(c[3], hr, ti));
        }
        yb[own0 + 16 * kTbWarps * r] = out;
        z[r] = out;
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
    float2 *X[2] = {reinterpret_cast<float2 *>(smem), reinterpret_cast<float2 *>(smem) + 2 * kTbPlane};
    Stage st;
    {
        float2 *base = reinterpret_cast<float2 *>(smem + kTbXBytes) + threadIdx.x;
        st.ps = base;
        st.bx = base + kTbItems * kTbThreads;
        st.bz = base + 2 * kTbItems * kTbThreads;
        st.on = reinterpret_cast<float *>(reinterpret_cast<float2 *>(smem + kTbXBytes) + 3 * kTbItems * kTbThreads) +
                threadIdx.x;
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sl = lane >> 4;                     // sublattice of this lane (0 = A, 1 = B)
    const int cl = lane & 15;                     // cell offset within a group of 16
    // item r of this warp: it = warp + kTbWarps r, cells c1 = it / 4, c2 = 16 (it % 4) + cl;
    // its shared-memory index is sl * plane + 16 it + cl. The neighbours sit on the
    // other plane at the same cell, one row back (A) or on (B), and one cell back
    // (A) or on (B); at the region's edges these offsets land on other in-bounds
    // cells of the same buffer, whose values only reach halo cells.
    const int own0 = sl * kTbPlane + 16 * warp + cl;
    const int oth0 = (1 - sl) * kTbPlane + 16 * warp + cl;
    const int d1 = sl == 0 ? -kTbW2 : kTbW2;
    const int d2 = sl == 0 ? -1 : 1;
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

    float2 ps[kTbItems], xo[kTbItems], zo[kTbItems];
    float on[kTbItems];
    if (blockIdx.x < ntiles) prefetch_tile(p, st, blockIdx.x, warp, sl, cl, first);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t1 = tile / p.tiles2, t2 = tile - t1 * p.tiles2;
        const int o1 = t1 * kTbT1 - kTbH, o2 = t2 * kTbT2 - kTbH;
        cp_async_wait_all();                      // this thread's own staging slots
        if (tile == (int)blockIdx.x) __syncthreads();   // the coefficient table
#pragma unroll
        for (int r = 0; r < kTbItems; ++r) {
            const int slot = r * kTbThreads;
            ps[r] = st.ps[slot];
            on[r] = st.on[slot];
            if (!first) {
                xo[r] = st.bx[slot];
                zo[r] = st.bz[slot];
            } else {
                xo[r] = ps[r];                    // the first sweep's operand is psi
                zo[r] = make_float2(0.0f, 0.0f);
            }
            X[0][own0 + 16 * kTbWarps * r] = xo[r];
        }
        // the staging slots are free again: fetch the next tile during the sweeps
        if (tile + (int)gridDim.x < ntiles) prefetch_tile(p, st, tile + gridDim.x, warp, sl, cl, first);
        __syncthreads();
        // the register arrays trade roles each sweep: even sweeps read b_{k+1} from
        // xo and overwrite zo with b_k, odd sweeps the reverse
        for (int q = 0; q < p.S; ++q) {
            const float *c = cf[q];
            const int form = cform[q];
            const float2 *xb = X[q & 1];
            float2 *yb = X[(q & 1) ^ 1];
            if ((q & 1) == 0) {
                if (form == 0) tb_items<0>(xb, yb, own0, oth0, d1, d2, ps, on, xo, zo, t, c);
                else if (form == 1) tb_items<1>(xb, yb, own0, oth0, d1, d2, ps, on, xo, zo, t, c);
                else tb_items<2>(xb, yb, own0, oth0, d1, d2, ps, on, xo, zo, t, c);
            } else {
                if (form == 0) tb_items<0>(xb, yb, own0, oth0, d1, d2, ps, on, zo, xo, t, c);
                else if (form == 1) tb_items<1>(xb, yb, own0, oth0, d1, d2, ps, on, zo, xo, t, c);
                else tb_items<2>(xb, yb, own0, oth0, d1, d2, ps, on, zo, xo, t, c);
            }
            __syncthreads();
        }
        // newest b (or psi(t_{n+1})) in zo after an odd number of sweeps, else in xo
        const bool odd = (p.S & 1) != 0;
        // interior: cells [kTbH, kTbH + T) of the region that lie on the lattice
#pragma unroll
        for (int r = 0; r < kTbItems; ++r) {
            const int it = warp + kTbWarps * r;
            const int c1 = it >> 2, c2 = ((it & 3) << 4) + cl;
            if (c1 < kTbH || c1 >= kTbH + kTbT1 || c2 < kTbH || c2 >= kTbH + kTbT2) continue;
            const int m1 = o1 + c1, m2 = o2 + c2;
            if (m1 >= p.L1 || m2 >= p.L2) continue;
            const int row = 2 * (m1 * p.L2 + m2) + sl;
            const float2 yn = odd ? zo[r] : xo[r], yp = odd ? xo[r] : zo[r];
            if (final) {
                __stcs(p.psi_out + row, yn);
                const float2 q0 = __ldcs(p.psi0 + row);
                // conj(q0) y = (q0.x y.x + q0.y y.y) + i (q0.x y.y - q0.y y.x), products exact
                sr.add_prod(q0.x, yn.x);
                sr.add_prod(q0.y, yn.y);
                si.add_prod(q0.x, yn.y);
                si.add_prod(-q0.y, yn.x);
            } else {
                __stcs(p.ox + row, yn);
                __stcs(p.oz + row, yp);
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
