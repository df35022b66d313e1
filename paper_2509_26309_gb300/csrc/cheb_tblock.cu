// Temporal blocking of the Clenshaw sweeps on the matrix-free graphene
// lattices (monolayer and AB bilayer; FP32 vectors, one state).
//
// Each Chebyshev term needs only the nearest neighbours of the previous term
// (the hopping convention of Sec. 3.2.1: A(m) couples to B(m), B(m - a1),
// B(m - a2); the bilayer adds the dimer A1(m)-B2(m)), so several consecutive
// sweeps of one time step can run on a tile of the lattice held on chip, with
// a halo that the sweeps eat into: HBM then carries each term's vectors once
// per block of kTbS sweeps instead of once per sweep. This is the per-term HBM
// floor the sparse product of Sec. 2.2.1 sits on, broken for the structured
// lattices only.
//
// Layout on chip. A tile region is W1 rows (m1) by W2 = 32 C2 cells (m2).
// Lane l of every warp owns the C2 consecutive cells m2 = o2 + C2 l + c; warp w
// owns R consecutive rows. Each thread keeps all PER orbitals of its cells in
// registers (A, B per layer): psi, the on-site energies, b_{k+1} and b_{k+2}.
// The neighbours B(m - a2) and A(m + a2) are in the thread's own registers
// between its cells, and one lane away (warp shuffles) at the ends of its run
// of C2 cells; B(m - a1) and A(m + a1) are one row away (the thread's own
// registers, or, across a warp boundary, a row that each warp publishes in
// shared memory once per sweep), the dimer partner in the same cell. Lanes at
// the region's left and right edges and rows at its top and bottom read
// stand-in values: those cells are halo.
//
// A block of S sweeps loads psi(t_n), b_{k+1}, b_{k+2} and the on-site
// energies for its region (cp.async into a per-thread staging area while the
// previous tile computes), runs the S sweeps, and stores the interior of its
// last two b's (or, for the block holding the final sweep, psi(t_{n+1}) and
// the <psi0|psi> partials). A-sites lose valid cells on the low side of each
// axis in odd sweeps and on the high side in even ones, B-sites the reverse
// (the dimer bond stays within a cell), so after S sweeps every orbital is
// valid ceil(S/2) cells inside the region: kTbH = ceil(kTbS/2). Blocks read
// one pair of global b buffers and write another, and the final block writes
// psi(t_{n+1}) to a second state buffer: halo loads of other tiles never race
// with stores.
#include "tbpm_internal.cuh"
#include "sweep_ops.cuh"

namespace tbpm {
namespace {

constexpr int kTbH = (kTbS + 1) / 2;            // halo cells per side

// Tile configuration of each kernel. The monolayer time steps run 1024
// threads of 3 rows x 1 cell (a 32 x 96-cell region, interior 26 x 90, 64
// registers per thread); the bilayer, with twice the state per cell, and the
// KPM passes, which also keep per-pass dot sums in registers, run 512 threads
// of 3 rows x 1 cell (32 x 48 cells). Two cells per lane (in-thread
// neighbours along m2, half the shuffles, a 64-cell-wide region; the staging
// loads stay coalesced) measured slower on GB300 for the monolayer time steps:
// 4.2e11 orbital-terms/s at 512 threads x 3 rows, 4.1e11 at 768 x 2 rows and
// 1024 x 1 row, against 6.1e11 here (4096^2).
template <int PER, bool KPM = false>
struct TbCfg {
    static constexpr bool kMonoSteps = PER == 2 && !KPM;
    static constexpr int C2 = 1;                // cells per lane along m2
    static constexpr int R = 3;                 // rows per warp
    static constexpr int threads = kMonoSteps ? 1024 : 512;
    static constexpr int warps = threads / 32;
    static constexpr int W1 = warps * R;        // region rows (m1)
    static constexpr int T1 = W1 - 2 * kTbH;    // interior rows
    static constexpr int W2 = 32 * C2;          // region cells along m2
    static constexpr int T2 = W2 - 2 * kTbH;    // interior cells along m2
    static constexpr int V4 = PER / 2;          // float4 per cell
    static constexpr int NC = R * C2;           // cells per thread
    static constexpr int N = PER * NC;          // orbitals per thread
    // shared memory: staging (per thread and cell: psi, b_{k+1}, b_{k+2} as V4
    // float4 each, on-site as V4 float2), then the boundary rows each warp
    // publishes per sweep (first row's A values, last row's B values, V4 x C2
    // of each per lane), double-buffered
    static constexpr size_t stage = (size_t)threads * NC * V4 * (3 * sizeof(float4) + sizeof(float2));
    static constexpr size_t exch = (size_t)2 * 2 * V4 * C2 * warps * 32 * sizeof(float2);
    static constexpr size_t smem = stage + exch;
    static_assert(smem <= 227 * 1024, "shared memory per block");
};

// Orbital o of cell c of row r in a thread's register arrays.
template <int PER, int C2>
__device__ __forceinline__ constexpr int tb_idx(int r, int c, int o)
{
    return (r * C2 + c) * PER + o;
}

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

// Block sums of NV two-sum pairs (every thread calls it; shared memory sm
// holds NV * WARPS float2): each warp's lane 0 stores its pairs, then thread
// v < NV adds the warps' pairs in warp order and returns value v in FP64
// (one conversion per value and block: GB300's FP64 pipe is narrow, so no
// per-thread FP64 reduction).
template <int NV, int WARPS>
__device__ __forceinline__ double block_sum_f2(F2Sum *a, float2 *sm, int warp, int lane)
{
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        warp_sum_f2(a[v]);
        if (lane == 0) sm[v * WARPS + warp] = make_float2(a[v].hi, a[v].lo);
    }
    __syncthreads();
    double out = 0.0;
    if ((int)threadIdx.x < NV) {
        F2Sum t;
        for (int w = 0; w < WARPS; ++w) {
            const float2 e = sm[threadIdx.x * WARPS + w];
            t.add(e.x);
            t.lo = __fadd_rn(t.lo, e.y);
        }
        out = t.value();
    }
    return out;
}

// The tile coordinates (t1, t2) of a block's tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...: one division for the first, then a step of gridDim.x tiles
// split once into whole rows of tiles (dq) and a remainder (dr), so that no
// tile pays for two integer divisions.
struct TileWalk {
    int t1, t2, dq, dr, tiles2;
    __device__ __forceinline__ void init(int tile, int step, int nt2)
    {
        tiles2 = nt2;
        t1 = tile / nt2;
        t2 = tile - t1 * nt2;
        dq = step / nt2;
        dr = step - dq * nt2;
    }
    __device__ __forceinline__ void next(int &n1, int &n2) const
    {
        n1 = t1 + dq;
        n2 = t2 + dr;
        if (n2 >= tiles2) {
            n2 -= tiles2;
            ++n1;
        }
    }
};

// This thread's staging slots: slot (cell j, v) at [(j * V4 + v) * threads].
struct Stage {
    float4 *ps, *bx, *bz;
    float2 *on;
};

template <int PER, bool KPM>
__device__ __forceinline__ void prefetch_tile(const TbParams &p, const Stage &st, int t1, int t2, int r0, int lane,
                                              bool first)
{
    typedef TbCfg<PER, KPM> C;
    const int o1 = t1 * C::T1 - kTbH, o2 = t2 * C::T2 - kTbH;
    const float4 *psi = reinterpret_cast<const float4 *>(p.psi);
    const float4 *bx = reinterpret_cast<const float4 *>(p.bx);
    const float4 *bz = reinterpret_cast<const float4 *>(p.bz);
    const float2 *on = reinterpret_cast<const float2 *>(p.onsite);
    // lane l fetches region column j = 32 c + l (coalesced) into the staging
    // slot of the column's owner, lane j / C2, cell j % C2 of the same warp (the
    // warp synchronises before the owners read and before the slots are refilled)
#pragma unroll
    for (int c = 0; c < C::C2; ++c) {
        const int j = 32 * c + lane;
        const int own = j / C::C2 - lane, oc = j % C::C2;   // owner's lane offset, its cell
        const int m2 = wrap(o2 + j, p.L2);
#pragma unroll
        for (int r = 0; r < C::R; ++r) {
            const int cell = wrap(o1 + r0 + r, p.L1) * p.L2 + m2;
#pragma unroll
            for (int v = 0; v < C::V4; ++v) {
                const int g = cell * C::V4 + v;         // float4 index: orbitals 2v, 2v+1 of the cell
                const int slot = ((r * C::C2 + oc) * C::V4 + v) * C::threads + own;
                if (!KPM) cp_async16(st.ps + slot, psi + g);
                if (p.onsite) cp_async8(st.on + slot, on + g);
                else st.on[slot] = make_float2(0.0f, 0.0f);
                if (!first) {
                    cp_async16(st.bx + slot, bx + g);
                    cp_async16(st.bz + slot, bz + g);
                }
            }
        }
    }
    cp_async_commit();
}

// One sweep over this thread's R x C2 cells (PER orbitals each, at
// tb_idx(r, c, o): A_L = 2L, B_L = 2L + 1). x holds b_{k+1}, z holds b_{k+2}
// on entry and the new b_k on exit. up[c][L] is the B_L value of cell c of the
// row above this warp's first row, dn[c][L] the A_L value of cell c of the row
// below its last row. The three in-layer neighbours are summed unscaled and
// enter through one FMA with t (the dimer partner of the bilayer through one
// with t_perp).
// FORM 0: a middle sweep with c_k real (out = a psi - z + A x); FORM 1: c_k
// imaginary (i a psi); FORM 3: no psi term (out = A x - z, the KPM pass);
// FORM 2: the general form
//   out = alpha psi - hz z + beta (d x + t sum of the neighbours).
template <int PER, int R, int C2, int FORM>
__device__ __forceinline__ void tb_rows(const float2 (&ps)[PER * R * C2], const float (&on)[PER * R * C2],
                                        const float2 (&x)[PER * R * C2], float2 (&z)[PER * R * C2],
                                        const float2 (&up)[C2][PER / 2], const float2 (&dn)[C2][PER / 2],
                                        float t, float tp, const float *c)
{
    // the sweep's coefficients, read from the block's table once
    const float c0 = c[0], c1 = c[1];
    const float c2 = FORM == 2 ? c[2] : 0.0f, c3 = FORM == 2 ? c[3] : 0.0f, c4 = FORM == 2 ? c[4] : 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float2 sum[C2][PER];                          // unscaled sum of each orbital's in-layer neighbours
#pragma unroll
        for (int L = 0; L < PER / 2; ++L) {
            // B of the last cell of the lane to the left, A of the first cell of the lane to the right
            const float2 xbl = x[tb_idx<PER, C2>(r, C2 - 1, 2 * L + 1)];
            const float2 xaf = x[tb_idx<PER, C2>(r, 0, 2 * L)];
            const float2 bw = make_float2(__shfl_up_sync(0xffffffffu, xbl.x, 1),
                                          __shfl_up_sync(0xffffffffu, xbl.y, 1));
            const float2 ae = make_float2(__shfl_down_sync(0xffffffffu, xaf.x, 1),
                                          __shfl_down_sync(0xffffffffu, xaf.y, 1));
#pragma unroll
            for (int cc = 0; cc < C2; ++cc) {
                const float2 xa = x[tb_idx<PER, C2>(r, cc, 2 * L)], xb = x[tb_idx<PER, C2>(r, cc, 2 * L + 1)];
                // A(m): B(m), B(m - a1) (row above), B(m - a2) (cell to the left)
                const float2 b1 = r > 0 ? x[tb_idx<PER, C2>(r - 1, cc, 2 * L + 1)] : up[cc][L];
                const float2 b2 = cc > 0 ? x[tb_idx<PER, C2>(r, cc - 1, 2 * L + 1)] : bw;
                // B(m): A(m), A(m + a1) (row below), A(m + a2) (cell to the right)
                const float2 a1 = r < R - 1 ? x[tb_idx<PER, C2>(r + 1, cc, 2 * L)] : dn[cc][L];
                const float2 a2 = cc < C2 - 1 ? x[tb_idx<PER, C2>(r, cc + 1, 2 * L)] : ae;
                sum[cc][2 * L] = make_float2(xb.x + b1.x + b2.x, xb.y + b1.y + b2.y);
                sum[cc][2 * L + 1] = make_float2(xa.x + a1.x + a2.x, xa.y + a1.y + a2.y);
            }
        }
#pragma unroll
        for (int cc = 0; cc < C2; ++cc) {
#pragma unroll
            for (int o = 0; o < PER; ++o) {
                const int i = tb_idx<PER, C2>(r, cc, o);
                const float2 xi = x[i], pv = ps[i], zz = z[i];
                const bool dimer = PER == 4 && (o == 0 || o == 3);
                const float2 pt = dimer ? x[tb_idx<PER, C2>(r, cc, 3 - o)] : make_float2(0.0f, 0.0f);
                float2 out;
                if (FORM != 2) {
                    // the psi and z terms, then d x, the dimer partner, t times the neighbours
                    float rx, ry;
                    if (FORM == 0) { rx = fmaf(c0, pv.x, -zz.x); ry = fmaf(c0, pv.y, -zz.y); }
                    else if (FORM == 1) { rx = fmaf(-c1, pv.y, -zz.x); ry = fmaf(c1, pv.x, -zz.y); }
                    else { rx = -zz.x; ry = -zz.y; }
                    rx = fmaf(on[i], xi.x, rx);
                    ry = fmaf(on[i], xi.y, ry);
                    if (dimer) { rx = fmaf(tp, pt.x, rx); ry = fmaf(tp, pt.y, ry); }
                    out.x = fmaf(t, sum[cc][o].x, rx);
                    out.y = fmaf(t, sum[cc][o].y, ry);
                } else {
                    const float tr = fmaf(-c4, zz.x, fmaf(c0, pv.x, -c1 * pv.y));
                    const float ti = fmaf(-c4, zz.y, fmaf(c0, pv.y, c1 * pv.x));
                    float dr = on[i] * xi.x, di = on[i] * xi.y;
                    if (dimer) { dr = fmaf(tp, pt.x, dr); di = fmaf(tp, pt.y, di); }
                    const float hr = fmaf(t, sum[cc][o].x, dr), hi = fmaf(t, sum[cc][o].y, di);
                    out.x = fmaf(c2, hr, fmaf(-c3, hi, tr));
                    out.y = fmaf(c2, hi, fmaf(c3, hr, ti));
                }
                z[i] = out;
            }
        }
    }
}

// Publishes this warp's boundary rows of x (the first row's A values, the last
// row's B values) into exchange buffer ex and, after the block barrier, reads
// the neighbouring warps' into up and dn (the region's first and last warps
// read their own values: those rows are halo).
// ex layout: [side][v][c][warp][lane] float2.
template <int PER, int R, int C2, int WARPS>
__device__ __forceinline__ void tb_exchange(float2 *ex, const float2 (&x)[PER * R * C2], float2 (&up)[C2][PER / 2],
                                            float2 (&dn)[C2][PER / 2], int warp, int lane)
{
    constexpr int V4 = PER / 2;
#pragma unroll
    for (int v = 0; v < V4; ++v)
#pragma unroll
        for (int c = 0; c < C2; ++c) {
            ex[((v * C2 + c) * WARPS + warp) * 32 + lane] = x[tb_idx<PER, C2>(0, c, 2 * v)];
            ex[(((V4 + v) * C2 + c) * WARPS + warp) * 32 + lane] = x[tb_idx<PER, C2>(R - 1, c, 2 * v + 1)];
        }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V4; ++v)
#pragma unroll
        for (int c = 0; c < C2; ++c) {
            up[c][v] = warp > 0 ? ex[(((V4 + v) * C2 + c) * WARPS + warp - 1) * 32 + lane]
                                : x[tb_idx<PER, C2>(0, c, 2 * v + 1)];
            dn[c][v] = warp < WARPS - 1 ? ex[((v * C2 + c) * WARPS + warp + 1) * 32 + lane]
                                        : x[tb_idx<PER, C2>(R - 1, c, 2 * v)];
        }
}

// Sweep forms of a launch, 3 bits per sweep position (0, 1: middle sweeps with
// c_k real or imaginary; 2: the general form; 7: no sweep at this position).
// PAT < 0: the forms are read from the block's coefficient table at run time.
constexpr int kPatEnd = 7;
constexpr int tb_pat(int f0, int f1, int f2, int f3, int f4, int f5)
{
    return f0 | (f1 << 3) | (f2 << 6) | (f3 << 9) | (f4 << 12) | (f5 << 15);
}
// The launches of a K = 18 time step (x = pi) and of odd-K steps of the same
// partition: first (first, second and four middle sweeps), middle (six middle
// sweeps), final (four middle sweeps and the final one), by parity of k.
constexpr int kPatFirst0 = tb_pat(2, 2, 0, 1, 0, 1), kPatFirst1 = tb_pat(2, 2, 1, 0, 1, 0);
constexpr int kPatMid0 = tb_pat(0, 1, 0, 1, 0, 1), kPatMid1 = tb_pat(1, 0, 1, 0, 1, 0);
constexpr int kPatFinal0 = tb_pat(0, 1, 0, 1, 2, kPatEnd), kPatFinal1 = tb_pat(1, 0, 1, 0, 2, kPatEnd);

template <int PER, int PAT>
__global__ void __launch_bounds__(TbCfg<PER>::threads, 1) tb_block_kernel(TbParams p)
{
    typedef TbCfg<PER> C;
    constexpr int N = C::N;                       // orbitals per thread
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
        const int span = C::NC * C::V4 * C::threads;
        st.ps = base;
        st.bx = base + span;
        st.bz = base + 2 * span;
        st.on = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(smem) + 3 * span) + threadIdx.x;
    }
    float2 *exch = reinterpret_cast<float2 *>(smem + C::stage);
    const int r0 = warp * C::R;                   // this warp's first region row
    const int K = p.K;
    const bool first = p.j0 == 0;
    const bool final = p.j0 + p.S == K - 1;
    const int ntiles = p.tiles1 * p.tiles2;
    const float t = p.t, tp = p.t_perp;

    if ((int)threadIdx.x < p.S) {
        // sweep j of FIRST, SECOND, MID..., FINAL in one form:
        //   out = alpha psi - hz z + beta (d x + t sum of the neighbours)
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

    float2 ps[N], xo[N], zo[N];
    float on[N];
    // sweeps run so far by this block: the exchange buffer alternates with it
    // (across tiles too), so a buffer is rewritten only two barriers after its reads
    int nsweep = 0;
    constexpr int kExch = 2 * C::V4 * C::C2 * C::warps * 32;   // float2 per exchange buffer
    TileWalk tw;
    tw.init(blockIdx.x, gridDim.x, p.tiles2);
    if ((int)blockIdx.x < ntiles) prefetch_tile<PER, false>(p, st, tw.t1, tw.t2, r0, lane, first);
    __syncthreads();                               // the coefficient table
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t1 = tw.t1, t2 = tw.t2;
        int n1, n2;                               // the block's next tile
        tw.next(n1, n2);
        const int o1 = t1 * C::T1 - kTbH, o2 = t2 * C::T2 - kTbH;
        cp_async_wait_all();                      // the staging slots this thread filled
        if (C::C2 > 1) __syncwarp();              // and those its warp's other lanes filled
#pragma unroll
        for (int j = 0; j < C::NC; ++j) {
#pragma unroll
            for (int v = 0; v < C::V4; ++v) {
                const int slot = (j * C::V4 + v) * C::threads;
                const int i = PER * j + 2 * v;
                const float4 q = st.ps[slot];
                ps[i] = make_float2(q.x, q.y);
                ps[i + 1] = make_float2(q.z, q.w);
                const float2 o = st.on[slot];
                on[i] = o.x;
                on[i + 1] = o.y;
                if (!first) {
                    const float4 bx = st.bx[slot], bz = st.bz[slot];
                    xo[i] = make_float2(bx.x, bx.y);
                    xo[i + 1] = make_float2(bx.z, bx.w);
                    zo[i] = make_float2(bz.x, bz.y);
                    zo[i + 1] = make_float2(bz.z, bz.w);
                } else {                          // the first sweep's operand is psi
                    xo[i] = ps[i];
                    xo[i + 1] = ps[i + 1];
                    zo[i] = make_float2(0.0f, 0.0f);
                    zo[i + 1] = make_float2(0.0f, 0.0f);
                }
            }
        }
        // the staging slots are free again: fetch the next tile during the sweeps
        if (C::C2 > 1) __syncwarp();              // every lane has read its slots
        if (tile + (int)gridDim.x < ntiles) prefetch_tile<PER, false>(p, st, n1, n2, r0, lane, first);
        tw.t1 = n1;
        tw.t2 = n2;
        // the register arrays trade roles each sweep: even sweeps read b_{k+1} from
        // xo and overwrite zo with b_k, odd sweeps the reverse. The loop is unrolled
        // over the kTbS sweep positions (each copy knows its arrays' roles and its
        // exchange buffer; 6.1e11 against 5.6e11 orbital-terms/s for the runtime loop)
#pragma unroll
        for (int q = 0; q < kTbS; ++q) {
            const int fq = PAT >= 0 ? ((PAT >> (3 * q)) & 7) : -1;   // compile-time after unrolling
            if (PAT >= 0 ? fq == kPatEnd : q >= p.S) break;
            const float *c = cf[q];
            const int form = PAT >= 0 ? fq : cform[q];
            float2 *ex = exch + (nsweep++ & 1) * kExch;
            float2 up[C::C2][C::V4], dn[C::C2][C::V4];
            if ((q & 1) == 0) {
                tb_exchange<PER, C::R, C::C2, C::warps>(ex, xo, up, dn, warp, lane);
                if (form == 0) tb_rows<PER, C::R, C::C2, 0>(ps, on, xo, zo, up, dn, t, tp, c);
                else if (form == 1) tb_rows<PER, C::R, C::C2, 1>(ps, on, xo, zo, up, dn, t, tp, c);
                else tb_rows<PER, C::R, C::C2, 2>(ps, on, xo, zo, up, dn, t, tp, c);
            } else {
                tb_exchange<PER, C::R, C::C2, C::warps>(ex, zo, up, dn, warp, lane);
                if (form == 0) tb_rows<PER, C::R, C::C2, 0>(ps, on, zo, xo, up, dn, t, tp, c);
                else if (form == 1) tb_rows<PER, C::R, C::C2, 1>(ps, on, zo, xo, up, dn, t, tp, c);
                else tb_rows<PER, C::R, C::C2, 2>(ps, on, zo, xo, up, dn, t, tp, c);
            }
        }
        // newest b (or psi(t_{n+1})) in zo after an odd number of sweeps, else in xo
        const bool odd = (p.S & 1) != 0;
#pragma unroll
        for (int cc = 0; cc < C::C2; ++cc) {
            const int l2 = C::C2 * lane + cc;       // region column
            const int m2 = o2 + l2;
            if (l2 < kTbH || l2 >= kTbH + C::T2 || m2 >= p.L2) continue;
#pragma unroll
            for (int r = 0; r < C::R; ++r) {
                const int c1 = r0 + r;
                const int m1 = o1 + c1;
                if (c1 < kTbH || c1 >= kTbH + C::T1 || m1 >= p.L1) continue;
                const int cell = m1 * p.L2 + m2;
#pragma unroll
                for (int v = 0; v < C::V4; ++v) {
                    const int i = tb_idx<PER, C::C2>(r, cc, 2 * v);
                    const int g = cell * C::V4 + v;
                    const float2 na = odd ? zo[i] : xo[i], nb = odd ? zo[i + 1] : xo[i + 1];
                    const float4 yn = make_float4(na.x, na.y, nb.x, nb.y);
                    if (final) {
                        __stcs(reinterpret_cast<float4 *>(p.psi_out) + g, yn);
                        const float4 q0 = __ldcs(reinterpret_cast<const float4 *>(p.psi0) + g);
                        // conj(q0) y = (q0.x y.x + q0.y y.y) + i (q0.x y.y - q0.y y.x), two orbitals
                        sr.add_dot(q0.x, yn.x, q0.y, yn.y);
                        si.add_dot(q0.x, yn.y, -q0.y, yn.x);
                        sr.add_dot(q0.z, yn.z, q0.w, yn.w);
                        si.add_dot(q0.z, yn.w, -q0.w, yn.z);
                    } else {
                        const float2 pa = odd ? xo[i] : zo[i], pb = odd ? xo[i + 1] : zo[i + 1];
                        __stcs(reinterpret_cast<float4 *>(p.ox) + g, yn);
                        __stcs(reinterpret_cast<float4 *>(p.oz) + g, make_float4(pa.x, pa.y, pb.x, pb.y));
                    }
                }
            }
        }
    }
    if (final) {                                  // one partial per block, slot delta
        __syncthreads();                          // staging reused as reduction scratch
        F2Sum a[2] = {sr, si};
        const double v = block_sum_f2<2, C::warps>(a, reinterpret_cast<float2 *>(smem), warp, lane);
        if ((int)threadIdx.x < 2)
            reinterpret_cast<double *>(p.partials + (int64_t)p.delta * gridDim.x + blockIdx.x)[threadIdx.x] = v;
    }
}


// Temporally blocked KPM passes: from T_{m-1} (bz) and T_m (bx), p.S passes
// T_{m+q+1} = A T_{m+q} - T_{m+q-1}, each with <T_{m+q}|T_{m+q}> and
// <T_{m+q+1}|T_{m+q}> over the interior cells, written as the partials of
// slot delta + q, one per block (W = blocks):
// partials[(2 slot) W + b] = (<T|T>, 0), partials[(2 slot + 1) W + b] = <T'|T>.
// The interior of the last two T's goes to ox (newest) and oz. A thread's
// contributions within one tile (at most 3 PER terms) are summed in FP32, then
// added to per-pass FP32 two-sum pairs that run over all tiles; the pairs are
// summed over the block in FP32 and converted to FP64 once per block.
template <int PER>
__global__ void __launch_bounds__(TbCfg<PER, true>::threads, 1) tb_kpm_kernel(TbParams p)
{
    typedef TbCfg<PER, true> C;
    constexpr int N = C::N;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Stage st;
    {
        float4 *base = reinterpret_cast<float4 *>(smem) + threadIdx.x;
        const int span = C::NC * C::V4 * C::threads;
        st.ps = base;
        st.bx = base + span;
        st.bz = base + 2 * span;
        st.on = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(smem) + 3 * span) + threadIdx.x;
    }
    float2 *exch = reinterpret_cast<float2 *>(smem + C::stage);
    const int r0 = warp * C::R;
    const int ntiles = p.tiles1 * p.tiles2;
    const float t = p.t, tp = p.t_perp;
    // T_{m+1} = A T_m - T_{m-1}: the middle-sweep form with no psi term
    const float cm[5] = {0.0f, 0.0f, 1.0f, 0.0f, 1.0f};
    float2 zero[N];
#pragma unroll
    for (int i = 0; i < N; ++i) zero[i] = make_float2(0.0f, 0.0f);
    F2Sum acc[kTbS][3];

    float2 xo[N], zo[N];
    float on[N];
    int nsweep = 0;
    constexpr int kExch = 2 * C::V4 * C::C2 * C::warps * 32;
    TileWalk tw;
    tw.init(blockIdx.x, gridDim.x, p.tiles2);
    if ((int)blockIdx.x < ntiles) prefetch_tile<PER, true>(p, st, tw.t1, tw.t2, r0, lane, false);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t1 = tw.t1, t2 = tw.t2;
        int n1, n2;                               // the block's next tile
        tw.next(n1, n2);
        const int o1 = t1 * C::T1 - kTbH, o2 = t2 * C::T2 - kTbH;
        cp_async_wait_all();
#pragma unroll
        for (int j = 0; j < C::NC; ++j) {
#pragma unroll
            for (int v = 0; v < C::V4; ++v) {
                const int slot = (j * C::V4 + v) * C::threads;
                const int i = PER * j + 2 * v;
                const float2 o = st.on[slot];
                on[i] = o.x;
                on[i + 1] = o.y;
                const float4 bx = st.bx[slot], bz = st.bz[slot];
                xo[i] = make_float2(bx.x, bx.y);
                xo[i + 1] = make_float2(bx.z, bx.w);
                zo[i] = make_float2(bz.x, bz.y);
                zo[i + 1] = make_float2(bz.z, bz.w);
            }
        }
        if (tile + (int)gridDim.x < ntiles) prefetch_tile<PER, true>(p, st, n1, n2, r0, lane, false);
        tw.t1 = n1;
        tw.t2 = n2;
        bool cell_in[C::R][C::C2];
#pragma unroll
        for (int cc = 0; cc < C::C2; ++cc) {
            const int l2 = C::C2 * lane + cc;
            const bool col_in = l2 >= kTbH && l2 < kTbH + C::T2 && o2 + l2 < p.L2;
#pragma unroll
            for (int r = 0; r < C::R; ++r) {
                const int c1 = r0 + r;
                cell_in[r][cc] = col_in && c1 >= kTbH && c1 < kTbH + C::T1 && o1 + c1 < p.L1;
            }
        }
#pragma unroll
        for (int q = 0; q < kTbS; ++q) {
            if (q < p.S) {
                float2 *ex = exch + (nsweep++ & 1) * kExch;
                float2 *x = (q & 1) ? zo : xo;
                float2 *y = (q & 1) ? xo : zo;
                float2 up[C::C2][C::V4], dn[C::C2][C::V4];
                if ((q & 1) == 0) {
                    tb_exchange<PER, C::R, C::C2, C::warps>(ex, xo, up, dn, warp, lane);
                    tb_rows<PER, C::R, C::C2, 3>(zero, on, xo, zo, up, dn, t, tp, cm);
                } else {
                    tb_exchange<PER, C::R, C::C2, C::warps>(ex, zo, up, dn, warp, lane);
                    tb_rows<PER, C::R, C::C2, 3>(zero, on, zo, xo, up, dn, t, tp, cm);
                }
                // the dots of this pass: x = T_{m+q}, y = T_{m+q+1}
                float nn = 0.0f, cr = 0.0f, ci = 0.0f;
#pragma unroll
                for (int r = 0; r < C::R; ++r) {
#pragma unroll
                    for (int cc = 0; cc < C::C2; ++cc) {
                        if (!cell_in[r][cc]) continue;
#pragma unroll
                        for (int o = 0; o < PER; ++o) {
                            const int i = tb_idx<PER, C::C2>(r, cc, o);
                            const float2 a = x[i], b = y[i];
                            nn = fmaf(a.x, a.x, fmaf(a.y, a.y, nn));
                            cr = fmaf(b.x, a.x, fmaf(b.y, a.y, cr));
                            ci = fmaf(b.x, a.y, fmaf(-b.y, a.x, ci));
                        }
                    }
                }
                acc[q][0].add(nn);
                acc[q][1].add(cr);
                acc[q][2].add(ci);
            }
        }
        const bool odd = (p.S & 1) != 0;
#pragma unroll
        for (int cc = 0; cc < C::C2; ++cc) {
            const int m2 = o2 + C::C2 * lane + cc;
#pragma unroll
            for (int r = 0; r < C::R; ++r) {
                if (!cell_in[r][cc]) continue;
                const int cell = (o1 + r0 + r) * p.L2 + m2;
#pragma unroll
                for (int v = 0; v < C::V4; ++v) {
                    const int i = tb_idx<PER, C::C2>(r, cc, 2 * v);
                    const float2 na = odd ? zo[i] : xo[i], nb = odd ? zo[i + 1] : xo[i + 1];
                    const float2 pa = odd ? xo[i] : zo[i], pb = odd ? xo[i + 1] : zo[i + 1];
                    __stcs(reinterpret_cast<float4 *>(p.ox) + cell * C::V4 + v, make_float4(na.x, na.y, nb.x, nb.y));
                    __stcs(reinterpret_cast<float4 *>(p.oz) + cell * C::V4 + v, make_float4(pa.x, pa.y, pb.x, pb.y));
                }
            }
        }
    }
    // one partial per block and pass: value 3 q + c of thread 3 q + c
    __syncthreads();                              // staging reused as reduction scratch
    const double v = block_sum_f2<3 * kTbS, C::warps>(&acc[0][0], reinterpret_cast<float2 *>(smem), warp, lane);
    const int q = threadIdx.x / 3, c = threadIdx.x - 3 * (threadIdx.x / 3);
    if ((int)threadIdx.x < 3 * p.S) {
        const int64_t W = gridDim.x;
        double *e = reinterpret_cast<double *>(p.partials + (2 * (int64_t)(p.delta + q) + (c > 0)) * W + blockIdx.x);
        if (c == 0) {
            e[0] = v;
            e[1] = 0.0;
        } else {
            e[c - 1] = v;
        }
    }
}

}  // namespace

int tb_tiles(int per, int64_t l1, int64_t l2, int *tiles1, int *tiles2)
{
    const int t1 = per == 2 ? TbCfg<2>::T1 : TbCfg<4>::T1;
    const int t2 = per == 2 ? TbCfg<2>::T2 : TbCfg<4>::T2;
    *tiles1 = (int)((l1 + t1 - 1) / t1);
    *tiles2 = (int)((l2 + t2 - 1) / t2);
    return *tiles1 * *tiles2;
}

namespace {

// The specialised form patterns, then the run-time one.
constexpr int kTbPats[7] = {kPatFirst0, kPatFirst1, kPatMid0, kPatMid1, kPatFinal0, kPatFinal1, -1};

template <int PER, int I = 0>
cudaError_t tb_prepare_all()
{
    if constexpr (I < 7) {
        cudaError_t e = cudaFuncSetAttribute(tb_block_kernel<PER, kTbPats[I]>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TbCfg<PER>::smem);
        if (e != cudaSuccess) return e;
        return tb_prepare_all<PER, I + 1>();
    }
    return cudaSuccess;
}

template <int PER, int I = 0>
cudaError_t tb_launch_pat(int pat, const TbParams &p, int grid, cudaStream_t s)
{
    if constexpr (I < 7) {
        if (kTbPats[I] == pat || kTbPats[I] < 0) {
            tb_block_kernel<PER, kTbPats[I]><<<grid, TbCfg<PER>::threads, TbCfg<PER>::smem, s>>>(p);
            return cudaGetLastError();
        }
        return tb_launch_pat<PER, I + 1>(pat, p, grid, s);
    }
    return cudaErrorInvalidValue;
}

// The form pattern of the launch of sweeps [j0, j0 + S) of a K-term step, as the
// kernel's coefficient table forms it.
int tb_launch_pattern(int K, int j0, int S)
{
    int pat = 0;
    for (int q = 0; q < kTbS; ++q) {
        int f = kPatEnd;
        if (q < S) {
            const int j = j0 + q;
            const bool is_first = j == 0, is_final = j == K - 2;
            const bool is_second = !is_first && !is_final && j == 1;
            const int k = is_final ? 0 : K - 2 - j;
            f = (is_first || is_second || is_final) ? 2 : (k & 1);
        }
        pat |= f << (3 * q);
    }
    return pat;
}

}  // namespace

cudaError_t tb_prepare(int per)
{
    return per == 2 ? tb_prepare_all<2>() : tb_prepare_all<4>();
}

int tb_kpm_tiles(int per, int64_t l1, int64_t l2, int *tiles1, int *tiles2)
{
    const int t1 = per == 2 ? TbCfg<2, true>::T1 : TbCfg<4, true>::T1;
    const int t2 = per == 2 ? TbCfg<2, true>::T2 : TbCfg<4, true>::T2;
    *tiles1 = (int)((l1 + t1 - 1) / t1);
    *tiles2 = (int)((l2 + t2 - 1) / t2);
    return *tiles1 * *tiles2;
}

cudaError_t tb_kpm_prepare(int per)
{
    if (per == 2)
        return cudaFuncSetAttribute(tb_kpm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TbCfg<2, true>::smem);
    return cudaFuncSetAttribute(tb_kpm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TbCfg<4, true>::smem);
}

cudaError_t launch_tb_kpm(int per, const TbParams &p, int grid, cudaStream_t s)
{
    if (per == 2) tb_kpm_kernel<2><<<grid, TbCfg<2, true>::threads, TbCfg<2, true>::smem, s>>>(p);
    else tb_kpm_kernel<4><<<grid, TbCfg<4, true>::threads, TbCfg<4, true>::smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tb_block(int per, const TbParams &p, int grid, cudaStream_t s)
{
    // a launch whose sweep forms match a specialised pattern runs the kernel
    // compiled for it (no form dispatch), any other the run-time form table
    const int pat = tb_launch_pattern(p.K, p.j0, p.S);
    return per == 2 ? tb_launch_pat<2>(pat, p, grid, s) : tb_launch_pat<4>(pat, p, grid, s);
}

}  // namespace tbpm
