// Cluster-resident propagation for small systems: the whole time evolution of
// one state in a single launch of one thread-block cluster.
//
// For a few thousand orbitals every sweep is a few microseconds of work, so a
// launch per Chebyshev term (graph or not) costs as much as the term itself.
// Here one cluster of up to 16 CTAs owns the system: CTA r keeps rows
// [r R, (r+1) R) of psi, b0 and b1 in its shared memory (R a power of two),
// gathers the neighbours' b_{k+1} (or psi) from the owning CTA through
// distributed shared memory, and the hardware cluster barrier separates the
// sweeps. The row arithmetic, the sweep sequence and the per-slice dot partials
// are those of cheb_sweep.cu, so the correlation equals the graph path's.
// The matrix stays in global memory (it is L2-resident at these sizes).
#include <cooperative_groups.h>

#include "tbpm_internal.cuh"

namespace cg = cooperative_groups;

namespace tbpm {
namespace {

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

struct ClusterParams {
    int64_t n_pad;
    int64_t nslices;
    const int64_t *slice_off;
    const int32_t *cols;
    const void *vals;
    const void *diag;
    const void *psi0;          // global, [n_pad]
    const double2 *coef;
    int K;                     // >= 3
    int n_steps;
    int log_rows;              // rows per CTA = 1 << log_rows
    double2 *partials;         // [n_steps][nslices] <psi0|psi(t_{n+1})> per slice
    void *psi_out;             // global, [n_pad]: final state (may be null)
    int max_width;             // widest slice (entries per row), for the shared copy
};

// Where a CTA reads its matrix rows: its own slices, copied once into shared
// memory (SMAT), or global memory. off is relative to `cols`/`vals`.
struct MatView {
    const int32_t *cols;
    const void *vals;
    const void *diag;          // indexed by the CTA-local row (SMAT) or the global row
    const int32_t *loff;       // SMAT: local slice offsets (rows/32 + 1 entries)
};

template <typename R, bool REALV, bool SMAT>
__device__ __forceinline__ void gather_row(const ClusterParams &p, const MatView &m, cg::cluster_group &cl,
                                           typename V2<R>::T *xs, int64_t s, int ls, int lane, R &ar, R &ai)
{
    typedef typename V2<R>::T V;
    int64_t off;
    int w;
    if (SMAT) {
        off = m.loff[ls];
        w = (m.loff[ls + 1] - m.loff[ls]) >> 5;
    } else {
        off = __ldg(p.slice_off + s);
        w = (int)((__ldg(p.slice_off + s + 1) - off) >> 5);
    }
    const int mask = (1 << p.log_rows) - 1;
    if (REALV && w == 3) {
        // monolayer rows: the columns, then the three remote loads, then the FMAs,
        // so the distributed-shared-memory round trips overlap
        const int64_t e = off + lane;
        const int c0 = m.cols[e], c1 = m.cols[e + 32], c2 = m.cols[e + 64];
        const R *vr = reinterpret_cast<const R *>(m.vals);
        const R v0 = vr[e], v1 = vr[e + 32], v2 = vr[e + 64];
        const V x0 = cl.map_shared_rank(xs, (unsigned)(c0 >> p.log_rows))[c0 & mask];
        const V x1 = cl.map_shared_rank(xs, (unsigned)(c1 >> p.log_rows))[c1 & mask];
        const V x2 = cl.map_shared_rank(xs, (unsigned)(c2 >> p.log_rows))[c2 & mask];
        ar = fma(v0, x0.x, ar); ai = fma(v0, x0.y, ai);
        ar = fma(v1, x1.x, ar); ai = fma(v1, x1.y, ai);
        ar = fma(v2, x2.x, ar); ai = fma(v2, x2.y, ai);
        return;
    }
    for (int j = 0; j < w; ++j) {
        const int c = m.cols[off + 32 * j + lane];
        const V *rx = cl.map_shared_rank(xs, (unsigned)(c >> p.log_rows));
        const V xv = rx[c & mask];
        if (REALV) {
            const R v = reinterpret_cast<const R *>(m.vals)[off + 32 * j + lane];
            ar = fma(v, xv.x, ar);
            ai = fma(v, xv.y, ai);
        } else {
            const V v = reinterpret_cast<const V *>(m.vals)[off + 32 * j + lane];
            ar = fma(v.x, xv.x, fma(-v.y, xv.y, ar));
            ai = fma(v.x, xv.y, fma(v.y, xv.x, ai));
        }
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// kind: 0 FIRST (x = psi, y = b_{K-2}), 1 SECOND, 2 MID, 3 FINAL
template <typename R, bool REALV, bool SMAT>
__device__ void cluster_sweep(const ClusterParams &p, const MatView &mv, cg::cluster_group &cl, const R *tab,
                              int kind, int k, typename V2<R>::T *xs, typename V2<R>::T *psi, typename V2<R>::T *y,
                              const typename V2<R>::T *z, int step)
{
    typedef typename V2<R>::T V;
    const int K = p.K;
    // a on psi and beta on A x, as in cheb_sweep.cu (c_k real for even k), from
    // the table the kernel formed once (no FP64 arithmetic per sweep)
    const int ka = kind == 0 ? K - 2 : kind == 1 ? K - 3 : kind == 2 ? k : 0;
    const bool aimag = (ka & 1) != 0;
    const R a = tab[ka];
    const bool bimag = kind == 0 && ((K - 1) & 1) != 0;
    const R beta = kind == 0 ? tab[K - 1] : kind == 3 ? (R)0.5 : (R)1;
    const bool fold = (kind == 1 || kind == 2);          // beta = 1: acc starts at t
    const unsigned rank = cl.block_rank();
    const int rows = 1 << p.log_rows;
    const int64_t row0 = (int64_t)rank * rows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const R *diag = reinterpret_cast<const R *>(mv.diag);
    const V *psi0 = reinterpret_cast<const V *>(p.psi0);
    for (int ls = warp; ls < (rows >> 5); ls += nw) {
        const int64_t s = (row0 >> 5) + ls;
        if (s >= p.nslices) break;
        const int li = (ls << 5) + lane;
        const int64_t row = row0 + li;
        const V ps = psi[li];
        R tr, ti;
        if (aimag) { tr = -a * ps.y; ti = a * ps.x; } else { tr = a * ps.x; ti = a * ps.y; }
        if (z) { const V zz = z[li]; tr -= zz.x; ti -= zz.y; }
        const V xi = xs[li];
        const R d = diag ? diag[SMAT ? (int64_t)li : row] : (R)0;
        R ar, ai;
        if (fold) { ar = fma(d, xi.x, tr); ai = fma(d, xi.y, ti); }
        else { ar = d * xi.x; ai = d * xi.y; }
        gather_row<R, REALV, SMAT>(p, mv, cl, xs, s, ls, lane, ar, ai);
        V out;
        if (fold) { out.x = ar; out.y = ai; }
        else if (!bimag) { out.x = fma(beta, ar, tr); out.y = fma(beta, ai, ti); }
        else { out.x = fma(-beta, ai, tr); out.y = fma(beta, ar, ti); }
        y[li] = out;
        if (kind == 3) {
            const V q = psi0[row];
            const double qr = (double)q.x, qi = (double)q.y;
            const double orr = (double)out.x, oi = (double)out.y;
            const double dr = warp_sum(fma(qr, orr, qi * oi));
            const double di = warp_sum(fma(qr, oi, -qi * orr));
            if (lane == 0) p.partials[(int64_t)step * p.nslices + s] = make_double2(dr, di);
        }
    }
}

template <typename R, bool REALV, bool SMAT>
__global__ void __launch_bounds__(1024) cluster_dos_kernel(ClusterParams p)
{
    typedef typename V2<R>::T V;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rows = 1 << p.log_rows;
    V *psi = reinterpret_cast<V *>(smem);
    V *b0 = psi + rows;
    V *b1 = b0 + rows;
    const int64_t row0 = (int64_t)cl.block_rank() * rows;
    MatView mv;
    mv.cols = p.cols;
    mv.vals = p.vals;
    mv.diag = p.diag;
    mv.loff = nullptr;
    if (SMAT) {
        // this CTA's slices: [s0, s1); entries [e0, e1) of the global SELL arrays
        const int64_t s0 = row0 >> 5;
        const int64_t s1 = min(s0 + (rows >> 5), p.nslices);
        const int64_t e0 = p.slice_off[min(s0, p.nslices)];
        const int64_t e1 = p.slice_off[s1];              // s1 >= min(s0, nslices)
        const int ent = rows * p.max_width;
        const int vsz = REALV ? (int)sizeof(R) : (int)sizeof(V);
        unsigned char *q = reinterpret_cast<unsigned char *>(b1 + rows);
        void *svals = q;
        q += (size_t)ent * vsz;
        R *sdiag = reinterpret_cast<R *>(q);
        q += (size_t)rows * sizeof(R);
        int32_t *scols = reinterpret_cast<int32_t *>(q);
        q += (size_t)ent * sizeof(int32_t);
        int32_t *sloff = reinterpret_cast<int32_t *>(q);
        for (int64_t i = threadIdx.x; i < e1 - e0; i += blockDim.x) {
            scols[i] = p.cols[e0 + i];
            if (REALV) reinterpret_cast<R *>(svals)[i] = reinterpret_cast<const R *>(p.vals)[e0 + i];
            else reinterpret_cast<V *>(svals)[i] = reinterpret_cast<const V *>(p.vals)[e0 + i];
        }
        for (int i = threadIdx.x; i <= (rows >> 5); i += blockDim.x) {
            const int64_t sg = s0 + i;
            sloff[i] = (int32_t)((sg <= s1 ? p.slice_off[sg] : e1) - e0);
        }
        const R *gd = reinterpret_cast<const R *>(p.diag);
        for (int i = threadIdx.x; i < rows; i += blockDim.x)
            sdiag[i] = (gd && row0 + i < p.n_pad) ? gd[row0 + i] : (R)0;
        mv.cols = scols;
        mv.vals = svals;
        mv.diag = p.diag ? sdiag : nullptr;
        mv.loff = sloff;
    }
    const V *g0 = reinterpret_cast<const V *>(p.psi0);
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const int64_t r = row0 + i;
        V v;
        if (r < p.n_pad) v = g0[r]; else { v.x = (R)0; v.y = (R)0; }
        psi[i] = v;
        b0[i] = v;                      // defined values for rows never written
        b1[i] = v;
    }
    // per-term coefficient table: tab[k] = a of the sweep producing term k (the
    // part of c_k that is nonzero, minus c_{K-1} for the second sweep and c_2 for
    // the final one at K = 3), tab[K-1] = beta of the first sweep
    __shared__ R tab[kMaxTerms];
    {
        const int K = p.K;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            double v;
            if (k == K - 1) v = ((K - 1) & 1) ? p.coef[K - 1].y : p.coef[K - 1].x;
            else {
                v = (k & 1) ? p.coef[k].y : p.coef[k].x;
                if (k == K - 3 && K >= 4) v -= (k & 1) ? p.coef[K - 1].y : p.coef[K - 1].x;
                if (k == 0 && K == 3) v -= p.coef[2].x;
            }
            tab[k] = (R)v;
        }
    }
    cl.sync();
    const int K = p.K;
    V *B[2] = {b0, b1};
    for (int step = 0; step < p.n_steps; ++step) {
        cluster_sweep<R, REALV, SMAT>(p, mv, cl, tab, 0, K - 2, psi, psi, B[0], nullptr, step);
        cl.sync();
        if (K >= 4) {
            cluster_sweep<R, REALV, SMAT>(p, mv, cl, tab, 1, K - 3, B[0], psi, B[1], nullptr, step);
            cl.sync();
        }
        for (int k = K - 4; k >= 1; --k) {
            V *yk = B[(K - 2 - k) & 1];
            cluster_sweep<R, REALV, SMAT>(p, mv, cl, tab, 2, k, B[(K - 3 - k) & 1], psi, yk, yk, step);
            cl.sync();
        }
        cluster_sweep<R, REALV, SMAT>(p, mv, cl, tab, 3, 0, B[(K - 3) & 1], psi, psi, K >= 4 ? B[(K - 4) & 1] : nullptr,
                                      step);
        cl.sync();
    }
    if (p.psi_out) {
        V *o = reinterpret_cast<V *>(p.psi_out);
        for (int i = threadIdx.x; i < rows; i += blockDim.x)
            if (row0 + i < p.n_pad) o[row0 + i] = psi[i];
    }
}

template <typename R, bool REALV, bool SMAT>
cudaError_t launch_t(const ClusterParams &p, int ncta, int threads, size_t smem, cudaStream_t s)
{
    auto kern = cluster_dos_kernel<R, REALV, SMAT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncta, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace

// Geometry of the cluster path for n_pad rows, or false if it does not fit:
// up to 16 CTAs, rows per CTA a power of two, three state vectors per CTA in
// shared memory.
bool cluster_fits(int precision, int64_t n_pad, int *log_rows, int *ncta, size_t *smem)
{
    const size_t vb = precision == TBPM_FP64 ? 16 : 8;
    for (int lr = 5; lr <= 14; ++lr) {
        const int64_t rows = (int64_t)1 << lr;
        const int64_t c = (n_pad + rows - 1) / rows;
        const size_t sm = 3 * vb * (size_t)rows;
        if (c <= 16 && sm <= 200 * 1024) {
            *log_rows = lr;
            *ncta = (int)c;
            *smem = sm;
            return true;
        }
        if (sm > 200 * 1024) break;
    }
    return false;
}

cudaError_t launch_cluster_dos(int precision, bool real_values, const SweepParams &op, int max_width,
                               const void *psi0, const double2 *coef, int K, int n_steps,
                               double2 *partials, void *psi_out, cudaStream_t s)
{
    int lr, ncta;
    size_t smem;
    if (!cluster_fits(precision, op.nslices * 32, &lr, &ncta, &smem)) return cudaErrorInvalidValue;
    ClusterParams p;
    p.n_pad = op.nslices * 32;
    p.nslices = op.nslices;
    p.slice_off = op.slice_off;
    p.cols = op.cols;
    p.vals = op.vals;
    p.diag = op.diag;
    p.psi0 = psi0;
    p.coef = coef;
    p.K = K;
    p.n_steps = n_steps;
    p.log_rows = lr;
    p.partials = partials;
    p.psi_out = psi_out;
    p.max_width = max_width;
    const int rows = 1 << lr;
    const int threads = rows >= 1024 ? 1024 : (rows < 64 ? 64 : rows);
    // the CTA's matrix rows in shared memory too, when they fit beside the vectors
    const size_t rsz = precision == TBPM_FP64 ? 8 : 4;
    const size_t vsz = real_values ? rsz : 2 * rsz;
    const size_t msm = (size_t)rows * max_width * (vsz + 4) + (size_t)rows * rsz + ((size_t)(rows >> 5) + 1) * 4;
    const bool smat = smem + msm <= 200 * 1024;
    if (smat) smem += msm;
    if (precision == TBPM_FP64) {
        if (smat) return real_values ? launch_t<double, true, true>(p, ncta, threads, smem, s)
                                     : launch_t<double, false, true>(p, ncta, threads, smem, s);
        return real_values ? launch_t<double, true, false>(p, ncta, threads, smem, s)
                           : launch_t<double, false, false>(p, ncta, threads, smem, s);
    }
    if (smat) return real_values ? launch_t<float, true, true>(p, ncta, threads, smem, s)
                                 : launch_t<float, false, true>(p, ncta, threads, smem, s);
    return real_values ? launch_t<float, true, false>(p, ncta, threads, smem, s)
                       : launch_t<float, false, false>(p, ncta, threads, smem, s);
}

}  // namespace tbpm
