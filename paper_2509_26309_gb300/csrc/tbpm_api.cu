// C ABI of libtbpm: argument and matrix validation, device layout, graph
// capture of the sweep sequences, and the calls declared in tbpm.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tbpm_internal.cuh"

using namespace tbpm;

namespace {

#define CU(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            if (ctx) ctx->last_error = std::string(#call) + ": " + cudaGetErrorString(e_); \
            return (e_ == cudaErrorMemoryAllocation) ? TBPM_ERR_OOM : TBPM_ERR_CUDA; \
        }                                                                        \
    } while (0)

// ------------------------------------------------------------- host matrix

// A validated Hermitian matrix: per row, off-diagonal entries sorted by column
// with duplicates summed, and the real diagonal apart.
struct HostMatrix {
    int64_t n = 0;
    std::vector<int64_t> rp;     // off-diagonal row pointers
    std::vector<int32_t> col;
    std::vector<double> re, im;
    std::vector<double> diag;
    double gershgorin = 0.0;
    bool real_values = true;
};

int build_host_matrix(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                      bool check_hermitian, HostMatrix &m)
{
    if (row_ptr[0] != 0) return TBPM_ERR_CSR;
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return TBPM_ERR_CSR;
    const int64_t nnz = row_ptr[n];
    for (int64_t p = 0; p < nnz; ++p)
        if (col[p] < 0 || (int64_t)col[p] >= n) return TBPM_ERR_CSR;
    for (int64_t p = 0; p < nnz; ++p)
        if (!std::isfinite(val[2 * p]) || !std::isfinite(val[2 * p + 1])) return TBPM_ERR_ARG;
    m.n = n;
    m.rp.assign(n + 1, 0);
    m.diag.assign(n, 0.0);
    m.col.reserve(nnz);
    m.re.reserve(nnz);
    m.im.reserve(nnz);
    std::vector<std::pair<int32_t, int64_t>> row;
    std::vector<double> dim(n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        row.clear();
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) row.emplace_back(col[p], p);
        std::sort(row.begin(), row.end());
        double gs = 0.0;
        size_t q = 0;
        while (q < row.size()) {
            const int32_t c = row[q].first;
            double sr = 0.0, si = 0.0;
            for (; q < row.size() && row[q].first == c; ++q) {
                sr += val[2 * row[q].second];
                si += val[2 * row[q].second + 1];
            }
            if (c == i) {
                m.diag[i] = sr;
                dim[i] = si;
            } else {
                m.col.push_back(c);
                m.re.push_back(sr);
                m.im.push_back(si);
                if (si != 0.0) m.real_values = false;
            }
            gs += std::hypot(sr, si);
        }
        m.rp[i + 1] = (int64_t)m.col.size();
        m.gershgorin = std::max(m.gershgorin, gs);
    }
    for (int64_t i = 0; i < n; ++i)
        if (dim[i] != 0.0) return TBPM_ERR_NOT_HERMITIAN;
    if (check_hermitian) {
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t p = m.rp[i]; p < m.rp[i + 1]; ++p) {
                const int32_t j = m.col[p];
                const int32_t *b = m.col.data() + m.rp[j], *e = m.col.data() + m.rp[j + 1];
                const int32_t *f = std::lower_bound(b, e, (int32_t)i);
                double tr = 0.0, ti = 0.0;
                if (f != e && *f == (int32_t)i) {
                    const int64_t q = f - m.col.data();
                    tr = m.re[q];
                    ti = -m.im[q];
                }
                const double scale = std::hypot(m.re[p], m.im[p]) + std::hypot(tr, ti);
                if (std::hypot(m.re[p] - tr, m.im[p] - ti) > 1e-13 * scale) return TBPM_ERR_NOT_HERMITIAN;
            }
        }
    }
    return TBPM_OK;
}

// The periodic lattice as a CSR matrix (tbpm_create_lattice with PATH_SELL).
void lattice_to_host_matrix(const tbpm_lattice &lat, HostMatrix &m)
{
    const int per = lat.kind == TBPM_LATTICE_GRAPHENE ? 2 : 4;
    const int64_t l1 = lat.l1, l2 = lat.l2, ncell = l1 * l2, n = ncell * per;
    m.n = n;
    m.rp.assign(n + 1, 0);
    m.diag.assign(n, 0.0);
    m.col.clear(); m.re.clear(); m.im.clear();
    m.real_values = true;
    std::vector<std::pair<int32_t, double>> row;
    double g = 0.0;
    for (int64_t c = 0; c < ncell; ++c) {
        const int64_t m1 = c / l2, m2 = c % l2;
        const int64_t cm1 = ((m1 + l1 - 1) % l1) * l2 + m2, cm2 = m1 * l2 + (m2 + l2 - 1) % l2;
        const int64_t cp1 = ((m1 + 1) % l1) * l2 + m2, cp2 = m1 * l2 + (m2 + 1) % l2;
        for (int o = 0; o < per; ++o) {
            const int64_t i = c * per + o;
            const int layer = o >> 1, s = o & 1;
            row.clear();
            if (s == 0) {
                row.emplace_back((int32_t)(c * per + 2 * layer + 1), lat.t);
                row.emplace_back((int32_t)(cm1 * per + 2 * layer + 1), lat.t);
                row.emplace_back((int32_t)(cm2 * per + 2 * layer + 1), lat.t);
            } else {
                row.emplace_back((int32_t)(c * per + 2 * layer), lat.t);
                row.emplace_back((int32_t)(cp1 * per + 2 * layer), lat.t);
                row.emplace_back((int32_t)(cp2 * per + 2 * layer), lat.t);
            }
            if (per == 4 && o == 0) row.emplace_back((int32_t)(c * 4 + 3), lat.t_perp);
            if (per == 4 && o == 3) row.emplace_back((int32_t)(c * 4), lat.t_perp);
            std::sort(row.begin(), row.end());
            double gs = 0.0;
            for (auto &e : row) {
                m.col.push_back(e.first);
                m.re.push_back(e.second);
                m.im.push_back(0.0);
                gs += std::fabs(e.second);
            }
            m.rp[i + 1] = (int64_t)m.col.size();
            m.diag[i] = lat.onsite ? lat.onsite[i] : 0.0;
            g = std::max(g, gs + std::fabs(m.diag[i]));
        }
    }
    m.gershgorin = g;
}

// ---------------------------------------------------------------- helpers

bool is_device_ptr(const void *p, int device, bool *bad_device)
{
    cudaPointerAttributes a;
    *bad_device = false;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (a.device != device) *bad_device = true;
        return true;
    }
    return false;
}

size_t vec_bytes(int precision) { return precision == TBPM_FP64 ? 16 : 8; }

int init_device(tbpm_ctx *ctx, const tbpm_opts &o)
{
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        ctx->last_error = "no CUDA device";
        return TBPM_ERR_NO_DEVICE;
    }
    int dev = o.device;
    if (dev < 0) CU(cudaGetDevice(&dev));
    if (dev >= count) return TBPM_ERR_ARG;
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, dev));
    if (!(prop.major == 10 && prop.minor == 3)) {
        ctx->last_error = "libtbpm is built for sm_103a only";
        return TBPM_ERR_NO_DEVICE;
    }
    CU(cudaSetDevice(dev));
    ctx->device = dev;
    ctx->num_sms = prop.multiProcessorCount;
    // NULL selects the legacy default stream, which orders the library's work
    // with every other blocking stream of the device (e.g. torch's default).
    ctx->stream = o.stream ? (cudaStream_t)o.stream : cudaStreamLegacy;
    ctx->own_stream = false;
    CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const int ncoef = std::max(1, ctx->ninst);
    CU(cudaMalloc(&ctx->d_coef, sizeof(double2) * kMaxTerms * ncoef));
    CU(cudaMalloc(&ctx->d_K, sizeof(int) * ncoef));
    CU(cudaMalloc(&ctx->d_counter, sizeof(int) * 4));
    CU(cudaMalloc(&ctx->d_misc, sizeof(double) * 8));
    return TBPM_OK;
}

template <typename R>
void to_sell(const HostMatrix &m, int64_t n_pad, const std::vector<double> &row_scale, bool real_values,
             std::vector<int64_t> &off, std::vector<int32_t> &cols, std::vector<R> &vals,
             std::vector<R> &diag, int &max_width)
{
    const int64_t nslices = n_pad / kSlice;
    off.assign(nslices + 1, 0);
    max_width = 0;
    for (int64_t sl = 0; sl < nslices; ++sl) {
        int w = 0;
        for (int l = 0; l < kSlice; ++l) {
            const int64_t r = sl * kSlice + l;
            if (r < m.n) w = std::max<int>(w, (int)(m.rp[r + 1] - m.rp[r]));
        }
        max_width = std::max(max_width, w);
        off[sl + 1] = off[sl] + (int64_t)w * kSlice;
    }
    const int64_t nent = off[nslices];
    const int cw = real_values ? 1 : 2;
    cols.assign(nent, 0);
    vals.assign(nent * cw, (R)0);
    diag.assign(n_pad, (R)0);
    for (int64_t sl = 0; sl < nslices; ++sl) {
        const int w = (int)((off[sl + 1] - off[sl]) / kSlice);
        for (int l = 0; l < kSlice; ++l) {
            const int64_t r = sl * kSlice + l;
            const int64_t len = r < m.n ? m.rp[r + 1] - m.rp[r] : 0;
            for (int j = 0; j < w; ++j) {
                const int64_t e = off[sl] + (int64_t)j * kSlice + l;
                if (j < len) {
                    const int64_t p = m.rp[r] + j;
                    cols[e] = m.col[p];
                    const double s = row_scale[r];
                    if (real_values) vals[e] = (R)(s * m.re[p]);
                    else { vals[2 * e] = (R)(s * m.re[p]); vals[2 * e + 1] = (R)(s * m.im[p]); }
                } else {
                    cols[e] = (int32_t)r;      // padding: own row, value 0
                }
            }
            if (r < m.n) diag[r] = (R)(row_scale[r] * m.diag[r]);
        }
    }
}

// The packed form of FP32 real SELL entries: for entry e of row r, the column
// offset (cols[e] - r) taken modulo n_pad into [-n_pad/2, n_pad/2), stored in
// 16 bits, and the index of vals[e] in a table of the distinct values (their
// bits), at most 256 (padding entries: offset 0, value 0). False, and nothing
// is kept, when an offset does not fit 16 bits or more than 256 values occur.
bool pack_sell(const std::vector<int32_t> &cols, const std::vector<float> &vals, const std::vector<int64_t> &off,
               int64_t n_pad, std::vector<int16_t> &cdelta, std::vector<uint8_t> &vidx, std::vector<float> &vtab)
{
    const int64_t nent = off.back();
    cdelta.assign(nent, 0);
    vidx.assign(nent, 0);
    vtab.clear();
    std::map<uint32_t, int> index;
    const int64_t nslices = (int64_t)off.size() - 1;
    for (int64_t sl = 0; sl < nslices; ++sl)
        for (int64_t e = off[sl]; e < off[sl + 1]; ++e) {
            const int64_t r = sl * kSlice + (e - off[sl]) % kSlice;
            int64_t d = ((int64_t)cols[e] - r) % n_pad;
            if (d >= (n_pad + 1) / 2) d -= n_pad;
            else if (d < -(n_pad / 2)) d += n_pad;
            if (d < INT16_MIN || d > INT16_MAX) return false;
            cdelta[e] = (int16_t)d;
            uint32_t bits;
            std::memcpy(&bits, &vals[e], sizeof(bits));
            auto it = index.find(bits);
            if (it == index.end()) {
                if (vtab.size() == 256) return false;
                it = index.emplace(bits, (int)vtab.size()).first;
                vtab.push_back(vals[e]);
            }
            vidx[e] = (uint8_t)it->second;
        }
    vtab.resize(256, 0.0f);
    return true;
}

// The per-row packed form of a packed matrix whose slices all have width 3 and
// whose entries take at most 32 values: row r's word holds the 16-bit offsets
// of its entries j = 0, 1, 2 in bits 16 j .. 16 j + 15 and their 5-bit value
// indices in bits 48 + 5 j .. 52 + 5 j. False when the matrix does not qualify.
bool pack_rows(const std::vector<int16_t> &cdelta, const std::vector<uint8_t> &vidx,
               const std::vector<int64_t> &off, std::vector<uint64_t> &rowpack)
{
    const int64_t nslices = (int64_t)off.size() - 1;
    for (int64_t sl = 0; sl < nslices; ++sl)
        if (off[sl + 1] - off[sl] != 3 * kSlice) return false;
    for (uint8_t k : vidx)
        if (k >= 32) return false;
    rowpack.assign(nslices * kSlice, 0);
    for (int64_t sl = 0; sl < nslices; ++sl)
        for (int lane = 0; lane < kSlice; ++lane) {
            uint64_t w = 0;
            for (int j = 0; j < 3; ++j) {
                const int64_t e = off[sl] + (int64_t)j * kSlice + lane;
                w |= (uint64_t)(uint16_t)cdelta[e] << (16 * j);
                w |= (uint64_t)vidx[e] << (48 + 5 * j);
            }
            rowpack[sl * kSlice + lane] = w;
        }
    return true;
}

template <typename T>
int upload(tbpm_ctx *ctx, void **dst, const std::vector<T> &src)
{
    const size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
    CU(cudaMalloc(dst, bytes));
    if (!src.empty()) CU(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return TBPM_OK;
}

// Stores A = 2 H / rescale (per row: 2 / rescale of the row's instance).
int setup_sell(tbpm_ctx *ctx, const HostMatrix &m, const std::vector<double> *row_scale = nullptr)
{
    const bool row_scale_given = row_scale != nullptr;          // a batch of instances
    std::vector<double> uniform;
    if (!row_scale) {
        uniform.assign(m.n, 2.0 / ctx->rescale);
        row_scale = &uniform;
    }
    const std::vector<double> &s = *row_scale;
    std::vector<int64_t> off;
    std::vector<int32_t> cols;
    int rc;
    ctx->sell.real_values = m.real_values;
    if (ctx->precision == TBPM_FP64) {
        std::vector<double> vals, diag;
        to_sell<double>(m, ctx->n_pad, s, m.real_values, off, cols, vals, diag, ctx->sell.max_width);
        if ((rc = upload(ctx, (void **)&ctx->sell.vals, vals))) return rc;
        if ((rc = upload(ctx, (void **)&ctx->sell.diag, diag))) return rc;
    } else {
        std::vector<float> vals, diag;
        to_sell<float>(m, ctx->n_pad, s, m.real_values, off, cols, vals, diag, ctx->sell.max_width);
        if ((rc = upload(ctx, (void **)&ctx->sell.vals, vals))) return rc;
        if ((rc = upload(ctx, (void **)&ctx->sell.diag, diag))) return rc;
        // a packed form, for a single instance with real values: one word per
        // row where the matrix allows it, else the per-entry form
        std::vector<int16_t> cdelta;
        std::vector<uint8_t> vidx;
        std::vector<float> vtab;
        std::vector<uint64_t> rowpack;
        if (!row_scale_given && m.real_values && !(ctx->flags & TBPM_F_PLAIN_SELL) &&
            pack_sell(cols, vals, off, ctx->n_pad, cdelta, vidx, vtab)) {
            if ((rc = upload(ctx, (void **)&ctx->sell.vtab, vtab))) return rc;
            if (pack_rows(cdelta, vidx, off, rowpack)) {
                if ((rc = upload(ctx, (void **)&ctx->sell.rowpack, rowpack))) return rc;
                ctx->sell.packed = 2;
            } else {
                if ((rc = upload(ctx, (void **)&ctx->sell.cdelta, cdelta))) return rc;
                if ((rc = upload(ctx, (void **)&ctx->sell.vidx, vidx))) return rc;
                ctx->sell.packed = 1;
            }
        }
    }
    ctx->sell.nslices = ctx->n_pad / kSlice;
    ctx->sell.nent = off.back();
    if ((rc = upload(ctx, (void **)&ctx->sell.slice_off, off))) return rc;
    if ((rc = upload(ctx, (void **)&ctx->sell.cols, cols))) return rc;
    ctx->nnz = (int64_t)m.col.size();
    ctx->op = OP_SELL;
    return TBPM_OK;
}

SweepVariant variant(const tbpm_ctx *ctx, int states)
{
    SweepVariant v;
    v.precision = ctx->precision;
    v.op = ctx->op;
    v.real_values = ctx->op == OP_SELL ? ctx->sell.real_values : true;
    v.packed = ctx->op == OP_SELL && ctx->precision == TBPM_FP32 && ctx->ninst == 0 ? ctx->sell.packed : 0;
    v.states = states;
    v.pdl = !(ctx->flags & TBPM_F_NO_PDL);
    v.block = ctx->sw_block;
    v.spw = ctx->sw_spw;
    return v;
}

// Warps of the single-state final sweep's grid: the number of per-warp dot
// partials a final sweep of one instance writes per slot.
int64_t sweep_warps(const tbpm_ctx *ctx) { return (int64_t)ctx->nblk_fin * ctx->sw_block / 32; }

// The grids of the first, second and final sweeps: one wave of each one's own
// occupancy at the context's block shape. Their register counts differ from a
// middle sweep's: the final sweep holds more (the FP64 <psi0|psi> and the
// norm), so the middle sweeps' grid of whole waves of their occupancy (FP64:
// three blocks of 512 threads per SM) would run it as one and a half waves,
// the last half wave on half the SM; the first and second sweeps of the FP32
// stored matrix hold fewer, and more resident blocks keep more of their
// dependent loads in flight. The middle sweeps keep the context's grid.
int kind_grid(const tbpm_ctx *ctx, const SweepVariant &v, SweepKind kind)
{
    // a renormalising context's final sweeps also sum |y|^2 (more registers)
    const int k = kind == SW_FINAL && (ctx->flags & TBPM_F_RENORM) ? SW_FINAL_NORM : (int)kind;
    const int occ = sweep_shape_occupancy(v, ctx->d_slice_inst != nullptr, k);
    return occ > 0 ? occ * ctx->num_sms : ctx->nblk;
}

void set_kind_grids(tbpm_ctx *ctx)
{
    const SweepVariant v = variant(ctx, 1);
    ctx->nblk_first = kind_grid(ctx, v, SW_FIRST);
    ctx->nblk_second = kind_grid(ctx, v, SW_SECOND);
    ctx->nblk_fin = kind_grid(ctx, v, SW_FINAL);
    ctx->nblk16_fin = sweep_grid_b16_final(v, ctx->num_sms, ctx->nblk16);
}

// The grid of one single-state sweep kind.
int sweep_kind_grid(const tbpm_ctx *ctx, SweepKind kind)
{
    return kind == SW_FIRST ? ctx->nblk_first : kind == SW_SECOND ? ctx->nblk_second
           : kind == SW_FINAL ? ctx->nblk_fin : ctx->nblk;
}

void fill_operator(const tbpm_ctx *ctx, SweepParams &p)
{
    memset(&p, 0, sizeof(p));
    p.n = ctx->n;
    p.nslices = ctx->n_pad / kSlice;
    if (ctx->op == OP_SELL) {
        p.slice_off = ctx->sell.slice_off;
        p.cols = ctx->sell.cols;
        p.vals = ctx->sell.vals;
        p.diag = ctx->sell.diag;
        p.cdelta = ctx->sell.cdelta;
        p.vidx = ctx->sell.vidx;
        p.vtab = ctx->sell.vtab;
        p.rowpack = ctx->sell.rowpack;
        p.npad = ctx->n_pad;
    } else {
        p.diag = ctx->sten.onsite;
        p.l1 = ctx->sten.l1;
        p.l2 = ctx->sten.l2;
        p.t = ctx->sten.t;
        p.t_perp = ctx->sten.t_perp;
    }
    p.nblk = ctx->nblk;
}

void destroy_graphs(tbpm_ctx *ctx)
{
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
}

// Work vectors for `states` interleaved states, partials, and per-call output.
int ensure_work(tbpm_ctx *ctx, int states, size_t out_elems, size_t stage_doubles)
{
    if (states > ctx->cap_states) {
        destroy_graphs(ctx);
        cudaFree(ctx->d_psi); cudaFree(ctx->d_b0); cudaFree(ctx->d_b1); cudaFree(ctx->d_psi0);
        cudaFree(ctx->d_partials); cudaFree(ctx->d_norm); cudaFree(ctx->d_scale);
        ctx->d_psi = ctx->d_b0 = ctx->d_b1 = ctx->d_psi0 = nullptr;
        ctx->d_partials = ctx->d_norm = nullptr;
        ctx->d_scale = nullptr;
        const size_t vb = vec_bytes(ctx->precision) * (size_t)ctx->n_pad * states;
        CU(cudaMalloc(&ctx->d_psi, vb));
        CU(cudaMalloc(&ctx->d_b0, vb));
        CU(cudaMalloc(&ctx->d_b1, vb));
        CU(cudaMalloc(&ctx->d_psi0, vb));
        CU(cudaMemsetAsync(ctx->d_b0, 0, vb, ctx->stream));
        CU(cudaMemsetAsync(ctx->d_b1, 0, vb, ctx->stream));
        // single-state partials: one per slice; 16-state partials: one per block and state
        const size_t nsl = (size_t)(ctx->n_pad / kSlice);
        // (the sweeps' per-warp partials, and those of the 512-thread dot and KPM kernels)
        const size_t W = std::max<size_t>((size_t)sweep_warps(ctx),
                                          (size_t)std::max(ctx->nblk, ctx->nblk_kpm) * (kBlockB1 / 32));
        const size_t per_slot = std::max<size_t>(std::max(std::max(2 * nsl, 2 * W), (size_t)ctx->num_sms * 32),
                                                 (size_t)ctx->nblk16 * kMaxBlockStates);
        ctx->partials_cap = (size_t)(kChunk + 1) * per_slot;
        CU(cudaMalloc(&ctx->d_partials, ctx->partials_cap * sizeof(double2)));
        if (ctx->flags & TBPM_F_RENORM) {
            CU(cudaMalloc(&ctx->d_norm, (size_t)kChunk * per_slot * sizeof(double2)));
            CU(cudaMalloc(&ctx->d_scale, sizeof(double) * std::max(kMaxBlockStates, ctx->ninst)));
        }
        ctx->cap_states = states;
    }
    if (out_elems > ctx->out_cap) {
        destroy_graphs(ctx);
        cudaFree(ctx->d_out);
        ctx->d_out = nullptr;
        CU(cudaMalloc(&ctx->d_out, out_elems * sizeof(double2)));
        ctx->out_cap = out_elems;
    }
    if (stage_doubles > ctx->stage_cap) {
        cudaFree(ctx->d_stage);
        ctx->d_stage = nullptr;
        CU(cudaMalloc(&ctx->d_stage, stage_doubles * sizeof(double)));
        ctx->stage_cap = stage_doubles;
    }
    return TBPM_OK;
}

// Chebyshev coefficients for x = dt * rescale on the device; K read back once per x.
int ensure_coeffs(tbpm_ctx *ctx, double x, int *K)
{
    if (ctx->K_cached > 0 && x == ctx->x_cached) {
        *K = ctx->K_cached;
        return TBPM_OK;
    }
    CU(launch_bessel(x, ctx->tol, ctx->d_coef, ctx->d_K, ctx->stream));
    int k = -1;
    CU(cudaMemcpyAsync(&k, ctx->d_K, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (k < 1) return TBPM_ERR_ARG;
    ctx->x_cached = x;
    ctx->K_cached = k;
    *K = k;
    return TBPM_OK;
}

// Enqueues `len` time steps (each K-1 sweeps) on stream s; step d of the
// chunk writes dot partials to slot d, then one reduction stores
// C(t_{base+1..base+len}) and the base counter advances.
int enqueue_dos_chunk(tbpm_ctx *ctx, int K, int len, int B, int64_t ld, cudaStream_t s,
                      int64_t *launches, bool qe = false)
{
    const SweepVariant v = variant(ctx, B);
    auto sweep = [&](SweepKind kind, bool a_imag, bool has_z, const SweepParams &p) {
        return B == 1 ? launch_sweep(v, kind, a_imag, has_z, p, sweep_kind_grid(ctx, kind), s)
                      : launch_sweep_b16(v, kind, a_imag, has_z, p, kind == SW_FINAL ? ctx->nblk16_fin : ctx->nblk16, s);
    };
    SweepParams p;
    fill_operator(ctx, p);
    p.coef = ctx->d_coef;
    p.psi = ctx->d_psi;
    p.psi0 = ctx->d_psi0;
    p.partials = ctx->d_partials;
    p.nblk = B == 1 ? ctx->nblk : ctx->nblk16_fin;            // the final sweep's partial stride
    const bool renorm = (ctx->flags & TBPM_F_RENORM) != 0;
    if (renorm) {
        p.scale = ctx->d_scale;
        p.norm_partials = ctx->d_norm;
    }
    const int nseg = std::max(1, ctx->ninst);
    p.slice_inst = ctx->d_slice_inst;                    // nullptr for a single instance
    // partials per slot: per slice for a batch, per warp of the grid otherwise
    const int64_t npart = ctx->ninst > 0 ? p.nslices : sweep_warps(ctx);
    void *Bv[2] = {ctx->d_b0, ctx->d_b1};
    for (int d = 0; d < len; ++d) {
        // FIRST: b_{K-2} = c_{K-2} psi + c_{K-1} A psi  -> B[0]
        p.x = ctx->d_psi; p.z = nullptr; p.y = Bv[0];
        p.ia = K - 2; p.ib = -1; p.ic = K - 1; p.bscale = 1.0;
        CU(sweep(SW_FIRST, ((K - 2) & 1) != 0, false, p));
        ++*launches;
        if (K >= 4) {
            // SECOND: b_{K-3} = (c_{K-3} - c_{K-1}) psi + A b_{K-2}  -> B[1]
            p.x = Bv[0]; p.z = nullptr; p.y = Bv[1];
            p.ia = K - 3; p.ib = K - 1; p.ic = -1; p.bscale = 1.0;
            CU(sweep(SW_SECOND, ((K - 3) & 1) != 0, false, p));
            ++*launches;
        }
        for (int k = K - 4; k >= 1; --k) {
            // b_k (in B[(K-2-k)&1], over b_{k+2}) = c_k psi + A b_{k+1} - b_{k+2}
            p.x = Bv[(K - 3 - k) & 1];
            p.y = Bv[(K - 2 - k) & 1];
            p.z = p.y;
            p.ia = k; p.ib = -1; p.ic = -1; p.bscale = 1.0;
            CU(sweep(SW_MID, (k & 1) != 0, true, p));
            ++*launches;
        }
        // FINAL: psi <- (c_0 - [K=3] c_2) psi + A b_1 / 2 - [K>=4] b_2, with <psi0|psi>
        p.x = Bv[(K - 3) & 1];
        p.z = K >= 4 ? Bv[(K - 4) & 1] : nullptr;
        p.y = ctx->d_psi;
        p.ia = 0; p.ib = K == 3 ? 2 : -1; p.ic = -1; p.bscale = 0.5;
        p.delta = d;
        CU(sweep(SW_FINAL, false, K >= 4, p));
        ++*launches;
        if (qe) {       // quasi-eigenstates: Q_e += dt/(2 pi) w_m exp(i E_e t_m) psi(t_m)
            CU(launch_qe_accumulate(ctx->precision, ctx->d_psi, ctx->d_qe, ctx->d_qe_e, ctx->qe_ne, ctx->n_pad,
                                    ctx->d_counter, d, ctx->qe_h, ctx->qe_N,
                                    std::fabs(ctx->qe_h) / (2.0 * 3.141592653589793238462643383279502884), s));
            ++*launches;
        }
        if (renorm) {   // 1/||psi(t_{n+1})|| for the next step's sweeps
            if (B == 1)
                CU(launch_renorm_seg(ctx->d_norm + (int64_t)d * npart, npart, ctx->d_seg_off, nseg,
                                     ctx->d_scale, s));
            else
                CU(launch_renorm(ctx->d_norm + (int64_t)d * p.nblk * B, p.nblk, B, ctx->d_scale, s));
            ++*launches;
        }
    }
    if (B == 1)
        CU(launch_reduce_seg(ctx->d_partials, len, 1, npart, ctx->d_seg_off, nseg, ctx->d_counter, 1,
                             ctx->d_out, ld, s));
    else CU(launch_reduce_b16(ctx->d_partials, len, ctx->nblk16_fin, ctx->d_counter, 1, ctx->d_out, ld, s));
    CU(launch_advance(ctx->d_counter, len, s));
    *launches += 2;
    return TBPM_OK;
}

// Enqueues `len` KPM sweeps starting at an odd pass index (T_q in B0 for odd q).
int enqueue_kpm_chunk(tbpm_ctx *ctx, int len, cudaStream_t s, int64_t *launches)
{
    const SweepVariant v = variant(ctx, 1);
    SweepParams op;
    fill_operator(ctx, op);
    KpmParams p;
    memset(&p, 0, sizeof(p));
    p.n = op.n; p.nslices = op.nslices; p.slice_off = op.slice_off; p.cols = op.cols;
    p.vals = op.vals; p.diag = op.diag; p.l1 = op.l1; p.l2 = op.l2; p.t = op.t; p.t_perp = op.t_perp;
    p.cdelta = op.cdelta; p.vidx = op.vidx; p.vtab = op.vtab; p.rowpack = op.rowpack; p.npad = op.npad;
    p.partials = ctx->d_partials;
    p.nblk = ctx->nblk_kpm;
    p.scale = 1.0;
    p.first = false;
    for (int d = 0; d < len; ++d) {
        // pass q (odd first): x = T_q, y = T_{q-1} -> T_{q+1}
        p.x = (d & 1) == 0 ? ctx->d_b0 : ctx->d_psi;
        p.y = (d & 1) == 0 ? ctx->d_psi : ctx->d_b0;
        p.delta = d;
        CU(launch_kpm(v, p, ctx->nblk_kpm, s));
        ++*launches;
    }
    CU(launch_reduce_seg(ctx->d_partials, len, 2, (int64_t)ctx->nblk_kpm * (kBlockB1 / 32), nullptr, 1,
                         ctx->d_counter, 1, ctx->d_out, 0, s));
    CU(launch_advance(ctx->d_counter, len, s));
    *launches += 2;
    return TBPM_OK;
}

// Enqueues `len` Haydock iterations starting at an even index n (u_n in
// d_psi for even n, in d_b0 for odd n); a_n and b_{n+1} go to d_out viewed as
// double[2 M] (a at [0, M), b at [M, 2 M)).
int enqueue_hay_chunk(tbpm_ctx *ctx, int len, int M, cudaStream_t s, int64_t *launches)
{
    const SweepVariant v = variant(ctx, 1);
    SweepParams p;
    fill_operator(ctx, p);
    p.partials = ctx->d_partials;
    double *aout = reinterpret_cast<double *>(ctx->d_out);
    double *bout = aout + M;
    double *part = reinterpret_cast<double *>(ctx->d_partials);        // nblk per-block sums
    unsigned *ticket = reinterpret_cast<unsigned *>(ctx->d_counter + 1);
    const int ga = ctx->hay_grid[0], gu = ctx->hay_grid[1];
    void *U[2] = {ctx->d_psi, ctx->d_b0};
    for (int d = 0; d < len; ++d) {
        p.x = U[d & 1];
        p.y = U[(d + 1) & 1];
        CU(launch_hay_apply(v, p, ctx->d_misc, 0.5 * ctx->rescale, part, ticket, aout, ctx->d_counter, ga, s));
        CU(launch_hay_update(v, U[d & 1], U[(d + 1) & 1], p.nslices, ctx->d_misc, 0.5 * ctx->rescale, part, ticket,
                             bout, ctx->d_counter, gu, s));
        *launches += 2;
    }
    return TBPM_OK;
}

// out = sum_{k<K} c_k T_k(H~) in by Clenshaw sweeps (K >= 3), one state.
// alt: the coefficients alternate between real (even k) and imaginary (odd
// k), as the time-step series c_k = (2 - delta_k0)(-i)^k J_k(x) does;
// otherwise all are real (the Fermi series), and the top coefficient c_{K-1}
// must be zero: the first sweep takes its beta from the imaginary part of
// c_{K-1}. in and out may be the same vector. The final sweep's <in|out>
// partials go to partial slot `slot`.
int enqueue_series(tbpm_ctx *ctx, const double2 *coef, int K, bool alt, void *in, void *out, int slot,
                   cudaStream_t s, int64_t *launches)
{
    const SweepVariant v = variant(ctx, 1);
    SweepParams p;
    fill_operator(ctx, p);
    p.coef = coef;
    p.psi = in;
    p.psi0 = in;
    p.partials = ctx->d_partials;
    p.nblk = ctx->nblk;
    void *Bv[2] = {ctx->d_b0, ctx->d_b1};
    auto im = [alt](int k) { return alt && (k & 1) != 0; };
    p.x = in; p.z = nullptr; p.y = Bv[0];
    p.ia = K - 2; p.ib = -1; p.ic = K - 1; p.bscale = 1.0;
    CU(launch_sweep(v, SW_FIRST, im(K - 2), false, p, ctx->nblk_first, s));
    if (K >= 4) {
        p.x = Bv[0]; p.z = nullptr; p.y = Bv[1];
        p.ia = K - 3; p.ib = K - 1; p.ic = -1;
        CU(launch_sweep(v, SW_SECOND, im(K - 3), false, p, ctx->nblk_second, s));
    }
    for (int k = K - 4; k >= 1; --k) {
        p.x = Bv[(K - 3 - k) & 1];
        p.y = Bv[(K - 2 - k) & 1];
        p.z = p.y;
        p.ia = k; p.ib = -1; p.ic = -1;
        CU(launch_sweep(v, SW_MID, im(k), true, p, ctx->nblk, s));
    }
    p.x = Bv[(K - 3) & 1];
    p.z = K >= 4 ? Bv[(K - 4) & 1] : nullptr;
    p.y = out;
    p.ia = 0; p.ib = K == 3 ? 2 : -1; p.ic = -1; p.bscale = 0.5;
    p.delta = slot;
    CU(launch_sweep(v, SW_FINAL, false, K >= 4, p, ctx->nblk_fin, s));
    *launches += K - 1;
    return TBPM_OK;
}

// The three AC vectors phi2, phi1_x, phi1_y (n_pad rows each) in d_ac.
void ac_vectors(tbpm_ctx *ctx, void *v[3])
{
    char *b = static_cast<char *>(ctx->d_ac);
    const size_t vb = sizeof(double2) * (size_t)ctx->n_pad;
    v[0] = b;
    v[1] = b + vb;
    v[2] = b + 2 * vb;
}

// `len` AC time steps: each advances phi2, phi1_x and phi1_y by one time
// step (K terms) and writes the four <phi2|J_a|phi1_b> partials of the new
// time to slot d; one reduction then stores C(t_{base+1..base+len}) into
// d_out as [step][4] and the base counter advances.
int enqueue_ac_chunk(tbpm_ctx *ctx, int K, int len, cudaStream_t s, int64_t *launches)
{
    void *v[3];
    ac_vectors(ctx, v);
    const int64_t W = (int64_t)ctx->nblk * (kBlockB1 / 32);
    int rc;
    for (int d = 0; d < len; ++d) {
        for (int q = 0; q < 3; ++q)
            if ((rc = enqueue_series(ctx, ctx->d_coef, K, true, v[q], v[q], kChunk, s, launches))) return rc;
        CU(launch_jdot(ctx->cur, v[0], v[1], v[2], ctx->d_acpart, d, ctx->nblk, s));
        ++*launches;
    }
    CU(launch_reduce_seg(ctx->d_acpart, len, 4, W, nullptr, 1, ctx->d_counter, 1, ctx->d_out, 0, s));
    CU(launch_advance(ctx->d_counter, len, s));
    *launches += 2;
    return TBPM_OK;
}

void free_ac(tbpm_ctx *ctx)
{
    cudaFree(ctx->d_ac); cudaFree(ctx->d_fnodes); cudaFree(ctx->d_fc); cudaFree(ctx->d_gc);
    cudaFree(ctx->d_kmax); cudaFree(ctx->d_acpart);
    ctx->d_ac = nullptr; ctx->d_fnodes = nullptr; ctx->d_fc = ctx->d_gc = nullptr;
    ctx->d_kmax = nullptr; ctx->d_acpart = nullptr;
    ctx->fermi_K = 0;
}

void free_current(tbpm_ctx *ctx)
{
    cudaFree(const_cast<int64_t *>(ctx->cur.slice_off));
    cudaFree(const_cast<int32_t *>(ctx->cur.cols));
    cudaFree(const_cast<double2 *>(ctx->cur.jx));
    cudaFree(const_cast<double2 *>(ctx->cur.jy));
    ctx->cur = CurrentOp();
    ctx->cur_nnz = 0;
}

// AC work buffers, allocated once per context.
int ensure_ac(tbpm_ctx *ctx)
{
    if (ctx->d_ac) return TBPM_OK;
    const size_t W = (size_t)ctx->nblk * (kBlockB1 / 32);
    const size_t vb = 3 * sizeof(double2) * (size_t)ctx->n_pad;
    cudaError_t e = cudaMalloc(&ctx->d_ac, vb);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_fnodes, sizeof(double) * 2 * kFermiCap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_fc, sizeof(double2) * kFermiCap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_gc, sizeof(double2) * kFermiCap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_kmax, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_acpart, sizeof(double2) * (kChunk + 1) * 4 * W);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_ac, 0, vb, ctx->stream);
    if (e != cudaSuccess) {
        free_ac(ctx);
        ctx->last_error = std::string("AC buffers: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? TBPM_ERR_OOM : TBPM_ERR_CUDA;
    }
    return TBPM_OK;
}

// Whether single-state time steps take the temporally blocked kernel: FP32
// lattice stencil without renormalisation, unless TBPM_F_NO_TBLOCK.
bool use_tblock(const tbpm_ctx *ctx)
{
    return (ctx->op == OP_STENCIL_MONO || ctx->op == OP_STENCIL_BI) && ctx->precision == TBPM_FP32 &&
           ctx->ninst == 0 && !(ctx->flags & (TBPM_F_RENORM | TBPM_F_NO_TBLOCK));
}

int tb_per(const tbpm_ctx *ctx) { return ctx->op == OP_STENCIL_MONO ? 2 : 4; }

// KPM moments on an FP32 lattice stencil run their passes blocked too.
bool use_tblock_kpm(const tbpm_ctx *ctx)
{
    return (ctx->op == OP_STENCIL_MONO || ctx->op == OP_STENCIL_BI) && ctx->precision == TBPM_FP32 &&
           !(ctx->flags & TBPM_F_NO_TBLOCK);
}

// The temporally blocked path's extra vectors (two b buffers, a second state).
int ensure_tb(tbpm_ctx *ctx)
{
    if (ctx->d_tb) return TBPM_OK;
    CU(tb_prepare(tb_per(ctx)));
    CU(tb_kpm_prepare(tb_per(ctx)));
    const size_t vb = 3 * sizeof(float2) * (size_t)ctx->n_pad;
    CU(cudaMalloc(&ctx->d_tb, vb));
    CU(cudaMemsetAsync(ctx->d_tb, 0, vb, ctx->stream));
    int t1, t2;
    ctx->tb_grid = std::min(ctx->num_sms, tb_tiles(tb_per(ctx), ctx->sten.l1, ctx->sten.l2, &t1, &t2));
    ctx->tb_kpm_grid = std::min(ctx->num_sms, tb_kpm_tiles(tb_per(ctx), ctx->sten.l1, ctx->sten.l2, &t1, &t2));
    return TBPM_OK;
}

// `len` single-state time steps by temporally blocked launches: each step runs
// its K - 1 sweeps as ceil((K-1)/kTbS) launches; blocks alternate between the
// b-buffer pairs (b0, b1) and (tb0, tb1), and each step writes psi(t_{n+1})
// to the other state buffer (a chunk of odd length copies it back, so every
// chunk ends with the state in d_psi). The final launch of step d writes the
// <psi0|psi> partials of slot d, one per block of the grid.
int enqueue_tb_chunk(tbpm_ctx *ctx, int K, int len, cudaStream_t s, int64_t *launches)
{
    const size_t vb = sizeof(float2) * (size_t)ctx->n_pad;
    char *tb = static_cast<char *>(ctx->d_tb);
    float2 *P[4] = {static_cast<float2 *>(ctx->d_b0), static_cast<float2 *>(ctx->d_b1),
                    reinterpret_cast<float2 *>(tb), reinterpret_cast<float2 *>(tb + vb)};
    float2 *S[2] = {static_cast<float2 *>(ctx->d_psi), reinterpret_cast<float2 *>(tb + 2 * vb)};
    TbParams p;
    memset(&p, 0, sizeof(p));
    p.L1 = (int)ctx->sten.l1;
    p.L2 = (int)ctx->sten.l2;
    const int per = tb_per(ctx);
    tb_tiles(per, ctx->sten.l1, ctx->sten.l2, &p.tiles1, &p.tiles2);
    p.t = (float)ctx->sten.t;
    p.t_perp = (float)ctx->sten.t_perp;
    p.onsite = static_cast<const float *>(ctx->sten.onsite);
    p.psi0 = static_cast<const float2 *>(ctx->d_psi0);
    p.partials = ctx->d_partials;
    p.coef = ctx->d_coef;
    p.K = K;
    const int grid = ctx->tb_grid;
    for (int d = 0; d < len; ++d) {
        p.psi = S[d & 1];
        p.psi_out = S[(d + 1) & 1];
        p.delta = d;
        int pair = 0;
        for (int j0 = 0; j0 < K - 1; j0 += kTbS) {
            p.j0 = j0;
            p.S = std::min(kTbS, K - 1 - j0);
            p.bx = P[2 * (pair ^ 1)];
            p.bz = P[2 * (pair ^ 1) + 1];
            p.ox = P[2 * pair];
            p.oz = P[2 * pair + 1];
            CU(launch_tb_block(per, p, grid, s));
            ++*launches;
            pair ^= 1;
        }
    }
    if (len & 1) CU(cudaMemcpyAsync(S[0], S[1], vb, cudaMemcpyDeviceToDevice, s));
    CU(launch_reduce_seg(ctx->d_partials, len, 1, (int64_t)grid, nullptr, 1, ctx->d_counter,
                         1, ctx->d_out, 0, s));
    CU(launch_advance(ctx->d_counter, len, s));
    *launches += 2;
    return TBPM_OK;
}

// `len` KPM passes (after the first) by blocked launches of up to kTbS passes:
// T_{m-1} in d_psi and T_m in d_b0 at the start; launches alternate between
// that pair and (tb0, tb1), and a chunk that ends on the other pair copies it
// back. The dots of pass d go to partial slot d as in enqueue_kpm_chunk.
constexpr int kTbKpmChunk = 2 * kTbS;   // two launches per full chunk

int enqueue_tbkpm_chunk(tbpm_ctx *ctx, int len, cudaStream_t s, int64_t *launches)
{
    const size_t vb = sizeof(float2) * (size_t)ctx->n_pad;
    char *tb = static_cast<char *>(ctx->d_tb);
    float2 *x0 = static_cast<float2 *>(ctx->d_b0), *z0 = static_cast<float2 *>(ctx->d_psi);
    float2 *x1 = reinterpret_cast<float2 *>(tb), *z1 = reinterpret_cast<float2 *>(tb + vb);
    TbParams p;
    memset(&p, 0, sizeof(p));
    const int per = tb_per(ctx);
    p.L1 = (int)ctx->sten.l1;
    p.L2 = (int)ctx->sten.l2;
    tb_kpm_tiles(per, ctx->sten.l1, ctx->sten.l2, &p.tiles1, &p.tiles2);
    p.t = (float)ctx->sten.t;
    p.t_perp = (float)ctx->sten.t_perp;
    p.onsite = static_cast<const float *>(ctx->sten.onsite);
    p.partials = ctx->d_partials;
    const int grid = ctx->tb_kpm_grid;
    int pr = 0;
    for (int d0 = 0; d0 < len; d0 += kTbS) {
        p.S = std::min(kTbS, len - d0);
        p.delta = d0;
        p.bx = pr ? x1 : x0;
        p.bz = pr ? z1 : z0;
        p.ox = pr ? x0 : x1;
        p.oz = pr ? z0 : z1;
        CU(launch_tb_kpm(per, p, grid, s));
        ++*launches;
        pr ^= 1;
    }
    if (pr) {
        CU(cudaMemcpyAsync(x0, x1, vb, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(z0, z1, vb, cudaMemcpyDeviceToDevice, s));
    }
    CU(launch_reduce_seg(ctx->d_partials, len, 2, (int64_t)grid, nullptr, 1, ctx->d_counter, 1,
                         ctx->d_out, 0, s));
    CU(launch_advance(ctx->d_counter, len, s));
    *launches += 2;
    return TBPM_OK;
}

// Runs (and on first use captures) the graph of one chunk.
int run_chunk(tbpm_ctx *ctx, int kind, int K, int len, int64_t *launches, int64_t ld = 0)
{
    // kind 0: DOS, one state; 1: KPM, one state; 2: DOS, 16 states; 3: DOS, batch of
    // instances (ld = n_steps + 1 for kinds 2 and 3); 4: Haydock (ld = M); 5: DOS with
    // quasi-eigenstate accumulation (one state; dropped at the end of the call);
    // 6: AC correlation (three states and the current-operator dots); 7: DOS, one
    // state, temporally blocked stencil sweeps; 8: KPM, temporally blocked passes
    const auto key = std::make_tuple(kind, len, K, (int)ld);
    auto it = ctx->graphs.find(key);
    int64_t nl = 0;
    if (it == ctx->graphs.end()) {
        cudaGraph_t g;
        CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = kind == 1   ? enqueue_kpm_chunk(ctx, len, ctx->cap_stream, &nl)
                 : kind == 4 ? enqueue_hay_chunk(ctx, len, (int)ld, ctx->cap_stream, &nl)
                 : kind == 6 ? enqueue_ac_chunk(ctx, K, len, ctx->cap_stream, &nl)
                 : kind == 7 ? enqueue_tb_chunk(ctx, K, len, ctx->cap_stream, &nl)
                 : kind == 8 ? enqueue_tbkpm_chunk(ctx, len, ctx->cap_stream, &nl)
                             : enqueue_dos_chunk(ctx, K, len, kind == 2 ? 16 : 1, ld, ctx->cap_stream, &nl,
                                                 kind == 5);
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (rc) return rc;
        CU(e);
        cudaGraphExec_t ex;
        cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CU(ei);
        it = ctx->graphs.emplace(key, ex).first;
    } else {
        nl = kind == 1   ? (int64_t)len + 2
             : kind == 4 ? 2 * (int64_t)len
             : kind == 6 ? (int64_t)len * (3 * (K - 1) + 1) + 2
             : kind == 7 ? (int64_t)len * ((K - 2) / kTbS + 1) + 2
             : kind == 8 ? (int64_t)(len + kTbS - 1) / kTbS + 2
                         : (int64_t)len * (K - 1) + 2;
        if (kind != 1 && kind != 4 && (ctx->flags & TBPM_F_RENORM)) nl += len;
        if (kind == 5) nl += len;
    }
    CU(cudaGraphLaunch(it->second, ctx->stream));
    *launches += nl;
    return TBPM_OK;
}

// Copies caller input (host or device, FP64 complex) for state j to a device
// pointer usable by the load kernel.
int stage_input(tbpm_ctx *ctx, const double *src, bool src_dev, size_t doubles, const double **out)
{
    if (src_dev) {
        *out = src;
        return TBPM_OK;
    }
    CU(cudaMemcpyAsync(ctx->d_stage, src, doubles * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    *out = ctx->d_stage;
    return TBPM_OK;
}

int classify(tbpm_ctx *ctx, const void *p, bool *dev)
{
    bool bad = false;
    *dev = is_device_ptr(p, ctx->device, &bad);
    return bad ? TBPM_ERR_ARG : TBPM_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

int tbpm_default_opts(tbpm_opts *o)
{
    if (!o) return TBPM_ERR_ARG;
    o->precision = TBPM_FP64;
    o->path = TBPM_PATH_AUTO;
    o->flags = 0;
    o->device = -1;
    o->stream = nullptr;
    o->bessel_tol = 0.0;
    o->block_threads = 0;
    o->slices_per_warp = 0;
    return TBPM_OK;
}

const char *tbpm_strerror(int s)
{
    switch (s) {
    case TBPM_OK: return "ok";
    case TBPM_ERR_ARG: return "invalid argument";
    case TBPM_ERR_CSR: return "malformed CSR matrix";
    case TBPM_ERR_NOT_HERMITIAN: return "matrix is not Hermitian";
    case TBPM_ERR_RESCALE: return "rescale below the Gershgorin bound of H";
    case TBPM_ERR_OOM: return "out of memory";
    case TBPM_ERR_CUDA: return "CUDA runtime error";
    case TBPM_ERR_TIMEOUT: return "bounded device wait timed out";
    case TBPM_ERR_NO_DEVICE: return "no usable sm_103 GPU";
    case TBPM_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

static int check_opts(const tbpm_opts *in, tbpm_opts *o)
{
    tbpm_default_opts(o);
    if (in) *o = *in;
    if (o->precision != TBPM_FP64 && o->precision != TBPM_FP32) return TBPM_ERR_ARG;
    if (o->path < TBPM_PATH_AUTO || o->path > TBPM_PATH_STENCIL) return TBPM_ERR_ARG;
    if (o->flags & ~(unsigned)(TBPM_F_NO_HERMITIAN_CHECK | TBPM_F_FORCE_RESCALE | TBPM_F_RENORM |
                               TBPM_F_NO_CLUSTER | TBPM_F_AUTOTUNE | TBPM_F_NO_TBLOCK | TBPM_F_NO_PDL |
                               TBPM_F_PLAIN_SELL))
        return TBPM_ERR_ARG;
    if (o->bessel_tol == 0.0) o->bessel_tol = 1e-12;
    if (!(o->bessel_tol > 0.0 && o->bessel_tol < 1e-2)) return TBPM_ERR_ARG;
    // 0 leaves the shape to the operator (apply_shape)
    if (o->block_threads != 0 && o->block_threads != 128 && o->block_threads != 256 && o->block_threads != 512 &&
        o->block_threads != 1024)
        return TBPM_ERR_ARG;
    if (o->slices_per_warp != 0 && o->slices_per_warp != 1 && o->slices_per_warp != 2 && o->slices_per_warp != 4)
        return TBPM_ERR_ARG;
    return TBPM_OK;
}

// Applies the requested launch shape of the single-state sweeps once the
// operator is known: TBPM_ERR_UNSUPPORTED if it is not built for this operator;
// the grid is whole waves of the shape's middle-sweep occupancy. Unset fields
// (0) take the operator's default: 512 threads and one slice per warp; for a
// stored matrix packed per entry, whose smaller entries leave its sweeps
// waiting on their dependent loads, 128 threads and four slices per warp
// (measured on GB300 for graphene 2048^2: 69.6 against 84.3 us per sweep at
// 512 x 1); packed per row, 256 threads and two slices (58.4 us, against 60.1
// at 128 x 4 and 61.0 at 512 x 1).
static int apply_shape(tbpm_ctx *ctx, const tbpm_opts &o)
{
    SweepVariant v = variant(ctx, 1);
    v.block = o.block_threads ? o.block_threads : v.packed == 2 ? 256 : v.packed == 1 ? 128 : kBlockB1;
    v.spw = o.slices_per_warp ? o.slices_per_warp : v.packed == 2 ? 2 : v.packed == 1 ? 4 : 1;
    if (v.block != kBlockB1 || v.spw != 1) {
        if (!sweep_shape_built(v)) return TBPM_ERR_UNSUPPORTED;
        const int occ = sweep_shape_occupancy(v, ctx->d_slice_inst != nullptr);
        if (occ < 1) return TBPM_ERR_UNSUPPORTED;
        ctx->sw_block = v.block;
        ctx->sw_spw = v.spw;
        ctx->nblk = occ * ctx->num_sms;
    }
    set_kind_grids(ctx);
    return TBPM_OK;
}

static int finish_create(tbpm_ctx *ctx, const tbpm_opts &o)
{
    int rc = init_device(ctx, o);
    if (rc) return rc;
    ctx->nblk = sweep_grid(variant(ctx, 1), ctx->num_sms);
    ctx->nblk_kpm = kpm_grid(variant(ctx, 1), ctx->num_sms);
    ctx->nblk16 = sweep_grid_b16(ctx->num_sms);
    return TBPM_OK;
}

// Autotuner (TBPM_F_AUTOTUNE): times whole time steps of this context's
// operator (the K = 18 sweep sequence of x = pi: first, second, 14 middle and
// the final sweep with its dot partials) over launch shapes: block widths of
// 128, 256, 512 and 1024 threads, 1, 2 or 4 consecutive 32-row slices per warp
// iteration (the shapes sweep_shape_built accepts for this operator), and for
// each the grids of occupancy/2, occupancy and twice the occupancy blocks per
// SM (all of 1 .. occupancy when that is at most 4). Every candidate is timed
// over 2 steps after one warm-up step; the four fastest and the context's shape
// before tuning (its default) are timed again over 6 steps,
// and the fastest of those is kept for the life of the context. The
// single-instance dot partials are per warp of the chosen grid, which is then
// fixed, so results stay reproducible from call to call. Runs once, before any
// graph is captured; the sweeps run on zero coefficients and overwrite the
// work vectors, which every call initialises.
static int autotune(tbpm_ctx *ctx)
{
    if (ctx->tuned) return TBPM_OK;
    int rc;
    if ((rc = ensure_work(ctx, 1, 1, 0))) return rc;
    CU(cudaMemsetAsync(ctx->d_coef, 0, sizeof(double2) * kMaxTerms * std::max(1, ctx->ninst), ctx->stream));
    ctx->K_cached = -1;
    ctx->dt_cached.clear();
    const bool multi = ctx->d_slice_inst != nullptr;
    struct Cand {
        int block, spw, grid;
        double us;
    };
    std::vector<Cand> cands;
    const SweepVariant base = variant(ctx, 1);
    // the context's shape before tuning: the default, or the packed default
    const int def_grid = ctx->nblk, def_block = ctx->sw_block, def_spw = ctx->sw_spw;
    int64_t max_warps = 0;
    for (int block : {128, 256, 512, 1024})
        for (int spw : {1, 2, 4}) {
            SweepVariant v = base;
            v.block = block;
            v.spw = spw;
            if (!sweep_shape_built(v)) continue;
            const int occ = sweep_shape_occupancy(v, multi);
            if (occ < 1) continue;
            std::vector<int> ks;
            if (occ <= 4)
                for (int k = 1; k <= occ; ++k) ks.push_back(k);
            else
                ks = {occ / 2, occ};
            ks.push_back(2 * occ);
            for (int k : ks) cands.push_back({block, spw, k * ctx->num_sms, 0.0});
            // the final sweep's partials, per warp of its own grid
            max_warps = std::max<int64_t>(max_warps, (int64_t)kind_grid(ctx, v, SW_FINAL) * block / 32);
        }
    bool have_def = false;
    for (const Cand &c : cands) have_def |= c.block == def_block && c.spw == def_spw && c.grid == def_grid;
    if (!have_def) cands.push_back({def_block, def_spw, def_grid, 0.0});
    // the final sweep's per-warp partials (slot 0) of the widest candidate shape
    double2 *part = ctx->d_partials;
    double2 *own_part = nullptr;
    if (!multi && (size_t)max_warps > ctx->partials_cap) {
        CU(cudaMalloc(&own_part, sizeof(double2) * (size_t)max_warps));
        part = own_part;
    }
    SweepParams p;
    fill_operator(ctx, p);
    p.coef = ctx->d_coef;
    p.psi = ctx->d_psi;
    p.psi0 = ctx->d_psi0;
    p.partials = part;
    p.delta = 0;
    p.slice_inst = ctx->d_slice_inst;
    void *Bv[2] = {ctx->d_b0, ctx->d_b1};
    constexpr int Kt = 18;
    auto step = [&](const SweepVariant &v, int grid) -> cudaError_t {
        cudaError_t e;
        p.x = ctx->d_psi; p.z = nullptr; p.y = Bv[0];
        p.ia = Kt - 2; p.ib = -1; p.ic = Kt - 1; p.bscale = 1.0;
        if ((e = launch_sweep(v, SW_FIRST, false, false, p, kind_grid(ctx, v, SW_FIRST), ctx->stream)) != cudaSuccess)
            return e;
        p.x = Bv[0]; p.y = Bv[1];
        p.ia = Kt - 3; p.ib = Kt - 1; p.ic = -1;
        if ((e = launch_sweep(v, SW_SECOND, true, false, p, kind_grid(ctx, v, SW_SECOND), ctx->stream)) != cudaSuccess)
            return e;
        for (int k = Kt - 4; k >= 1; --k) {
            p.x = Bv[(Kt - 3 - k) & 1];
            p.y = Bv[(Kt - 2 - k) & 1];
            p.z = p.y;
            p.ia = k; p.ib = -1; p.ic = -1;
            if ((e = launch_sweep(v, SW_MID, (k & 1) != 0, true, p, grid, ctx->stream)) != cudaSuccess) return e;
        }
        p.x = Bv[(Kt - 3) & 1];
        p.z = Bv[(Kt - 4) & 1];
        p.y = ctx->d_psi;
        p.ia = 0; p.ib = -1; p.ic = -1; p.bscale = 0.5;
        return launch_sweep(v, SW_FINAL, false, true, p, kind_grid(ctx, v, SW_FINAL), ctx->stream);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto time_us = [&](const Cand &c, int reps, double *us) -> int {
        SweepVariant v = base;
        v.block = c.block;
        v.spw = c.spw;
        CU(step(v, c.grid));                                                // warm
        CU(cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < reps; ++r) CU(step(v, c.grid));
        CU(cudaEventRecord(e1, ctx->stream));
        CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        *us = 1e3 * ms / reps / (Kt - 1);                                  // per sweep
        return TBPM_OK;
    };
    std::vector<Cand> fin;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = TBPM_ERR_CUDA;
        ctx->last_error = "autotune: cudaEventCreate failed";
    }
    for (size_t i = 0; i < cands.size() && !rc; ++i) rc = time_us(cands[i], 2, &cands[i].us);
    if (!rc) {
        std::vector<Cand> sorted = cands;
        std::sort(sorted.begin(), sorted.end(), [](const Cand &a, const Cand &b) { return a.us < b.us; });
        for (size_t i = 0; i < sorted.size() && i < 4; ++i) fin.push_back(sorted[i]);
        bool def_in = false;
        for (const Cand &c : fin) def_in |= c.block == def_block && c.spw == def_spw && c.grid == def_grid;
        if (!def_in) fin.push_back({def_block, def_spw, def_grid, 0.0});
        for (size_t i = 0; i < fin.size() && !rc; ++i) rc = time_us(fin[i], 6, &fin[i].us);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (own_part) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(own_part);
    }
    if (rc) return rc;
    Cand best = fin[0];
    double def_us = 0.0;
    for (const Cand &c : fin) {
        if (c.us < best.us) best = c;
        if (c.block == def_block && c.spw == def_spw && c.grid == def_grid) def_us = c.us;
    }
    // work buffers and graphs depend on the shape: rebuild them for the new one
    destroy_graphs(ctx);
    ctx->nblk = best.grid;
    ctx->sw_block = best.block;
    ctx->sw_spw = best.spw;
    set_kind_grids(ctx);
    ctx->cap_states = 0;
    ctx->tuned = true;
    ctx->tune_candidates = (int)cands.size();
    ctx->tune_default_us = def_us;
    ctx->tune_best_us = best.us;
    return TBPM_OK;
}

int tbpm_create(tbpm_ctx **out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const double *val, double rescale, const tbpm_opts *opts)
{
    if (!out) return TBPM_ERR_ARG;
    *out = nullptr;
    tbpm_opts o;
    int rc = check_opts(opts, &o);
    if (rc) return rc;
    if (n < 1 || n >= ((int64_t)1 << 31) - kSlice || !row_ptr) return TBPM_ERR_ARG;
    if (row_ptr[n] > 0 && (!col || !val)) return TBPM_ERR_ARG;
    if (!(rescale > 0.0) || !std::isfinite(rescale)) return TBPM_ERR_ARG;
    if (o.path == TBPM_PATH_STENCIL) return TBPM_ERR_ARG;
    HostMatrix m;
    try {
        rc = build_host_matrix(n, row_ptr, col, val, !(o.flags & TBPM_F_NO_HERMITIAN_CHECK), m);
    } catch (const std::bad_alloc &) {
        return TBPM_ERR_OOM;
    }
    if (rc) return rc;
    if (m.gershgorin > rescale && !(o.flags & TBPM_F_FORCE_RESCALE)) return TBPM_ERR_RESCALE;
    tbpm_ctx *ctx = new (std::nothrow) tbpm_ctx;
    if (!ctx) return TBPM_ERR_OOM;
    ctx->precision = o.precision;
    ctx->path = TBPM_PATH_SELL;
    ctx->flags = o.flags;
    ctx->tol = o.bessel_tol;
    ctx->n = n;
    ctx->n_pad = (n + kSlice - 1) / kSlice * kSlice;
    ctx->rescale = rescale;
    ctx->gershgorin = m.gershgorin;
    if ((rc = finish_create(ctx, o)) || (rc = setup_sell(ctx, m)) || (rc = apply_shape(ctx, o)) ||
        ((o.flags & TBPM_F_AUTOTUNE) && (rc = autotune(ctx)))) {
        tbpm_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return TBPM_OK;
}

int tbpm_create_lattice(tbpm_ctx **out, const tbpm_lattice *lat, double rescale,
                        const tbpm_opts *opts)
{
    if (!out || !lat) return TBPM_ERR_ARG;
    *out = nullptr;
    tbpm_opts o;
    int rc = check_opts(opts, &o);
    if (rc) return rc;
    if (lat->kind != TBPM_LATTICE_GRAPHENE && lat->kind != TBPM_LATTICE_AB_BILAYER) return TBPM_ERR_ARG;
    if (lat->l1 < 3 || lat->l2 < 3) return TBPM_ERR_ARG;
    const int per = lat->kind == TBPM_LATTICE_GRAPHENE ? 2 : 4;
    if (lat->l1 > ((int64_t)1 << 30) / lat->l2 / per) return TBPM_ERR_ARG;
    const int64_t n = lat->l1 * lat->l2 * per;
    if (!std::isfinite(lat->t) || !std::isfinite(lat->t_perp)) return TBPM_ERR_ARG;
    if (!(rescale > 0.0) || !std::isfinite(rescale)) return TBPM_ERR_ARG;
    double maxe = 0.0;
    if (lat->onsite)
        for (int64_t i = 0; i < n; ++i) {
            if (!std::isfinite(lat->onsite[i])) return TBPM_ERR_ARG;
            maxe = std::max(maxe, std::fabs(lat->onsite[i]));
        }
    const double gersh = 3.0 * std::fabs(lat->t) + (per == 4 ? std::fabs(lat->t_perp) : 0.0) + maxe;
    if (gersh > rescale && !(o.flags & TBPM_F_FORCE_RESCALE)) return TBPM_ERR_RESCALE;
    tbpm_ctx *ctx = new (std::nothrow) tbpm_ctx;
    if (!ctx) return TBPM_ERR_OOM;
    ctx->precision = o.precision;
    ctx->flags = o.flags;
    ctx->tol = o.bessel_tol;
    ctx->n = n;
    ctx->n_pad = (n + kSlice - 1) / kSlice * kSlice;
    ctx->rescale = rescale;
    ctx->gershgorin = gersh;
    rc = finish_create(ctx, o);
    if (!rc) {
        if (o.path == TBPM_PATH_SELL) {
            HostMatrix m;
            try {
                lattice_to_host_matrix(*lat, m);
                ctx->path = TBPM_PATH_SELL;
                rc = setup_sell(ctx, m);
            } catch (const std::bad_alloc &) {
                rc = TBPM_ERR_OOM;
            }
        } else {
            ctx->path = TBPM_PATH_STENCIL;
            ctx->op = per == 2 ? OP_STENCIL_MONO : OP_STENCIL_BI;
            // grids in whole waves of this operator's kernels
            ctx->nblk = sweep_grid(variant(ctx, 1), ctx->num_sms);
            ctx->nblk_kpm = kpm_grid(variant(ctx, 1), ctx->num_sms);
            ctx->sten.kind = lat->kind;
            ctx->sten.l1 = lat->l1;
            ctx->sten.l2 = lat->l2;
            const double s = 2.0 / rescale;
            ctx->sten.t = s * lat->t;
            ctx->sten.t_perp = s * lat->t_perp;
            if (lat->onsite) {
                if (ctx->precision == TBPM_FP64) {
                    std::vector<double> e(ctx->n_pad, 0.0);
                    for (int64_t i = 0; i < n; ++i) e[i] = s * lat->onsite[i];
                    rc = upload(ctx, &ctx->sten.onsite, e);
                } else {
                    std::vector<float> e(ctx->n_pad, 0.0f);
                    for (int64_t i = 0; i < n; ++i) e[i] = (float)(s * lat->onsite[i]);
                    rc = upload(ctx, &ctx->sten.onsite, e);
                }
            }
        }
    }
    if (!rc) rc = apply_shape(ctx, o);
    if (!rc && (o.flags & TBPM_F_AUTOTUNE)) rc = autotune(ctx);
    if (rc) {
        tbpm_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return TBPM_OK;
}

void tbpm_destroy(tbpm_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_graphs(ctx);
    cudaFree(ctx->sell.slice_off); cudaFree(ctx->sell.cols); cudaFree(ctx->sell.vals);
    cudaFree(ctx->sell.diag); cudaFree(ctx->sten.onsite);
    cudaFree(ctx->sell.cdelta); cudaFree(ctx->sell.vidx); cudaFree(ctx->sell.vtab); cudaFree(ctx->sell.rowpack);
    cudaFree(ctx->d_coef); cudaFree(ctx->d_K); cudaFree(ctx->d_counter);
    cudaFree(ctx->d_psi); cudaFree(ctx->d_b0); cudaFree(ctx->d_b1); cudaFree(ctx->d_psi0);
    cudaFree(ctx->d_partials); cudaFree(ctx->d_out); cudaFree(ctx->d_stage); cudaFree(ctx->d_misc);
    cudaFree(ctx->d_norm); cudaFree(ctx->d_scale);
    cudaFree(ctx->d_slice_inst); cudaFree(ctx->d_seg_off); cudaFree(ctx->d_cpart);
    cudaFree(ctx->d_qe); cudaFree(ctx->d_qe_e);
    free_ac(ctx);
    free_current(ctx);
    cudaFree(ctx->d_tb);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

// Time evolution of nstates states: C(t_n) into corr and/or psi(t_{n_steps})
// into psi_out (either may be null, not both).
static int run_dos(tbpm_ctx *ctx, const double *psi0, int nstates, double dt, int n_steps,
                   double *corr, double *psi_out)
{
    if (!ctx || !psi0 || (!corr && !psi_out) || nstates < 1 || n_steps < 0) return TBPM_ERR_ARG;
    if (ctx->ninst > 0) return TBPM_ERR_UNSUPPORTED;
    if (!(dt != 0.0) || !std::isfinite(dt)) return TBPM_ERR_ARG;
    const double x = dt * ctx->rescale;
    if (!(std::fabs(x) <= 40.0)) return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, out_dev = true, psi_dev = true;
    int rc;
    if ((rc = classify(ctx, psi0, &in_dev)) || (corr && (rc = classify(ctx, corr, &out_dev))) ||
        (psi_out && (rc = classify(ctx, psi_out, &psi_dev))))
        return rc;
    const bool renorm = (ctx->flags & TBPM_F_RENORM) != 0;
    // copies state `col` of an interleaved buffer to psi_out (state j)
    auto store = [&](int B, int col, int j) -> int {
        double *dst = psi_out + (size_t)2 * ctx->n * j;
        double *d = psi_dev ? dst : ctx->d_stage;
        CU(launch_store_column(ctx->precision, ctx->d_psi, ctx->n, B, col, renorm ? ctx->d_scale : nullptr, d,
                               ctx->stream));
        if (!psi_dev) {
            CU(cudaMemcpyAsync(dst, d, sizeof(double2) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
        }
        return TBPM_OK;
    };
    int K;
    if ((rc = ensure_coeffs(ctx, x, &K))) return rc;
    const int Ke = std::max(K, 3);
    const int64_t n = ctx->n;
    int64_t launches = 0;
    // FP32 with several states: blocks of 16 states per sweep, except on the
    // monolayer stencil, where there is no stored matrix to share and the
    // temporally blocked single-state kernel runs the states one after another
    if (ctx->precision == TBPM_FP32 && nstates > 1 && !use_tblock(ctx)) {
        // blocks of 16 states advance together; missing states of the last
        // block are zero vectors, which stay zero
        const int B = kMaxBlockStates;
        const int64_t ld = (int64_t)n_steps + 1;
        if ((rc = ensure_work(ctx, B, (size_t)B * ld, (in_dev && psi_dev) ? 0 : (size_t)2 * n))) return rc;
        const size_t vb = vec_bytes(ctx->precision) * (size_t)ctx->n_pad * B;
        for (int j0 = 0; j0 < nstates; j0 += B) {
            const int nb = std::min(B, nstates - j0);
            if (in_dev) {
                CU(launch_load_states(ctx->precision, psi0, n, ctx->n_pad, nstates, j0, B, ctx->d_psi0,
                                      ctx->d_psi, ctx->stream));
                ++launches;
            } else {
                CU(cudaMemsetAsync(ctx->d_psi0, 0, vb, ctx->stream));
                CU(cudaMemsetAsync(ctx->d_psi, 0, vb, ctx->stream));
                for (int q = 0; q < nb; ++q) {
                    const double *src;
                    if ((rc = stage_input(ctx, psi0 + (size_t)2 * n * (j0 + q), false, (size_t)2 * n, &src)))
                        return rc;
                    CU(launch_load_column(ctx->precision, src, n, B, q, ctx->d_psi0, ctx->d_psi, ctx->stream));
                    CU(cudaStreamSynchronize(ctx->stream));        // staging reuse
                    ++launches;
                }
            }
            CU(launch_dot_b16(ctx->d_psi0, ctx->d_psi0, ctx->n_pad / kSlice, ctx->d_partials, ctx->nblk16,
                              ctx->stream));
            CU(launch_reduce_b16(ctx->d_partials, 1, ctx->nblk16, nullptr, 0, ctx->d_out, ld, ctx->stream));
            CU(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
            launches += 2;
            if (ctx->flags & TBPM_F_RENORM) {
                CU(launch_renorm(nullptr, 0, B, ctx->d_scale, ctx->stream));
                ++launches;
            }
            int done = 0;
            while (done < n_steps) {
                const int len = std::min(kChunk, n_steps - done);
                if ((rc = run_chunk(ctx, 2, Ke, len, &launches, ld))) return rc;
                done += len;
            }
            if (corr) {
                CU(cudaMemcpyAsync(corr + (size_t)2 * ld * j0, ctx->d_out, sizeof(double2) * ld * nb,
                                   out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
                if (!out_dev) CU(cudaStreamSynchronize(ctx->stream));
            }
            if (psi_out)
                for (int q = 0; q < nb; ++q)
                    if ((rc = store(B, q, j0 + q))) return rc;
        }
        if (!out_dev || !in_dev) CU(cudaStreamSynchronize(ctx->stream));
        CU(cudaGetLastError());
        ctx->last_K = Ke;
        ctx->last_passes = (int64_t)((nstates + B - 1) / B) * n_steps * (Ke - 1);
        ctx->last_launches = launches;
        return TBPM_OK;
    }
    if ((rc = ensure_work(ctx, 1, (size_t)n_steps + 1, (in_dev && psi_dev) ? 0 : (size_t)2 * n))) return rc;
    int clr, cnc;
    size_t csm;
    const bool use_cluster = ctx->op == OP_SELL && !(ctx->flags & (TBPM_F_NO_CLUSTER | TBPM_F_RENORM)) &&
                             cluster_fits(ctx->precision, ctx->n_pad, &clr, &cnc, &csm);
    for (int j = 0; j < nstates; ++j) {
        const double *src;
        if ((rc = stage_input(ctx, psi0 + (size_t)2 * n * j, in_dev, (size_t)2 * n, &src))) return rc;
        CU(launch_load_states(ctx->precision, src, n, ctx->n_pad, 1, 0, 1, ctx->d_psi0, ctx->d_psi,
                              ctx->stream));
        CU(launch_dot(ctx->precision, ctx->d_psi0, ctx->d_psi0, ctx->n_pad / kSlice, ctx->d_partials, ctx->nblk,
                      false, ctx->stream));
        CU(launch_reduce_seg(ctx->d_partials, 1, 1, (int64_t)ctx->nblk * (kBlockB1 / 32), nullptr, 1, nullptr, 0,
                             ctx->d_out, 0, ctx->stream));
        CU(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
        launches += 3;
        if (ctx->flags & TBPM_F_RENORM) {
            CU(launch_renorm(nullptr, 0, 1, ctx->d_scale, ctx->stream));
            ++launches;
        }
        int lr, ncta;
        size_t smem;
        const int64_t nsl = ctx->n_pad / kSlice;
        if (use_cluster && n_steps > 0) {
            // whole evolution in one launch of one cluster, then one reduction
            const size_t need = (size_t)n_steps * nsl;
            if (need > ctx->cpart_cap) {
                cudaFree(ctx->d_cpart);
                ctx->d_cpart = nullptr;
                ctx->cpart_cap = 0;
                CU(cudaMalloc(&ctx->d_cpart, need * sizeof(double2)));
                ctx->cpart_cap = need;
            }
            SweepParams op;
            fill_operator(ctx, op);
            CU(launch_cluster_dos(ctx->precision, ctx->sell.real_values, op, ctx->sell.max_width, ctx->d_psi0,
                                  ctx->d_coef, Ke,
                                  n_steps, ctx->d_cpart, psi_out ? ctx->d_psi : nullptr, ctx->stream));
            CU(launch_reduce_seg(ctx->d_cpart, n_steps, 1, nsl, nullptr, 1, nullptr, 1, ctx->d_out, 0,
                                 ctx->stream));
            launches += 2;
        } else {
            const bool tbk = use_tblock(ctx);
            if (tbk && (rc = ensure_tb(ctx))) return rc;
            int done = 0;
            while (done < n_steps) {
                const int len = std::min(kChunk, n_steps - done);
                if ((rc = run_chunk(ctx, tbk ? 7 : 0, Ke, len, &launches))) return rc;
                done += len;
            }
        }
        (void)lr; (void)ncta; (void)smem;
        if (corr) {
            double *dst = corr + (size_t)2 * (n_steps + 1) * j;
            CU(cudaMemcpyAsync(dst, ctx->d_out, sizeof(double2) * (n_steps + 1),
                               out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (psi_out && (rc = store(1, 0, j))) return rc;
        if (!in_dev && nstates > 1) CU(cudaStreamSynchronize(ctx->stream));  // staging reuse
    }
    if (!out_dev || !in_dev) CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGetLastError());
    ctx->last_K = Ke;
    ctx->last_passes = (int64_t)nstates * n_steps * (Ke - 1);
    ctx->last_launches = launches;
    return TBPM_OK;
}

int tbpm_dos_corr(tbpm_ctx *ctx, const double *psi0, int nstates, double dt, int n_steps,
                  double *corr)
{
    if (!corr) return TBPM_ERR_ARG;
    return run_dos(ctx, psi0, nstates, dt, n_steps, corr, nullptr);
}

int tbpm_propagate(tbpm_ctx *ctx, const double *psi0, int nstates, double dt, int n_steps,
                   double *psi_out, double *corr)
{
    if (!psi_out) return TBPM_ERR_ARG;
    return run_dos(ctx, psi0, nstates, dt, n_steps, corr, psi_out);
}

int kpm_moments(tbpm_ctx *ctx, const double *psi0, int nstates, int M, double *mu)
{
    if (!ctx || !psi0 || !mu || nstates < 1 || M < 1) return TBPM_ERR_ARG;
    if (ctx->ninst > 0) return TBPM_ERR_UNSUPPORTED;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, out_dev;
    int rc;
    if ((rc = classify(ctx, psi0, &in_dev)) || (rc = classify(ctx, mu, &out_dev))) return rc;
    const int64_t n = ctx->n;
    const int P = (M + 1) / 2 - 1;                        // sweeps after the first
    const size_t ndots = 2 * (size_t)(P + 1);
    if ((rc = ensure_work(ctx, 1, ndots + (size_t)M, in_dev ? 0 : (size_t)2 * n))) return rc;
    const SweepVariant v = variant(ctx, 1);
    int64_t launches = 0;
    for (int j = 0; j < nstates; ++j) {
        const double *src;
        if ((rc = stage_input(ctx, psi0 + (size_t)2 * n * j, in_dev, (size_t)2 * n, &src))) return rc;
        CU(launch_load_states(ctx->precision, src, n, ctx->n_pad, 1, 0, 1, ctx->d_psi0, ctx->d_psi,
                              ctx->stream));
        // first sweep: T_1 = A T_0 / 2 into B0, dots (<T_0|T_0>, <T_1|T_0>) -> dots[0..1]
        SweepParams op;
        fill_operator(ctx, op);
        KpmParams p;
        memset(&p, 0, sizeof(p));
        p.n = op.n; p.nslices = op.nslices; p.slice_off = op.slice_off; p.cols = op.cols;
        p.vals = op.vals; p.diag = op.diag; p.l1 = op.l1; p.l2 = op.l2; p.t = op.t; p.t_perp = op.t_perp;
        p.cdelta = op.cdelta; p.vidx = op.vidx; p.vtab = op.vtab; p.rowpack = op.rowpack; p.npad = op.npad;
        p.x = ctx->d_psi; p.y = ctx->d_b0; p.scale = 0.5; p.first = true;
        p.partials = ctx->d_partials; p.delta = 0; p.nblk = ctx->nblk_kpm;
        CU(launch_kpm(v, p, ctx->nblk_kpm, ctx->stream));
        CU(launch_reduce_seg(ctx->d_partials, 1, 2, (int64_t)ctx->nblk_kpm * (kBlockB1 / 32), nullptr, 1, nullptr, 0,
                             ctx->d_out, 0, ctx->stream));
        CU(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
        launches += 3;
        const bool tbk = use_tblock_kpm(ctx);
        if (tbk && (rc = ensure_tb(ctx))) return rc;
        int done = 0;
        while (done < P) {
            const int len = std::min(tbk ? kTbKpmChunk : kChunk, P - done);
            if ((rc = run_chunk(ctx, tbk ? 8 : 1, 0, len, &launches))) return rc;
            done += len;
        }
        double2 *dmu = ctx->d_out + ndots;
        CU(launch_kpm_finalize(ctx->d_out, M, 1, dmu, ctx->stream));
        ++launches;
        double *dst = mu + (size_t)2 * M * j;
        CU(cudaMemcpyAsync(dst, dmu, sizeof(double2) * M,
                           out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
        if (!in_dev && nstates > 1) CU(cudaStreamSynchronize(ctx->stream));
    }
    if (!out_dev || !in_dev) CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGetLastError());
    ctx->last_passes = (int64_t)nstates * (P + 1);
    ctx->last_launches = launches;
    return TBPM_OK;
}

int tbpm_dos_from_corr(tbpm_ctx *ctx, const double *corr, int n_steps, double dt,
                       double *energies, double *dos)
{
    if (!ctx || !corr || !energies || !dos || n_steps < 1) return TBPM_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt) || n_steps > (1 << 28)) return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, e_dev, d_dev;
    int rc;
    if ((rc = classify(ctx, corr, &in_dev)) || (rc = classify(ctx, energies, &e_dev)) ||
        (rc = classify(ctx, dos, &d_dev)))
        return rc;
    const size_t nc = (size_t)n_steps + 1, ne = 2 * (size_t)n_steps;
    if ((rc = ensure_work(ctx, 1, 0, 2 * nc + 2 * ne))) return rc;
    const double2 *c = reinterpret_cast<const double2 *>(corr);
    if (!in_dev) {
        CU(cudaMemcpyAsync(ctx->d_stage, corr, nc * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        c = reinterpret_cast<const double2 *>(ctx->d_stage);
    }
    double *de = e_dev ? energies : ctx->d_stage + 2 * nc;
    double *dd = d_dev ? dos : ctx->d_stage + 2 * nc + ne;
    CU(launch_dos_hann(c, n_steps, dt, de, dd, ctx->stream));
    if (!e_dev) CU(cudaMemcpyAsync(energies, de, ne * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (!d_dev) CU(cudaMemcpyAsync(dos, dd, ne * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (!in_dev || !e_dev || !d_dev) CU(cudaStreamSynchronize(ctx->stream));
    ctx->last_launches = 1;
    return TBPM_OK;
}

int kpm_dos_jackson(tbpm_ctx *ctx, const double *mu, int M, int n_e, double *energies,
                    double *rho_out)
{
    if (!ctx || !mu || !energies || !rho_out || M < 1 || n_e < 1) return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, e_dev, r_dev;
    int rc;
    if ((rc = classify(ctx, mu, &in_dev)) || (rc = classify(ctx, energies, &e_dev)) ||
        (rc = classify(ctx, rho_out, &r_dev)))
        return rc;
    if ((rc = ensure_work(ctx, 1, 0, 2 * (size_t)M + 2 * (size_t)n_e))) return rc;
    const double2 *m = reinterpret_cast<const double2 *>(mu);
    if (!in_dev) {
        CU(cudaMemcpyAsync(ctx->d_stage, mu, M * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        m = reinterpret_cast<const double2 *>(ctx->d_stage);
    }
    double *de = e_dev ? energies : ctx->d_stage + 2 * (size_t)M;
    double *dr = r_dev ? rho_out : ctx->d_stage + 2 * (size_t)M + n_e;
    CU(launch_kpm_dos(m, M, n_e, ctx->rescale, de, dr, ctx->stream));
    if (!e_dev) CU(cudaMemcpyAsync(energies, de, n_e * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (!r_dev) CU(cudaMemcpyAsync(rho_out, dr, n_e * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (!in_dev || !e_dev || !r_dev) CU(cudaStreamSynchronize(ctx->stream));
    ctx->last_launches = 1;
    return TBPM_OK;
}

int tbpm_create_batch(tbpm_ctx **out, int ninst, const tbpm_instance *inst, const tbpm_opts *opts)
{
    if (!out) return TBPM_ERR_ARG;
    *out = nullptr;
    if (ninst < 1 || ninst > 4096 || !inst) return TBPM_ERR_ARG;
    tbpm_opts o;
    int rc = check_opts(opts, &o);
    if (rc) return rc;
    if (o.path == TBPM_PATH_STENCIL) return TBPM_ERR_ARG;
    // validate every instance, then assemble the block-diagonal operator
    HostMatrix all;
    std::vector<int64_t> rows(ninst + 1, 0);
    std::vector<double> row_scale;
    double gmax = 0.0, rmax = 0.0;
    try {
        for (int g = 0; g < ninst; ++g) {
            const tbpm_instance &I = inst[g];
            if (I.n < 1 || !I.row_ptr || (I.row_ptr[I.n] > 0 && (!I.col || !I.val))) return TBPM_ERR_ARG;
            if (!(I.rescale > 0.0) || !std::isfinite(I.rescale)) return TBPM_ERR_ARG;
            rows[g + 1] = rows[g] + (I.n + kSlice - 1) / kSlice * kSlice;
            if (rows[g + 1] >= ((int64_t)1 << 31) - kSlice) return TBPM_ERR_ARG;
        }
        const int64_t ntot = rows[ninst];
        all.n = ntot;
        all.rp.assign(ntot + 1, 0);
        all.diag.assign(ntot, 0.0);
        all.real_values = true;
        row_scale.assign(ntot, 0.0);
        for (int g = 0; g < ninst; ++g) {
            const tbpm_instance &I = inst[g];
            HostMatrix m;
            rc = build_host_matrix(I.n, I.row_ptr, I.col, I.val, !(o.flags & TBPM_F_NO_HERMITIAN_CHECK), m);
            if (rc) return rc;
            if (m.gershgorin > I.rescale && !(o.flags & TBPM_F_FORCE_RESCALE)) return TBPM_ERR_RESCALE;
            gmax = std::max(gmax, m.gershgorin);
            rmax = std::max(rmax, I.rescale);
            all.real_values = all.real_values && m.real_values;
            const int64_t r0 = rows[g];
            for (int64_t i = 0; i < rows[g + 1] - r0; ++i) {
                const int64_t r = r0 + i;
                if (i < I.n) {
                    for (int64_t q = m.rp[i]; q < m.rp[i + 1]; ++q) {
                        all.col.push_back((int32_t)(m.col[q] + r0));
                        all.re.push_back(m.re[q]);
                        all.im.push_back(m.im[q]);
                    }
                    all.diag[r] = m.diag[i];
                }
                all.rp[r + 1] = (int64_t)all.col.size();
                row_scale[r] = 2.0 / I.rescale;
            }
        }
    } catch (const std::bad_alloc &) {
        return TBPM_ERR_OOM;
    }
    tbpm_ctx *ctx = new (std::nothrow) tbpm_ctx;
    if (!ctx) return TBPM_ERR_OOM;
    ctx->precision = o.precision;
    ctx->path = TBPM_PATH_SELL;
    ctx->flags = o.flags;
    ctx->tol = o.bessel_tol;
    ctx->n = rows[ninst];
    ctx->n_pad = rows[ninst];
    ctx->rescale = rmax;
    ctx->gershgorin = gmax;
    ctx->ninst = ninst;
    ctx->inst_row = rows;
    for (int g = 0; g < ninst; ++g) {
        ctx->inst_n.push_back(inst[g].n);
        ctx->inst_rescale.push_back(inst[g].rescale);
    }
    if ((rc = finish_create(ctx, o)) || (rc = setup_sell(ctx, all, &row_scale))) {
        tbpm_destroy(ctx);
        return rc;
    }
    // slice -> instance map and the slice range of each instance
    const int64_t nsl = ctx->n_pad / kSlice;
    std::vector<int32_t> sinst(nsl);
    std::vector<int64_t> seg(ninst + 1);
    for (int g = 0; g <= ninst; ++g) seg[g] = rows[g] / kSlice;
    for (int g = 0; g < ninst; ++g)
        for (int64_t q = seg[g]; q < seg[g + 1]; ++q) sinst[q] = g;
    if ((rc = upload(ctx, (void **)&ctx->d_slice_inst, sinst)) || (rc = upload(ctx, (void **)&ctx->d_seg_off, seg)) ||
        (rc = apply_shape(ctx, o)) || ((o.flags & TBPM_F_AUTOTUNE) && (rc = autotune(ctx)))) {
        tbpm_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return TBPM_OK;
}

int tbpm_batch_dos_corr(tbpm_ctx *ctx, const double *psi0, const double *dt, int n_steps, double *corr)
{
    if (!ctx || !psi0 || !dt || !corr || n_steps < 0) return TBPM_ERR_ARG;
    if (ctx->ninst < 1) return TBPM_ERR_UNSUPPORTED;
    const int G = ctx->ninst;
    for (int g = 0; g < G; ++g) {
        if (!(dt[g] != 0.0) || !std::isfinite(dt[g])) return TBPM_ERR_ARG;
        if (!(std::fabs(dt[g] * ctx->inst_rescale[g]) <= 40.0)) return TBPM_ERR_ARG;
    }
    CU(cudaSetDevice(ctx->device));
    bool in_dev, out_dev;
    int rc;
    if ((rc = classify(ctx, psi0, &in_dev)) || (rc = classify(ctx, corr, &out_dev))) return rc;
    int64_t launches = 0;
    // per-instance coefficients (read back K once per set of time steps)
    if (ctx->dt_cached.size() != (size_t)G || !std::equal(ctx->dt_cached.begin(), ctx->dt_cached.end(), dt)) {
        for (int g = 0; g < G; ++g)
            CU(launch_bessel(dt[g] * ctx->inst_rescale[g], ctx->tol, ctx->d_coef + (int64_t)g * kMaxTerms,
                             ctx->d_K + g, ctx->stream));
        CU(launch_mask_coef(ctx->d_coef, ctx->d_K, G, ctx->stream));
        std::vector<int> K(G);
        CU(cudaMemcpyAsync(K.data(), ctx->d_K, sizeof(int) * G, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        int Kmax = 3;
        for (int g = 0; g < G; ++g) {
            if (K[g] < 1) return TBPM_ERR_ARG;
            Kmax = std::max(Kmax, K[g]);
        }
        ctx->K_batch = Kmax;
        ctx->dt_cached.assign(dt, dt + G);
        launches += G + 1;
    }
    const int Ke = ctx->K_batch;
    const int64_t ld = (int64_t)n_steps + 1;
    int64_t nmax = 0;
    for (int g = 0; g < G; ++g) nmax = std::max(nmax, ctx->inst_n[g]);
    if ((rc = ensure_work(ctx, 1, (size_t)G * ld, in_dev ? 0 : (size_t)2 * nmax))) return rc;
    const size_t vb = vec_bytes(ctx->precision);
    int64_t src_off = 0;
    for (int g = 0; g < G; ++g) {
        const double *src;
        if ((rc = stage_input(ctx, psi0 + 2 * src_off, in_dev, (size_t)2 * ctx->inst_n[g], &src))) return rc;
        char *d0 = static_cast<char *>(ctx->d_psi0) + vb * ctx->inst_row[g];
        char *d1 = static_cast<char *>(ctx->d_psi) + vb * ctx->inst_row[g];
        CU(launch_load_states(ctx->precision, src, ctx->inst_n[g], ctx->inst_row[g + 1] - ctx->inst_row[g], 1, 0,
                              1, d0, d1, ctx->stream));
        if (!in_dev) CU(cudaStreamSynchronize(ctx->stream));        // staging reuse
        src_off += ctx->inst_n[g];
        ++launches;
    }
    const int64_t nsl = ctx->n_pad / kSlice;
    CU(launch_dot(ctx->precision, ctx->d_psi0, ctx->d_psi0, nsl, ctx->d_partials, ctx->nblk, true, ctx->stream));
    CU(launch_reduce_seg(ctx->d_partials, 1, 1, nsl, ctx->d_seg_off, G, nullptr, 0, ctx->d_out, ld, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
    launches += 2;
    if (ctx->flags & TBPM_F_RENORM) {
        CU(launch_fill(ctx->d_scale, G, 1.0, ctx->stream));
        ++launches;
    }
    int done = 0;
    while (done < n_steps) {
        const int len = std::min(kChunk, n_steps - done);
        if ((rc = run_chunk(ctx, 3, Ke, len, &launches, ld))) return rc;
        done += len;
    }
    CU(cudaMemcpyAsync(corr, ctx->d_out, sizeof(double2) * ld * G,
                       out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (!out_dev || !in_dev) CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGetLastError());
    ctx->last_K = Ke;
    ctx->last_passes = (int64_t)n_steps * (Ke - 1);
    ctx->last_launches = launches;
    return TBPM_OK;
}

int tbpm_quasi_eigenstates(tbpm_ctx *ctx, const double *psi0, double dt, int n_steps, const double *energies,
                           int n_e, double *qe)
{
    if (!ctx || !psi0 || !energies || !qe || n_steps < 1 || n_e < 1 || n_e > 4096) return TBPM_ERR_ARG;
    if (ctx->ninst > 0) return TBPM_ERR_UNSUPPORTED;
    if (!(dt > 0.0) || !std::isfinite(dt) || !(dt * ctx->rescale <= 40.0)) return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, e_dev, q_dev;
    int rc;
    if ((rc = classify(ctx, psi0, &in_dev)) || (rc = classify(ctx, energies, &e_dev)) || (rc = classify(ctx, qe, &q_dev)))
        return rc;
    const int64_t n = ctx->n, n_pad = ctx->n_pad;
    if ((rc = ensure_work(ctx, 1, (size_t)n_steps + 1, in_dev ? 0 : (size_t)2 * n))) return rc;
    const size_t qcap = (size_t)n_e * n_pad;
    if (qcap > ctx->qe_cap) {
        destroy_graphs(ctx);
        cudaFree(ctx->d_qe);
        ctx->d_qe = nullptr;
        ctx->qe_cap = 0;
        CU(cudaMalloc(&ctx->d_qe, qcap * sizeof(double2)));
        ctx->qe_cap = qcap;
    }
    if ((size_t)n_e > ctx->qe_e_cap) {
        destroy_graphs(ctx);
        cudaFree(ctx->d_qe_e);
        ctx->d_qe_e = nullptr;
        ctx->qe_e_cap = 0;
        CU(cudaMalloc(&ctx->d_qe_e, sizeof(double) * n_e));
        ctx->qe_e_cap = n_e;
    }
    CU(cudaMemcpyAsync(ctx->d_qe_e, energies, sizeof(double) * n_e,
                       e_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    const double *src;
    if ((rc = stage_input(ctx, psi0, in_dev, (size_t)2 * n, &src))) return rc;
    CU(launch_load_states(ctx->precision, src, n, n_pad, 1, 0, 1, ctx->d_psi0, ctx->d_psi, ctx->stream));
    const double pre = dt / (2.0 * 3.141592653589793238462643383279502884);
    CU(launch_qe_init(ctx->precision, ctx->d_psi0, ctx->d_qe, n_e, n_pad, pre, ctx->stream));
    // the quasi-eigenstate graphs bake dt and the number of energies into their
    // accumulation launches (the energies themselves are read from d_qe_e): they
    // are kept across calls with the same two and rebuilt otherwise
    if (dt != ctx->qe_graph_dt || n_e != ctx->qe_graph_ne) {
        for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
            if (std::get<0>(it->first) == 5) {
                cudaGraphExecDestroy(it->second);
                it = ctx->graphs.erase(it);
            } else {
                ++it;
            }
        }
        ctx->qe_graph_dt = dt;
        ctx->qe_graph_ne = n_e;
    }
    int64_t launches = 2, passes = 0;
    for (int dir = 0; dir < 2; ++dir) {
        const double h = dir == 0 ? dt : -dt;
        int K;
        if ((rc = ensure_coeffs(ctx, h * ctx->rescale, &K))) return rc;
        const int Ke = std::max(K, 3);
        passes += (int64_t)n_steps * (Ke - 1);
        CU(cudaMemcpyAsync(ctx->d_psi, ctx->d_psi0, vec_bytes(ctx->precision) * n_pad, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CU(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), ctx->stream));
        if (ctx->flags & TBPM_F_RENORM) {
            CU(launch_renorm(nullptr, 0, 1, ctx->d_scale, ctx->stream));
            ++launches;
        }
        ctx->qe_h = h;
        ctx->qe_N = n_steps;
        ctx->qe_ne = n_e;
        int done = 0;
        while (done < n_steps) {
            const int len = std::min(kChunk, n_steps - done);
            if ((rc = run_chunk(ctx, 5, Ke, len, &launches, 2 * (int64_t)n_steps + dir))) return rc;
            done += len;
        }
    }
    CU(cudaMemcpy2DAsync(qe, sizeof(double2) * n, ctx->d_qe, sizeof(double2) * n_pad, sizeof(double2) * n, n_e,
                         q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGetLastError());
    ctx->last_passes = passes;
    ctx->last_launches = launches;
    return TBPM_OK;
}

int tbpm_haydock(tbpm_ctx *ctx, const double *psi0, int M, double *a, double *b)
{
    if (!ctx || !psi0 || !a || !b || M < 1) return TBPM_ERR_ARG;
    if (ctx->ninst > 0) return TBPM_ERR_UNSUPPORTED;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, a_dev, b_dev;
    int rc;
    if ((rc = classify(ctx, psi0, &in_dev)) || (rc = classify(ctx, a, &a_dev)) || (rc = classify(ctx, b, &b_dev)))
        return rc;
    const int64_t n = ctx->n;
    if ((rc = ensure_work(ctx, 1, (size_t)M, in_dev ? 0 : (size_t)2 * n))) return rc;
    const size_t vb = vec_bytes(ctx->precision) * (size_t)ctx->n_pad;
    const double *src;
    if ((rc = stage_input(ctx, psi0, in_dev, (size_t)2 * n, &src))) return rc;
    CU(launch_load_states(ctx->precision, src, n, ctx->n_pad, 1, 0, 1, ctx->d_psi0, ctx->d_psi, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_b0, 0, vb, ctx->stream));                 // u_{-1} = 0
    const int64_t W = (int64_t)ctx->nblk * (kBlockB1 / 32);
    CU(launch_dot(ctx->precision, ctx->d_psi, ctx->d_psi, ctx->n_pad / kSlice, ctx->d_partials, ctx->nblk, false,
                  ctx->stream));
    CU(launch_hay_init(ctx->d_partials, W, ctx->d_misc, 0.5 * ctx->rescale, ctx->d_counter, ctx->stream));
    if (ctx->hay_grid[0] == 0) hay_grids(variant(ctx, 1), ctx->num_sms, &ctx->hay_grid[0], &ctx->hay_grid[1]);
    int64_t launches = 3;
    int done = 0;
    while (done < M) {
        const int len = std::min(kChunk, M - done);
        if ((rc = run_chunk(ctx, 4, 0, len, &launches, M))) return rc;
        done += len;
    }
    const double *dout = reinterpret_cast<const double *>(ctx->d_out);
    CU(cudaMemcpyAsync(a, dout, sizeof(double) * M, a_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaMemcpyAsync(b, dout + M, sizeof(double) * M, b_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (!in_dev || !a_dev || !b_dev) CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaGetLastError());
    ctx->last_passes = 2 * (int64_t)M;
    ctx->last_launches = launches;
    return TBPM_OK;
}

int tbpm_haydock_ldos(tbpm_ctx *ctx, const double *a, const double *b, int M, const double *energies, int n_e,
                      double eta, double *ldos)
{
    if (!ctx || !a || !b || !energies || !ldos || M < 1 || n_e < 1) return TBPM_ERR_ARG;
    if (!(eta > 0.0) || !std::isfinite(eta)) return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool a_dev, b_dev, e_dev, l_dev;
    int rc;
    if ((rc = classify(ctx, a, &a_dev)) || (rc = classify(ctx, b, &b_dev)) || (rc = classify(ctx, energies, &e_dev)) ||
        (rc = classify(ctx, ldos, &l_dev)))
        return rc;
    if ((rc = ensure_work(ctx, 1, 0, 2 * (size_t)M + 2 * (size_t)n_e))) return rc;
    double *st = ctx->d_stage;
    const double *da = a, *db = b, *de = energies;
    if (!a_dev) { CU(cudaMemcpyAsync(st, a, sizeof(double) * M, cudaMemcpyHostToDevice, ctx->stream)); da = st; }
    if (!b_dev) { CU(cudaMemcpyAsync(st + M, b, sizeof(double) * M, cudaMemcpyHostToDevice, ctx->stream)); db = st + M; }
    if (!e_dev) {
        CU(cudaMemcpyAsync(st + 2 * M, energies, sizeof(double) * n_e, cudaMemcpyHostToDevice, ctx->stream));
        de = st + 2 * M;
    }
    double *dl = l_dev ? ldos : st + 2 * M + n_e;
    CU(launch_hay_ldos(da, db, M, de, n_e, eta, dl, ctx->stream));
    if (!l_dev) CU(cudaMemcpyAsync(ldos, dl, sizeof(double) * n_e, cudaMemcpyDeviceToHost, ctx->stream));
    if (!a_dev || !b_dev || !e_dev || !l_dev) CU(cudaStreamSynchronize(ctx->stream));
    ctx->last_launches = 1;
    return TBPM_OK;
}

int tbpm_set_current(tbpm_ctx *ctx, const int64_t *row_ptr, const int32_t *col, const double *jx,
                     const double *jy)
{
    if (!ctx || !row_ptr) return TBPM_ERR_ARG;
    if (ctx->ninst > 0 || ctx->precision != TBPM_FP64) return TBPM_ERR_UNSUPPORTED;
    const int64_t n = ctx->n;
    if (row_ptr[0] != 0) return TBPM_ERR_CSR;
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return TBPM_ERR_CSR;
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && (!col || !jx || !jy)) return TBPM_ERR_ARG;
    for (int64_t q = 0; q < nnz; ++q)
        if (col[q] < 0 || (int64_t)col[q] >= n) return TBPM_ERR_CSR;
    for (int64_t q = 0; q < 2 * nnz; ++q)
        if (!std::isfinite(jx[q]) || !std::isfinite(jy[q])) return TBPM_ERR_ARG;
    // rows sorted by column, duplicates summed
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> cc;
    std::vector<double2> vx, vy;
    cc.reserve(nnz); vx.reserve(nnz); vy.reserve(nnz);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int64_t i = 0; i < n; ++i) {
        row.clear();
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) row.emplace_back(col[q], q);
        std::sort(row.begin(), row.end());
        size_t a = 0;
        while (a < row.size()) {
            const int32_t c = row[a].first;
            double2 x = make_double2(0.0, 0.0), y = make_double2(0.0, 0.0);
            for (; a < row.size() && row[a].first == c; ++a) {
                const int64_t q = row[a].second;
                x.x += jx[2 * q]; x.y += jx[2 * q + 1];
                y.x += jy[2 * q]; y.y += jy[2 * q + 1];
            }
            cc.push_back(c); vx.push_back(x); vy.push_back(y);
        }
        rp[i + 1] = (int64_t)cc.size();
    }
    if (!(ctx->flags & TBPM_F_NO_HERMITIAN_CHECK)) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
                const int32_t j = cc[q];
                const int32_t *b = cc.data() + rp[j], *e = cc.data() + rp[j + 1];
                const int32_t *f = std::lower_bound(b, e, (int32_t)i);
                double2 tx = make_double2(0.0, 0.0), ty = make_double2(0.0, 0.0);
                if (f != e && *f == (int32_t)i) {
                    const int64_t r = f - cc.data();
                    tx = make_double2(vx[r].x, -vx[r].y);
                    ty = make_double2(vy[r].x, -vy[r].y);
                }
                const double sx = std::hypot(vx[q].x, vx[q].y) + std::hypot(tx.x, tx.y);
                const double sy = std::hypot(vy[q].x, vy[q].y) + std::hypot(ty.x, ty.y);
                if (std::hypot(vx[q].x - tx.x, vx[q].y - tx.y) > 1e-13 * sx ||
                    std::hypot(vy[q].x - ty.x, vy[q].y - ty.y) > 1e-13 * sy)
                    return TBPM_ERR_NOT_HERMITIAN;
            }
    }
    // SELL-32, padding entries: own row, value 0
    const int64_t nsl = ctx->n_pad / kSlice;
    std::vector<int64_t> off(nsl + 1, 0);
    for (int64_t sl = 0; sl < nsl; ++sl) {
        int64_t w = 0;
        for (int l = 0; l < kSlice; ++l) {
            const int64_t r = sl * kSlice + l;
            if (r < n) w = std::max(w, rp[r + 1] - rp[r]);
        }
        off[sl + 1] = off[sl] + w * kSlice;
    }
    const int64_t nent = off[nsl];
    std::vector<int32_t> scol(nent);
    std::vector<double2> sx(nent, make_double2(0.0, 0.0)), sy(nent, make_double2(0.0, 0.0));
    for (int64_t sl = 0; sl < nsl; ++sl) {
        const int64_t w = (off[sl + 1] - off[sl]) / kSlice;
        for (int l = 0; l < kSlice; ++l) {
            const int64_t r = sl * kSlice + l;
            const int64_t len = r < n ? rp[r + 1] - rp[r] : 0;
            for (int64_t q = 0; q < w; ++q) {
                const int64_t e = off[sl] + q * kSlice + l;
                if (q < len) {
                    scol[e] = cc[rp[r] + q];
                    sx[e] = vx[rp[r] + q];
                    sy[e] = vy[rp[r] + q];
                } else {
                    scol[e] = (int32_t)r;
                }
            }
        }
    }
    CU(cudaSetDevice(ctx->device));
    if (ctx->stream) CU(cudaStreamSynchronize(ctx->stream));
    free_current(ctx);
    int rc;
    void *d_off = nullptr, *d_col = nullptr, *d_x = nullptr, *d_y = nullptr;
    if ((rc = upload(ctx, &d_off, off)) || (rc = upload(ctx, &d_col, scol)) || (rc = upload(ctx, &d_x, sx)) ||
        (rc = upload(ctx, &d_y, sy))) {
        cudaFree(d_off); cudaFree(d_col); cudaFree(d_x); cudaFree(d_y);
        return rc;
    }
    ctx->cur.nslices = nsl;
    ctx->cur.slice_off = static_cast<int64_t *>(d_off);
    ctx->cur.cols = static_cast<int32_t *>(d_col);
    ctx->cur.jx = static_cast<double2 *>(d_x);
    ctx->cur.jy = static_cast<double2 *>(d_y);
    ctx->cur.imag = true;
    for (int64_t e = 0; e < nent && ctx->cur.imag; ++e) ctx->cur.imag = sx[e].x == 0.0 && sy[e].x == 0.0;
    ctx->cur_nnz = (int64_t)cc.size();
    destroy_graphs(ctx);
    return TBPM_OK;
}

int tbpm_ac_corr(tbpm_ctx *ctx, const double *psi0, double beta, double mu, double dt, int n_steps,
                 double *corr)
{
    if (!ctx || !psi0 || !corr || n_steps < 0) return TBPM_ERR_ARG;
    if (ctx->ninst > 0 || ctx->precision != TBPM_FP64) return TBPM_ERR_UNSUPPORTED;
    if (!ctx->cur.slice_off) {
        ctx->last_error = "tbpm_ac_corr: no current operators (tbpm_set_current)";
        return TBPM_ERR_ARG;
    }
    if (!(beta > 0.0) || !std::isfinite(beta) || !std::isfinite(mu)) return TBPM_ERR_ARG;
    if (!(dt != 0.0) || !std::isfinite(dt)) return TBPM_ERR_ARG;
    const double x = dt * ctx->rescale;
    if (!(std::fabs(x) <= 40.0)) return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool in_dev, out_dev;
    int rc;
    if ((rc = classify(ctx, psi0, &in_dev)) || (rc = classify(ctx, corr, &out_dev))) return rc;
    const int64_t n = ctx->n, np1 = (int64_t)n_steps + 1;
    int K;
    if ((rc = ensure_coeffs(ctx, x, &K))) return rc;
    const int Ke = std::max(K, 3);
    if ((rc = ensure_work(ctx, 1, (size_t)4 * np1,
                          (in_dev && out_dev) ? 0 : (size_t)std::max<int64_t>(2 * n, 8 * np1))))
        return rc;
    if ((rc = ensure_ac(ctx))) return rc;
    cudaStream_t s = ctx->stream;
    int64_t launches = 0;
    if (ctx->fermi_K == 0 || beta != ctx->fermi_beta || mu != ctx->fermi_mu) {
        ctx->fermi_K = 0;
        CU(launch_fermi_coeffs(beta, mu, ctx->rescale, 1e-12, kFermiCap, ctx->d_fnodes, ctx->d_fc, ctx->d_gc,
                               ctx->d_kmax, s));
        int kf = 0;
        CU(cudaMemcpyAsync(&kf, ctx->d_kmax, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        launches += 2;
        if (kf >= kFermiCap) {
            ctx->last_error = "tbpm_ac_corr: the Fermi series needs more than TBPM_FERMI_MAX_TERMS terms";
            return TBPM_ERR_ARG;
        }
        kf = std::max(kf, 1);
        // zero tail: the series below runs max(kf + 1, 4) terms with a zero top coefficient
        CU(cudaMemsetAsync(ctx->d_fc + kf, 0, sizeof(double2) * (kFermiCap - kf), s));
        CU(cudaMemsetAsync(ctx->d_gc + kf, 0, sizeof(double2) * (kFermiCap - kf), s));
        ctx->fermi_K = kf;
        ctx->fermi_beta = beta;
        ctx->fermi_mu = mu;
    }
    const int Kp = std::max(ctx->fermi_K + 1, 4);
    void *v[3];
    ac_vectors(ctx, v);
    const double *src;
    if ((rc = stage_input(ctx, psi0, in_dev, (size_t)2 * n, &src))) return rc;
    CU(launch_load_states(ctx->precision, src, n, ctx->n_pad, 1, 0, 1, ctx->d_psi0, ctx->d_psi, s));
    ++launches;
    // phi2 = f(H~) phi;  phi1_b = [1 - f(H~)] J_b phi
    if ((rc = enqueue_series(ctx, ctx->d_fc, Kp, false, ctx->d_psi0, v[0], kChunk, s, &launches))) return rc;
    for (int b = 0; b < 2; ++b) {
        CU(launch_jmul(ctx->cur, b == 0 ? ctx->cur.jx : ctx->cur.jy, ctx->d_psi0, ctx->d_psi, 2 * ctx->nblk, s));
        ++launches;
        if ((rc = enqueue_series(ctx, ctx->d_gc, Kp, false, ctx->d_psi, v[1 + b], kChunk, s, &launches)))
            return rc;
    }
    // C(t_0), then the time steps
    const int64_t W = (int64_t)ctx->nblk * (kBlockB1 / 32);
    CU(launch_jdot(ctx->cur, v[0], v[1], v[2], ctx->d_acpart, 0, ctx->nblk, s));
    CU(launch_reduce_seg(ctx->d_acpart, 1, 4, W, nullptr, 1, nullptr, 0, ctx->d_out, 0, s));
    CU(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), s));
    launches += 2;
    int done = 0;
    while (done < n_steps) {
        const int len = std::min(kChunk, n_steps - done);
        if ((rc = run_chunk(ctx, 6, Ke, len, &launches))) return rc;
        done += len;
    }
    double2 *dst = out_dev ? reinterpret_cast<double2 *>(corr) : reinterpret_cast<double2 *>(ctx->d_stage);
    CU(launch_ac_transpose(ctx->d_out, np1, dst, s));
    ++launches;
    if (!out_dev) CU(cudaMemcpyAsync(corr, dst, sizeof(double2) * 4 * np1, cudaMemcpyDeviceToHost, s));
    if (!out_dev || !in_dev) CU(cudaStreamSynchronize(s));
    CU(cudaGetLastError());
    ctx->last_K = Ke;
    ctx->last_passes = (int64_t)3 * n_steps * (Ke - 1) + 3 * (int64_t)(Kp - 1) + 2 + (int64_t)n_steps + 1;
    ctx->last_launches = launches;
    return TBPM_OK;
}

int tbpm_ac_cond(tbpm_ctx *ctx, const double *corr, int n_steps, double dt, double beta, double area,
                 const double *omegas, int n_w, double *sigma)
{
    if (!ctx || !corr || !omegas || !sigma || n_steps < 1 || n_w < 1) return TBPM_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt) || !(beta > 0.0) || !std::isfinite(beta) || !(area > 0.0) ||
        !std::isfinite(area) || n_steps > (1 << 28) || n_w > (1 << 24))
        return TBPM_ERR_ARG;
    CU(cudaSetDevice(ctx->device));
    bool c_dev, w_dev, s_dev;
    int rc;
    if ((rc = classify(ctx, corr, &c_dev)) || (rc = classify(ctx, omegas, &w_dev)) ||
        (rc = classify(ctx, sigma, &s_dev)))
        return rc;
    const size_t nc = 8 * ((size_t)n_steps + 1);
    if ((rc = ensure_work(ctx, 1, 0, nc + (size_t)n_w + 4 * (size_t)n_w))) return rc;
    cudaStream_t s = ctx->stream;
    const double2 *c = reinterpret_cast<const double2 *>(corr);
    if (!c_dev) {
        CU(cudaMemcpyAsync(ctx->d_stage, corr, nc * sizeof(double), cudaMemcpyHostToDevice, s));
        c = reinterpret_cast<const double2 *>(ctx->d_stage);
    }
    const double *w = omegas;
    if (!w_dev) {
        CU(cudaMemcpyAsync(ctx->d_stage + nc, omegas, n_w * sizeof(double), cudaMemcpyHostToDevice, s));
        w = ctx->d_stage + nc;
    }
    double *dsg = s_dev ? sigma : ctx->d_stage + nc + n_w;
    CU(launch_ac_cond(c, n_steps, dt, beta, area, w, n_w, dsg, s));
    if (!s_dev) CU(cudaMemcpyAsync(sigma, dsg, 4 * (size_t)n_w * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!c_dev || !w_dev || !s_dev) CU(cudaStreamSynchronize(s));
    ctx->last_launches = 1;
    return TBPM_OK;
}

const char *tbpm_last_error(const tbpm_ctx *ctx)
{
    return ctx ? ctx->last_error.c_str() : "";
}

int tbpm_get_info(const tbpm_ctx *ctx, tbpm_info *info)
{
    if (!ctx || !info) return TBPM_ERR_ARG;
    info->n = ctx->n;
    info->nnz = ctx->op == OP_SELL ? ctx->nnz : 0;
    info->path = ctx->path;
    info->precision = ctx->precision;
    info->real_values = ctx->op == OP_SELL ? (int)ctx->sell.real_values : 1;
    info->num_terms = ctx->last_K;
    info->passes = ctx->last_passes;
    info->kernel_launches = ctx->last_launches;
    info->gershgorin = ctx->gershgorin;
    info->rescale = ctx->rescale;
    info->grid_blocks = ctx->nblk;
    info->tuned = ctx->tuned ? 1 : 0;
    info->fermi_terms = ctx->fermi_K;
    info->block_threads = ctx->sw_block;
    info->slices_per_warp = ctx->sw_spw;
    info->tune_candidates = ctx->tune_candidates;
    info->tune_default_us = ctx->tune_default_us;
    info->tune_best_us = ctx->tune_best_us;
    info->packed = ctx->op == OP_SELL ? ctx->sell.packed : 0;
    return TBPM_OK;
}

}  // extern "C"
