// Internal declarations of libtbpm: device layouts, kernel parameter blocks,
// and the launch entry points each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "tbpm.h"

namespace tbpm {

constexpr int kSlice = 32;          // SELL slice height = warp width
constexpr int kBlock = 256;         // threads per block of the 16-state and helper kernels
constexpr int kBlockB1 = 512;       // threads per block of the single-state sweeps and dots
constexpr int kMaxTerms = 128;      // Chebyshev coefficients generated on device
constexpr int kChunk = 16;          // time steps (or KPM passes) per captured graph
constexpr int kMaxBlockStates = 16; // states advanced together (FP32 batched)

// ------------------------------------------------- programmatic launches

// Programmatic dependent launch (sm_90 and later). A grid launched with the
// programmatic-serialisation attribute may be scheduled once every block of the
// previous kernel in the stream has started and released it;
// griddepcontrol.wait then blocks until that kernel has completed and its
// writes are visible. The kernels launched this way (the single-state sweeps,
// the KPM passes, the Haydock passes) call pdl_wait_release() before their
// first memory access, so the next grid's blocks take each SM as this grid's
// blocks leave it and start the moment it completes. For a plain launch both
// instructions do nothing.
__device__ __forceinline__ void pdl_wait_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kern<<<grid, block, 0, s>>>(args...), as a programmatic dependent launch if pdl.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), int grid, int block, bool pdl, cudaStream_t s, A... args)
{
    if (!pdl) {
        kern<<<grid, block, 0, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---------------------------------------------------------------- layouts

// Sliced ELLPACK with slice height 32 and no row sorting (the lattice order of
// the rows is kept for the locality of the gathers). Slice s covers rows
// [32 s, 32 s + 32); its entry (lane, j) sits at slice_off[s] + 32 j + lane.
// Padding entries point at their own row with value 0. The diagonal is kept
// apart as a real array (a Hermitian matrix has a real diagonal).
struct Sell {
    int64_t nslices = 0;
    int64_t nent = 0;             // stored off-diagonal slots incl. padding
    int64_t *slice_off = nullptr; // int64[nslices + 1]
    int32_t *cols = nullptr;      // int32[nent]
    void *vals = nullptr;         // real: R[nent]; complex: R2[nent]
    void *diag = nullptr;         // R[n_pad]
    bool real_values = true;
    int max_width = 0;
    // a packed form of the same entries (FP32, real values, when every
    // column offset fits 16 bits modulo n_pad and at most 256 values occur):
    // entry e is column (row + cdelta[e]) mod n_pad, value vtab[vidx[e]]; when
    // besides every slice has width 3 and at most 32 values occur, one word
    // per row instead (rowpack[r]: offset j in bits 16j..16j+15, value index j
    // in bits 48+5j..52+5j)
    int packed = 0;               // 0: plain only; 1: also per entry; 2: also per row
    int16_t *cdelta = nullptr;    // per entry (packed 1): int16[nent]
    uint8_t *vidx = nullptr;      // per entry (packed 1): uint8[nent]
    uint64_t *rowpack = nullptr;  // per row (packed 2, every slice of width 3): uint64[n_pad]
    void *vtab = nullptr;         // R[256]
};

// Periodic graphene / AB-bilayer stencil (matrix-free H v).
struct Stencil {
    int kind = TBPM_LATTICE_GRAPHENE;
    int64_t l1 = 0, l2 = 0;
    double t = 0, t_perp = 0;
    void *onsite = nullptr;       // R[n_pad] or nullptr
};

// Parameters of one Clenshaw sweep (see cheb_sweep.cu for the recurrence).
struct SweepParams {
    // operator
    int64_t n;                    // rows holding orbitals (rows >= n are padding)
    int64_t nslices;              // SELL slices, or stencil cells / 32 rounded up
    const int64_t *slice_off;
    const int32_t *cols;
    const void *vals;
    const void *diag;
    const int16_t *cdelta;        // the packed form (VM_PACKED kernels): column offsets,
    const uint8_t *vidx;          // value indices and the value table, offsets taken
    const void *vtab;             // modulo npad
    const uint64_t *rowpack;      // the per-row packed form (VM_ROWS kernels)
    int64_t npad;
    int64_t l1, l2;               // stencil geometry
    double t, t_perp;
    // vectors (all padded to n_pad rows, B states interleaved per row)
    const void *x;                // gathered operand
    const void *psi;              // current state psi(t_n)
    void *y;                      // output (may alias z, or psi in the final sweep)
    const void *z;                // b_{k+2} (subtracted), or nullptr
    // coefficients, on device: a = c[ia] - (ib >= 0 ? c[ib] : 0),
    // beta = bscale * (ic >= 0 ? c[ic] : 1)
    const double2 *coef;
    int ia, ib, ic;
    double bscale;
    // final sweep: <psi0|y> partials of slot `delta`: one per warp of the grid
    // for a single instance, one per slice for a batch (slice_inst != nullptr)
    const void *psi0;
    double2 *partials;
    int delta;
    int nblk;
    // optional renormalisation: psi is read as scale[j] * psi for state j
    // (nullptr: no scaling); the final sweep writes sum |y|^2 partials to
    // norm_partials[(delta * nblk + block) * B + j] (nullptr: none)
    const double *scale;
    double2 *norm_partials;
    // batch of instances: instance of each slice (nullptr: one instance);
    // coefficients of instance g at coef + g * kMaxTerms, its scale at scale[g]
    const int32_t *slice_inst;
};

// Current operators J_x, J_y on one SELL-32 pattern (complex values, any
// diagonal entries kept among the entries; padding: own row, value 0).
struct CurrentOp {
    int64_t nslices = 0;
    const int64_t *slice_off = nullptr;
    const int32_t *cols = nullptr;
    const double2 *jx = nullptr;
    const double2 *jy = nullptr;
    bool imag = false;            // every stored value of J_x and J_y is purely imaginary
};

constexpr int kFermiCap = TBPM_FERMI_MAX_TERMS;   // Fermi series terms; 2x as many quadrature nodes

// Temporally blocked sweeps on the lattice stencils, FP32, one state
// (cheb_tblock.cu): one launch runs sweeps [j0, j0 + S) of a time step's
// K - 1 Clenshaw sweeps (j = 0 first, j = K - 2 final) over lattice tiles.
// per = orbitals per cell: 2 (monolayer) or 4 (AB bilayer).
constexpr int kTbS = 6;            // sweeps per block
struct TbParams {
    int L1, L2;
    int tiles1, tiles2;
    float t, t_perp;               // pre-scaled hoppings 2 t / rescale, 2 t_perp / rescale
    const float *onsite;           // pre-scaled on-site energies, or nullptr
    const float2 *psi;             // psi(t_n)
    const float2 *bx, *bz;         // b_{k+1}, b_{k+2} at the block start (unused for j0 = 0)
    float2 *ox, *oz;               // the block's newest b and the one before (non-final blocks)
    float2 *psi_out;               // psi(t_{n+1}) (the block holding the final sweep)
    const float2 *psi0;
    double2 *partials;             // final block: <psi0|psi> partials, slot delta, one per block
    int delta;
    const double2 *coef;
    int K, j0, S;
};
int tb_tiles(int per, int64_t l1, int64_t l2, int *tiles1, int *tiles2);
// Opts the kernel in to its shared memory on the current device (before any capture).
cudaError_t tb_prepare(int per);
cudaError_t launch_tb_block(int per, const TbParams &p, int grid, cudaStream_t s);
// The blocked KPM passes (512 threads per block for both lattices): p.S passes
// from T_{m-1} (bz), T_m (bx), dot partials of slots delta .. delta + S - 1
// (one per block), the last two T's to ox (newest) and oz.
int tb_kpm_tiles(int per, int64_t l1, int64_t l2, int *tiles1, int *tiles2);
cudaError_t tb_kpm_prepare(int per);
cudaError_t launch_tb_kpm(int per, const TbParams &p, int grid, cudaStream_t s);

// KPM sweep: T_{m+1} = 2 H~ T_m - T_{m-1} with <T_m|T_m> and <T_{m+1}|T_m>.
struct KpmParams {
    int64_t n;
    int64_t nslices;
    const int64_t *slice_off;
    const int32_t *cols;
    const void *vals;
    const void *diag;
    const int16_t *cdelta;        // the packed forms, as in SweepParams
    const uint8_t *vidx;
    const void *vtab;
    const uint64_t *rowpack;
    int64_t npad;
    int64_t l1, l2;
    double t, t_perp;
    const void *x;                // T_m
    void *y;                      // in: T_{m-1}, out: T_{m+1} (nullptr z => first)
    double scale;                 // 2/rescale, or 1/rescale for T_1 = H~ T_0
    bool first;                   // y = scale * H T_0 (no subtraction)
    double2 *partials;            // [slot][2][nblk][B]
    int delta;
    int nblk;
};

enum OpKind { OP_SELL = 0, OP_STENCIL_MONO = 1, OP_STENCIL_BI = 2 };

// Signature of a device kernel variant chosen on the host.
struct SweepVariant {
    int precision;                // TBPM_FP64 | TBPM_FP32
    int op;                       // OpKind
    bool real_values;
    int packed = 0;               // the operator's packed form used (FP32 SELL, real values):
                                  // 0 none, 1 per entry (VM_PACKED), 2 per row (VM_ROWS)
    int states;                   // B: 1 or 16
    bool pdl;                     // B = 1 sweeps as programmatic dependent launches
    int block = kBlockB1;         // B = 1 sweeps: threads per block (32 .. 1024)
    int spw = 1;                  // B = 1 sweeps: 32-row slices a warp works on at once
};

// ---------------------------------------------------------------- context

}  // namespace tbpm

struct tbpm_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;   // private stream used for graph capture
    int precision = TBPM_FP64;
    int path = TBPM_PATH_SELL;
    unsigned flags = 0;
    double tol = 1e-12;
    int64_t n = 0, n_pad = 0;
    double rescale = 1.0, gershgorin = 0.0;
    int op = tbpm::OP_SELL;
    tbpm::Sell sell;
    tbpm::Stencil sten;
    int64_t nnz = 0;
    // sweep grids (fixed per context so the dot partials are deterministic)
    int nblk = 0;                    // single-state kernels
    int nblk_first = 0;              // the single-state first, second and final sweeps:
    int nblk_second = 0;             // one wave of each one's own occupancy at the
    int nblk_fin = 0;                // context's block shape
    int nblk_kpm = 0;                // the single-state KPM kernel
    int nblk16 = 0;                  // 16-state kernels
    int nblk16_fin = 0;              // the 16-state final sweep (its dot partials per block of it)
    // coefficients
    double2 *d_coef = nullptr;       // [kMaxTerms]
    int *d_K = nullptr;
    double x_cached = 0.0;
    int K_cached = -1;
    // work vectors, sized for `cap_states` interleaved states
    int cap_states = 0;
    void *d_psi = nullptr, *d_b0 = nullptr, *d_b1 = nullptr, *d_psi0 = nullptr;
    double2 *d_partials = nullptr;   // [(kChunk+1) * 2 * nblk * B]
    size_t partials_cap = 0;
    double2 *d_out = nullptr;        // per-call device results
    size_t out_cap = 0;
    double *d_stage = nullptr;       // FP64 staging for host inputs
    size_t stage_cap = 0;
    int *d_counter = nullptr;        // chunk base counter for graphs
    double *d_misc = nullptr;        // small scratch (norms, moment bases)
    int hay_grid[2] = {0, 0};        // Haydock product and update grids (set at first use)
    double *d_scale = nullptr;       // [16] 1/||psi_j|| for the renormalised FP32 path
    double2 *d_norm = nullptr;       // [kChunk][nblk][B] ||y||^2 partials (renormalisation)
    double2 *d_cpart = nullptr;      // [n_steps][nslices] partials of the cluster path
    size_t cpart_cap = 0;
    // batch of instances (tbpm_create_batch); ninst == 0 for a single instance
    int ninst = 0;
    std::vector<int64_t> inst_n;         // orbitals of each instance
    std::vector<int64_t> inst_row;       // first (padded) row of each instance, size ninst+1
    std::vector<double> inst_rescale;
    int32_t *d_slice_inst = nullptr;     // instance of each slice
    int64_t *d_seg_off = nullptr;        // first slice of each instance, size ninst+1
    std::vector<double> dt_cached;
    int K_batch = 0;                     // max over instances of max(K_g, 3)
    // quasi-eigenstates of the current call (enqueued after each final sweep)
    double2 *d_qe = nullptr;             // [n_e][n_pad]
    double *d_qe_e = nullptr;            // energies [n_e]
    size_t qe_cap = 0, qe_e_cap = 0;
    int qe_ne = 0, qe_N = 0;
    double qe_h = 0.0;
    double qe_graph_dt = 0.0;        // dt and energy count the kind-5 graphs were built for
    int qe_graph_ne = 0;
    // AC conductivity: current operators (tbpm_set_current) and their work buffers
    tbpm::CurrentOp cur;
    int64_t cur_nnz = 0;
    void *d_ac = nullptr;                // phi2, phi1_x, phi1_y: [3][n_pad] double2
    double *d_fnodes = nullptr;          // [2 kFermiCap] f at the quadrature nodes
    double2 *d_fc = nullptr, *d_gc = nullptr;   // [kFermiCap] series of f and of 1 - f
    int *d_kmax = nullptr;
    double2 *d_acpart = nullptr;         // [(kChunk + 1) * 4 * warps] jdot partials
    double fermi_beta = 0.0, fermi_mu = 0.0;
    // temporally blocked stencil path: b buffers P2, P3 and the second state buffer
    void *d_tb = nullptr;                // [3][n_pad] float2
    int tb_grid = 0;
    int tb_kpm_grid = 0;
    int fermi_K = 0;                     // 0: no coefficients cached
    // launch shape of the single-state sweeps (nblk blocks of sw_block threads,
    // sw_spw slices per warp iteration); dot partials: one per warp of that grid
    int sw_block = tbpm::kBlockB1;
    int sw_spw = 1;
    // autotuner: candidates timed, middle-sweep microseconds at the default and
    // at the chosen shape
    bool tuned = false;
    int tune_candidates = 0;
    double tune_default_us = 0.0, tune_best_us = 0.0;
    // cached executable graphs keyed by (kind, len, K, states)
    std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;
    // counters of the last call
    int last_K = 0;
    int64_t last_passes = 0;
    int64_t last_launches = 0;
    std::string last_error;
};

namespace tbpm {

// ------------------------------------------------------------ launchers
// Each returns cudaSuccess or the launch error.

// Chebyshev coefficients c_k, k < kMaxTerms, and K into d_K (bessel.cu).
cudaError_t launch_bessel(double x, double tol, double2 *d_coef, int *d_K, cudaStream_t s);

// One Clenshaw sweep of the given kind (cheb_sweep.cu) at the launch shape
// v.block x v.spw: every operator takes spw = 1 with blocks of up to 512
// threads; the stored matrix also takes spw = 1 with 1024 threads and spw = 2
// or 4 with up to 512 (cheb_sweep_s*.cu). Other shapes are refused
// (cudaErrorInvalidValue).
enum SweepKind { SW_FIRST = 0, SW_SECOND = 1, SW_MID = 2, SW_FINAL = 3 };
// for occupancy queries only: the final sweep that also sums |y|^2
constexpr int SW_FINAL_NORM = 4;
cudaError_t launch_sweep(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                         const SweepParams &p, int grid, cudaStream_t s);
// Resident blocks per SM of one sweep kind (a SweepKind) at v's shape (0:
// shape not built).
int sweep_shape_occupancy(const SweepVariant &v, bool multi, int kind = SW_MID);
bool sweep_shape_built(const SweepVariant &v);
// The stored-matrix shapes built in their own translation units.
cudaError_t launch_sell_s1_b1024(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                                 const SweepParams &p, int grid, cudaStream_t s);
cudaError_t launch_sell_s2_b512(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                                const SweepParams &p, int grid, cudaStream_t s);
cudaError_t launch_sell_s4_b512(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                                const SweepParams &p, int grid, cudaStream_t s);
int occupancy_sell_s1_b1024(const SweepVariant &v, bool multi, int kind);
int occupancy_sell_s2_b512(const SweepVariant &v, bool multi, int kind);
int occupancy_sell_s4_b512(const SweepVariant &v, bool multi, int kind);

// KPM sweep (cheb_sweep.cu).
cudaError_t launch_kpm(const SweepVariant &v, const KpmParams &p, int grid, cudaStream_t s);

// <a|b> = sum_i conj(a_i) b_i of one state over nslices 32-row slices: one
// partial per slice (per_slice, partials[s]) or one per warp of the grid
// (partials[w], w < grid * kBlockB1 / 32) (aux.cu).
cudaError_t launch_dot(int precision, const void *a, const void *b, int64_t nslices,
                       double2 *partials, int grid, bool per_slice, cudaStream_t s);

// Deterministic reduction of per-block partials laid out [nslot][nterm][nblk]:
//   out[(base + offset + d) * nterm + q] = sum_b partials[(d * nterm + q) * nblk + b]
// with base = *counter (0 when counter is nullptr) (aux.cu).
cudaError_t launch_reduce(const double2 *partials, int nslot, int nterm, int nblk,
                          const int *counter, int offset, double2 *out, cudaStream_t s);

// Segmented fixed-order reduction of per-slice partials [nslot][nterm][nslices]:
//   out[g * ld + (base + offset + d) * nterm + q] = sum over slices of segment g,
// segments [seg_off[g], seg_off[g+1]) (seg_off == nullptr: one segment) (aux.cu).
cudaError_t launch_reduce_seg(const double2 *partials, int nslot, int nterm, int64_t nslices,
                              const int64_t *seg_off, int nseg, const int *counter, int offset,
                              double2 *out, int64_t ld, cudaStream_t s);
// scale[g] = 1/sqrt(sum of norm[s].x over segment g) (aux.cu).
cudaError_t launch_renorm_seg(const double2 *norm, int64_t nslices, const int64_t *seg_off, int nseg,
                              double *scale, cudaStream_t s);
cudaError_t launch_fill(double *p, int n, double v, cudaStream_t s);
// Single-launch cluster path for small systems (cheb_cluster.cu): whether n_pad
// rows fit, and the launch of n_steps steps writing per-slice <psi0|psi>
// partials [n_steps][nslices] and, if psi_out is not null, the final state.
bool cluster_fits(int precision, int64_t n_pad, int *log_rows, int *ncta, size_t *smem);
cudaError_t launch_cluster_dos(int precision, bool real_values, const SweepParams &op, int max_width,
                               const void *psi0, const double2 *coef, int K, int n_steps,
                               double2 *partials, void *psi_out, cudaStream_t s);

// AC conductivity (ac.cu). Fermi series: fc[k] = a_k, gc[k] = delta_k0 - a_k
// for k < kcap (fj: 2 kcap doubles of scratch), *kmax = 1 + the last k with
// |a_k| >= tol.
cudaError_t launch_fermi_coeffs(double beta, double mu, double rescale, double tol, int kcap, double *fj,
                                double2 *fc, double2 *gc, int *kmax, cudaStream_t s);
// y = J x (one of j.jx, j.jy as vals), FP64 complex vectors of n_pad rows.
cudaError_t launch_jmul(const CurrentOp &j, const double2 *vals, const void *x, void *y, int grid, cudaStream_t s);
// <phi2|J_a|phi1_b> for ab = xx, xy, yx, yy: per-warp partials
// partials[(slot * 4 + q) * W + w], W = grid * kBlockB1 / 32.
cudaError_t launch_jdot(const CurrentOp &j, const void *phi2, const void *p1x, const void *p1y,
                        double2 *partials, int slot, int grid, cudaStream_t s);
// [n+1][4] -> [4][n+1]
cudaError_t launch_ac_transpose(const double2 *src, int64_t np1, double2 *dst, cudaStream_t s);
// Re sigma_q(w_j) for the 4 correlation rows of corr [4][n_steps+1]: sigma [4][n_w].
cudaError_t launch_ac_cond(const double2 *corr, int n_steps, double dt, double beta, double area,
                           const double *omegas, int n_w, double *sigma, cudaStream_t s);

// dst (FP64 complex [n]) = scale[col] * column col of an interleaved [n_pad][B]
// buffer (scale may be null) (aux.cu).
cudaError_t launch_store_column(int precision, const void *src, int64_t n, int B, int col,
                                const double *scale, double *dst, cudaStream_t s);

// Haydock recursion (haydock.cu). Device scalars sc[7] = {s_n, b_n, s_{n-1},
// a_n, rho_n, h s_n^2, a_n / h} (h = rescale/2; the stored vectors are scaled,
// v_n = s_n u_n); counter[0] = n, counter[1] the ticket of the last-block sums
// (zeroed by init).
// apply: wt = A u_n - rho_n u_{n-1} into p.y (= u_{n-1}), p.x = u_n;
//        a_n = h s_n^2 Re <u_n|wt> to sc[3] and a_out[n];
// update: u_{n+1} = wt - (a_n / h) u_n (in place); b_{n+1} = h s_n ||u_{n+1}||
//        to b_out[n], the next scalars, n + 1;
// both use part[grid] doubles of per-block sums (grids from hay_grids);
// init: s_0 from the ||psi0||^2 per-warp partials of launch_dot.
cudaError_t launch_hay_apply(const SweepVariant &v, const SweepParams &p, double *sc, double half_rescale,
                             double *part, unsigned *ticket, double *a_out, const int *counter, int grid,
                             cudaStream_t s);
cudaError_t launch_hay_update(const SweepVariant &v, const void *u, void *w, int64_t nslices, double *sc,
                              double half_rescale, double *part, unsigned *ticket, double *b_out, int *counter,
                              int grid, cudaStream_t s);
cudaError_t launch_hay_init(const double2 *partials, int64_t W, double *sc, double half_rescale, int *counter,
                            cudaStream_t s);
// Whole-wave grids of the product and update passes for this operator.
void hay_grids(const SweepVariant &v, int num_sms, int *apply_grid, int *update_grid);
cudaError_t launch_hay_ldos(const double *a, const double *b, int M, const double *energies, int n_e,
                            double eta, double *ldos, cudaStream_t s);

// Quasi-eigenstates (aux.cu): Q [n_e][n_pad] FP64 complex.
//   init: Q_e = pre psi;  accumulate after step m = *counter + delta + 1:
//   Q_e += pre w_m exp(i E_e m h) psi, w_m = (1 + cos(pi m / N)) / 2.
cudaError_t launch_qe_accumulate(int precision, const void *psi, double2 *Q, const double *energies, int n_e,
                                 int64_t n_pad, const int *counter, int delta, double h, int N, double pre,
                                 cudaStream_t s);
cudaError_t launch_qe_init(int precision, const void *psi, double2 *Q, int n_e, int64_t n_pad, double pre,
                           cudaStream_t s);

// coef[g * kMaxTerms + k] = 0 for k >= max(K[g], 3) (aux.cu).
cudaError_t launch_mask_coef(double2 *coef, const int *K, int ninst, cudaStream_t s);
cudaError_t launch_advance(int *counter, int by, cudaStream_t s);

// State layout conversion: src FP64 complex state-major [nstates][n] ->
// dst (precision) interleaved [n_pad][B] for states [j0, j0 + B) (aux.cu).
cudaError_t launch_load_states(int precision, const double *src, int64_t n, int64_t n_pad,
                               int nstates_src, int j0, int B, void *dst0, void *dst1,
                               cudaStream_t s);

// scale[j] = 1 / sqrt(sum_b norm_partials[b * B + j].x) for j < B, from one
// slot of final-sweep norm partials; with norm_partials == nullptr, scale[j] = 1
// (aux.cu).
cudaError_t launch_renorm(const double2 *norm_partials, int nblk, int B, double *scale,
                          cudaStream_t s);

// KPM moments from the reduced dot products (aux.cu).
cudaError_t launch_kpm_finalize(const double2 *dots, int M, int states, double2 *mu,
                                cudaStream_t s);

// DOS transforms (dos.cu).
cudaError_t launch_dos_hann(const double2 *corr, int n_steps, double dt, double *energies,
                            double *dos, cudaStream_t s);
cudaError_t launch_kpm_dos(const double2 *mu, int M, int n_e, double rescale, double *energies,
                           double *rho, cudaStream_t s);

// Block count of the sweep kernels at full occupancy (cheb_sweep.cu).
int sweep_grid(const SweepVariant &v, int num_sms);
int kpm_grid(const SweepVariant &v, int num_sms);

// Batched FP32 sweeps over 16 interleaved states (cheb_batch.cu).
cudaError_t launch_sweep_b16(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                             const SweepParams &p, int grid, cudaStream_t s);
// <a_j|b_j> partials [grid][16] over nslices 32-row slices.
cudaError_t launch_dot_b16(const void *a, const void *b, int64_t nslices, double2 *partials,
                           int grid, cudaStream_t s);
// out[j * ld + base + offset + d] = sum_b partials[(d * nblk + b) * 16 + j].
cudaError_t launch_reduce_b16(const double2 *partials, int nslot, int nblk, const int *counter,
                              int offset, double2 *out, int64_t ld, cudaStream_t s);
int sweep_grid_b16(int num_sms);
// The batched final sweep's grid: one wave of its own occupancy, at most grid.
int sweep_grid_b16_final(const SweepVariant &v, int num_sms, int grid);

// One FP64 state (device, [n] complex) into column `col` of an interleaved
// [n_pad][B] buffer of the given precision, in both dst0 and dst1 (aux.cu).
cudaError_t launch_load_column(int precision, const double *src, int64_t n, int B, int col,
                               void *dst0, void *dst1, cudaStream_t s);

}  // namespace tbpm
