/*
 * tbpm.h - C ABI of the GB300 (sm_103a) TBPM hot-path library (libtbpm.so).
 *
 * The tight-binding propagation method (TBPLaS 2.0, arXiv 2509.26309) evolves
 * random-phase states with the Chebyshev expansion of exp(-iHt) and records
 * the correlation C(t_n) = <psi0|psi(t_n)> (Sec. 2.2.1, the propagation
 * listings; Sec. 3.2.3, calc_corr_dos), and evaluates kernel-polynomial
 * moments mu_m = <psi0|T_m(H~)|psi0> (Sec. 1). The calls follow the order of
 * the paper's workflow (Sec. 2.2.2, Sec. 3.2.3): build the model, create the
 * solver with its rescale factor, run calc_corr_dos, analyse the DOS.
 *
 * Conventions shared by every call:
 *   - Complex numbers are two doubles (re, im), interleaved.
 *   - Energies in eV, times in hbar/eV (hbar = 1). H~ = H / rescale.
 *   - Pointers to state, correlation, moment and DOS arrays may be host
 *     memory (pageable or pinned) or device memory of the context's GPU; the
 *     library tells them apart with cudaPointerGetAttributes. With host
 *     buffers a call returns after its results are in host memory. With
 *     device buffers a call only enqueues work on the context's stream and
 *     returns; synchronise that stream before reading the results.
 *   - The caller owns every buffer it passes; the library copies what it
 *     needs and never keeps a caller pointer after a call returns.
 *   - Every function returns TBPM_OK (0) or a negative status; no exception
 *     crosses this boundary. Arguments are validated before any GPU work.
 *   - A context serves one host thread at a time; calls on one context are
 *     ordered on its stream.
 */
#ifndef TBPM_H
#define TBPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ statuses */
#define TBPM_OK                 0
#define TBPM_ERR_ARG           -1  /* NULL pointer, size or option out of range   */
#define TBPM_ERR_CSR           -2  /* row_ptr not monotone, column out of range    */
#define TBPM_ERR_NOT_HERMITIAN -3  /* H_ij != conj(H_ji), or complex diagonal      */
#define TBPM_ERR_RESCALE       -4  /* rescale below the Gershgorin bound of H     */
#define TBPM_ERR_OOM           -5  /* device or host allocation failed            */
#define TBPM_ERR_CUDA          -6  /* a CUDA runtime call failed                  */
#define TBPM_ERR_TIMEOUT       -7  /* a bounded device wait gave up (reserved: no
                                       kernel of this library waits on a flag; all
                                       device-side waits are block or cluster
                                       barriers and the hardware wait of a
                                       programmatic launch for the kernel before
                                       it in the stream)                         */
#define TBPM_ERR_NO_DEVICE     -8  /* no usable sm_103 GPU                         */
#define TBPM_ERR_UNSUPPORTED   -9  /* valid request this build does not serve     */

/* ------------------------------------------------------------- options */
#define TBPM_FP64 0                /* complex128 vectors, FP64 matrix values        */
#define TBPM_FP32 1                /* complex64 vectors and hoppings; Bessel
                                      coefficients, dots and moments stay FP64     */

#define TBPM_PATH_AUTO    0        /* stencil for lattice contexts, SELL otherwise */
#define TBPM_PATH_SELL    1        /* stored matrix, sliced ELLPACK (32-row slices) */
#define TBPM_PATH_STENCIL 2        /* matrix-free lattice stencil (lattice only)   */

#define TBPM_F_NO_HERMITIAN_CHECK 0x1u /* skip the O(nnz) H = H^dagger check        */
#define TBPM_F_FORCE_RESCALE      0x2u /* accept rescale below the Gershgorin bound */
#define TBPM_F_RENORM             0x4u /* tbpm_dos_corr renormalises psi to unit
                                          norm (FP64 norm) after each step; meant
                                          for FP32 contexts, whose rounding lets
                                          the norm drift                           */
#define TBPM_F_NO_CLUSTER         0x8u /* never use the single-launch cluster path
                                          that single-state tbpm_dos_corr takes for
                                          systems of up to 16 x 4096 (FP64) or
                                          16 x 8192 (FP32) padded rows; the result
                                          is the same either way                   */
#define TBPM_F_AUTOTUNE           0x10u /* at create, time whole time steps of
                                          this operator's sweeps over launch
                                          shapes (block width 128 .. 1024 threads,
                                          1, 2 or 4 32-row slices per warp
                                          iteration, grids of whole waves) and keep
                                          the fastest for the context's life
                                          (tbpm_info reports it)                  */
#define TBPM_F_NO_TBLOCK          0x20u /* FP32 monolayer stencil contexts run each
                                          time step's sweeps in temporally blocked
                                          launches (several sweeps per pass over a
                                          lattice tile in shared memory); this flag
                                          keeps one launch per sweep instead       */
#define TBPM_F_NO_PDL             0x40u /* launch the single-state sweeps in plain
                                          stream order. By default each one is a
                                          programmatic dependent launch: its blocks
                                          are scheduled while the previous sweep's
                                          last blocks run and wait in hardware for
                                          that sweep to complete before touching
                                          any vector; results are identical      */
#define TBPM_F_PLAIN_SELL         0x80u /* FP32 stored matrices with real values
                                          are by default also kept packed, when
                                          every entry's column lies within 32767
                                          rows of its own (modulo the padded row
                                          count) and at most 256 distinct values
                                          occur: a 16-bit column offset and an
                                          8-bit value index per entry (3 B instead
                                          of 8), which the single-state sweeps and
                                          KPM passes read; when moreover every
                                          32-row slice holds 3 entries per row and
                                          at most 32 values occur, one 64-bit word
                                          per row instead (three offsets and
                                          three 5-bit indices). This flag keeps
                                          only the plain form. Results are
                                          identical                              */

typedef struct tbpm_opts {
    int precision;       /* TBPM_FP64 | TBPM_FP32                                  */
    int path;            /* TBPM_PATH_*                                            */
    unsigned flags;      /* TBPM_F_* bit set                                       */
    int device;          /* CUDA device ordinal; -1 = the calling thread's current */
    void *stream;        /* cudaStream_t to order work on; NULL = the legacy
                            default stream of the device                           */
    double bessel_tol;   /* Chebyshev cutoff |J_k| < tol; 0 selects 1e-12          */
    int block_threads;   /* launch shape of the single-state sweeps: threads per
                            block, 128 | 256 | 512 | 1024; 0 selects 512 (128 for
                            a stored matrix packed per entry, 256 packed per row,
                            see TBPM_F_PLAIN_SELL). 1024 and
                            slices_per_warp > 1 are built for the stored-matrix
                            path only (TBPM_ERR_UNSUPPORTED on a stencil)         */
    int slices_per_warp; /* 32-row slices a warp works on at once: 1 | 2 | 4 (2
                            and 4 with at most 512 threads); 0 selects 1 (4 for
                            a stored matrix packed per entry, 2 per row). The
                            grid is whole waves of the shape's occupancy.
                            TBPM_F_AUTOTUNE replaces both with the tuned shape    */
} tbpm_opts;

/* Fills *opts with the defaults: FP64, PATH_AUTO, no flags, current device,
 * legacy default stream, tolerance 1e-12, the default launch shape (512
 * threads, one slice per warp). Returns TBPM_ERR_ARG if opts is NULL. */
int tbpm_default_opts(tbpm_opts *opts);

typedef struct tbpm_ctx tbpm_ctx;

/* --------------------------------------------------------------- create */

/* tbpm_create: the solver for a Hamiltonian given in CSR form (the sparse
 * H_csr of Sec. 2.2.1; the rescale of config.rescale, Sec. 3.2.3).
 *   n        number of orbitals, 1 <= n < 2^31
 *   row_ptr  HOST int64[n+1], row_ptr[0] = 0, non-decreasing
 *   col      HOST int32[nnz] column indices in [0, n), nnz = row_ptr[n]
 *   val      HOST double[2*nnz] complex values H_ij (re, im)
 *   rescale  > 0; H~ = H / rescale must have spectrum in [-1, 1]. Rejected
 *            with TBPM_ERR_RESCALE if below max_i sum_j |H_ij| unless
 *            TBPM_F_FORCE_RESCALE is set.
 *   opts     NULL for defaults.
 * Checks (host, before any GPU work): CSR structure (TBPM_ERR_CSR); real
 * diagonal and, unless TBPM_F_NO_HERMITIAN_CHECK, H_ij = conj(H_ji)
 * (TBPM_ERR_NOT_HERMITIAN). Repeated (i, j) entries are summed. The matrix is
 * converted to the device layout once; a matrix whose values are all real is
 * stored with real values. *out receives a context that owns all device
 * memory until tbpm_destroy. */
int tbpm_create(tbpm_ctx **out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const double *val, double rescale, const tbpm_opts *opts);

#define TBPM_LATTICE_GRAPHENE   0  /* monolayer: i = 2*(m1*L2 + m2) + s, s = A, B */
#define TBPM_LATTICE_AB_BILAYER 1  /* AB bilayer: i = 4*(m1*L2 + m2) + o,
                                      o = A1, B1, A2, B2; dimer pair A1-B2       */

typedef struct tbpm_lattice {
    int kind;              /* TBPM_LATTICE_*                                     */
    int64_t l1, l2;        /* periodic supercell of L1 x L2 primitive cells     */
    double t;              /* nearest-neighbour hopping (eV), -2.7 for graphene */
    double t_perp;         /* interlayer dimer hopping (eV), bilayer only       */
    const double *onsite;  /* HOST double[N] on-site energies, or NULL (zero)   */
} tbpm_lattice;

/* tbpm_create_lattice: the solver for a periodic graphene or AB-bilayer
 * supercell (the graphene primitive cell and hopping convention of Sec.
 * 3.2.1: <A,0|H|B,0> = t, <B,0|H|A,a1> = t, <B,0|H|A,a2> = t, completed by
 * H_ij(R) = H_ji(-R)^*). With TBPM_PATH_STENCIL (the AUTO choice) no matrix
 * is stored: the kernels compute H~ v from the lattice and the on-site array.
 * With TBPM_PATH_SELL the same matrix is assembled and stored. Requires
 * L1, L2 >= 3. Errors as tbpm_create. */
int tbpm_create_lattice(tbpm_ctx **out, const tbpm_lattice *lat, double rescale,
                        const tbpm_opts *opts);

/* One lattice of an uneven batch (tbpm_create_batch). */
typedef struct tbpm_instance {
    int64_t n;               /* orbitals of this instance, >= 1                */
    const int64_t *row_ptr;  /* HOST CSR of this instance, as tbpm_create     */
    const int32_t *col;
    const double *val;
    double rescale;          /* this instance's rescale factor, > 0          */
} tbpm_instance;

/* tbpm_create_batch: one solver for many independent Hamiltonians of uneven
 * size (the random-sample and model parallelism of Sec. 2.4.2, here in one
 * GPU launch sequence). The instances are stored as one block-diagonal
 * operator, each padded to a multiple of 32 rows and pre-scaled by its own
 * 2/rescale; every sweep covers all instances, and each instance keeps its
 * own coefficients, state and correlation.
 *   ninst  1 <= ninst <= 4096;  inst  HOST array of ninst descriptors.
 * Each instance is validated as in tbpm_create (same statuses); the sum of
 * the padded sizes must stay below 2^31. tbpm_dos_corr and kpm_moments are
 * not available on a batch context (TBPM_ERR_UNSUPPORTED); use
 * tbpm_batch_dos_corr. */
int tbpm_create_batch(tbpm_ctx **out, int ninst, const tbpm_instance *inst,
                      const tbpm_opts *opts);

/* tbpm_batch_dos_corr: tbpm_dos_corr for every instance of a batch context,
 * one state per instance, all advanced in the same sweeps.
 *   psi0  double[2 * sum_g n_g]: instance g's state at offset 2 * sum_{h<g} n_h
 *   dt    HOST double[ninst]: per-instance time step (x_g = dt_g * rescale_g,
 *         |x_g| <= 40); instances with fewer terms K_g run the largest K with
 *         their coefficients beyond K_g set to zero, which leaves their
 *         results those of K_g terms
 *   n_steps >= 0;  corr double[2 * ninst * (n_steps + 1)], instance-major.
 * psi0 and corr may be host or device memory, as for tbpm_dos_corr. */
int tbpm_batch_dos_corr(tbpm_ctx *ctx, const double *psi0, const double *dt, int n_steps,
                        double *corr);

/* Releases every resource of ctx (NULL is ignored). */
void tbpm_destroy(tbpm_ctx *ctx);

/* ------------------------------------------------------------ hot path */

/* tbpm_dos_corr: time evolution and DOS correlation (calc_corr_dos,
 * Sec. 3.2.3; the series loop of Sec. 2.2.1).
 * For each state j, psi(t_0) = psi0_j and, for n = 0..n_steps-1,
 *   psi(t_{n+1}) = sum_{k<K} c_k T_k(H~) psi(t_n),
 *   c_k = (2 - delta_k0) (-i)^k J_k(dt * rescale),
 * K = the first k > |dt*rescale| with |J_k| < bessel_tol; the coefficients
 * are generated on the GPU. Writes corr[j*(n_steps+1) + n] = <psi0_j|psi(t_n)>
 * for n = 0..n_steps (complex, so 2*(n_steps+1) doubles per state).
 *   psi0     double[2*n*nstates], state-major: state j at offset 2*n*j
 *   nstates  >= 1. FP32 contexts advance up to 16 states together as one
 *            block; FP64 contexts advance states one after another.
 *   dt       time step, dt != 0, |dt*rescale| <= 40 (K <= 64)
 *   n_steps  >= 0
 * The states are not normalised by the library. */
int tbpm_dos_corr(tbpm_ctx *ctx, const double *psi0, int nstates, double dt, int n_steps,
                  double *corr);

/* tbpm_propagate: the time-dependent wave function (WFT, one of the TBPM
 * capabilities benchmarked in Sec. 4.2.2): the same evolution as tbpm_dos_corr,
 * returning psi(t_{n_steps}) of every state.
 *   psi_out  double[2*n*nstates], state-major as psi0 (host or device)
 *   corr     as tbpm_dos_corr, or NULL when the correlation is not wanted
 * With TBPM_F_RENORM the returned state is normalised to 1. */
int tbpm_propagate(tbpm_ctx *ctx, const double *psi0, int nstates, double dt, int n_steps,
                   double *psi_out, double *corr);

/* kpm_moments: mu_m = <psi0_j|T_m(H~)|psi0_j>, m = 0..M-1 (the kernel
 * polynomial method named in Sec. 1), written as complex numbers to
 * mu[j*M + m]. The GPU uses the product identities
 *   mu_{2m} = 2<T_m|T_m> - mu_0,  mu_{2m+1} = 2<T_{m+1}|T_m> - mu_1
 * (T_m = T_m(H~) psi0), so about M/2 matrix products are made. The moments
 * of a Hermitian H are real: their imaginary parts are zero, or of rounding
 * size where a path forms them.
 *   psi0  as tbpm_dos_corr;  M >= 1. */
int kpm_moments(tbpm_ctx *ctx, const double *psi0, int nstates, int M, double *mu);

/* tbpm_quasi_eigenstates: quasi-eigenstates (QE, a TBPM capability benchmarked
 * in Sec. 4.2.2), the windowed Fourier transform of the evolved state over
 * positive and negative times,
 *   Psi(E_e) = dt/(2 pi) sum_{m=-N}^{N} w_m exp(i E_e t_m) psi(t_m),
 *   psi(t) = exp(-iHt) psi0, t_m = m dt, w_m = (1 + cos(pi m / N)) / 2,
 * with psi(t_m) from the same Chebyshev steps as tbpm_dos_corr (one forward
 * and one backward evolution). Accumulated in FP64.
 *   psi0      double[2n] one state;  dt > 0;  n_steps = N >= 1
 *   energies  double[n_e] (eV), 1 <= n_e <= 4096
 *   qe        double[2 * n_e * n] out, energy-major (Psi(E_e) at offset 2 n e)
 * Host or device buffers. Not available on batch contexts. */
int tbpm_quasi_eigenstates(tbpm_ctx *ctx, const double *psi0, double dt, int n_steps,
                           const double *energies, int n_e, double *qe);

/* tbpm_haydock: the recursion (Lanczos) coefficients of the local density
 * of states by the Haydock method (the LDOS capability of the TBPM solver,
 * Sec. 1; the LDOS row of the benchmarks, Sec. 4.2.2). With H not rescaled,
 * v_0 = psi0/||psi0||, v_{-1} = 0, b_0 = 0, for n = 0..M-1:
 *   w = H v_n - b_n v_{n-1},  a_n = Re <v_n|w>,  u = w - a_n v_n,
 *   b_{n+1} = ||u||,  v_{n+1} = u / b_{n+1}.
 *   psi0  double[2n] start state (a site state e_i gives the LDOS at site i),
 *         host or device, not necessarily normalised
 *   M     >= 1 levels;  a, b  double[M] out: a[n] = a_n, b[n] = b_{n+1}
 * A b_{n+1} at rounding level, <= tol (|a_n| + b_n) with tol = 1e-12 for FP64
 * contexts and 1e-6 for FP32 ones, marks an invariant subspace: it is returned
 * as 0 and every later a and b is 0. */
int tbpm_haydock(tbpm_ctx *ctx, const double *psi0, int M, double *a, double *b);

/* tbpm_haydock_ldos: rho(E_j) = -Im G(E_j + i eta) / pi with the continued
 * fraction G(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ... b_{M-1}^2/(z - a_{M-1}))),
 * on the GPU. a, b as returned by tbpm_haydock; energies double[n_e] (eV);
 * eta > 0 the broadening (eV); ldos double[n_e] out. Host or device. */
int tbpm_haydock_ldos(tbpm_ctx *ctx, const double *a, const double *b, int M, const double *energies,
                      int n_e, double eta, double *ldos);

/* ------------------------------------------------- AC conductivity */

/* Longest Fermi-operator series; its coefficients come from Chebyshev-Gauss
 * quadrature on 2 * TBPM_FERMI_MAX_TERMS nodes. */
#define TBPM_FERMI_MAX_TERMS 8192

/* tbpm_set_current: the current operators J_x, J_y of the context's
 * Hamiltonian (TBPM solvers take the Hamiltonian and the current operators as
 * sparse matrices, Sec. 2.3.4), used by tbpm_ac_corr. One CSR pattern, two
 * value arrays; with hbar = e = 1, (J_a)_ij = i (r_j - r_i)_a H_ij for each
 * hopping, r_j - r_i its bond vector.
 *   row_ptr  int64[n+1], col int32[nnz] (nnz = row_ptr[n]), host memory
 *   jx, jy   double[2*nnz] complex values, host memory
 * Duplicate (row, col) entries are summed. Each J_a must be Hermitian
 * (checked unless TBPM_F_NO_HERMITIAN_CHECK; TBPM_ERR_NOT_HERMITIAN).
 * Replaces earlier current operators. Copies the arrays; FP64 contexts of one
 * Hamiltonian only (batches: TBPM_ERR_UNSUPPORTED). */
int tbpm_set_current(tbpm_ctx *ctx, const int64_t *row_ptr, const int32_t *col, const double *jx,
                     const double *jy);

/* tbpm_ac_corr: the current-current correlation of the AC (optical)
 * conductivity, a TBPM capability of Sec. 1 benchmarked in Sec. 4.2.2, in the
 * standard TBPM form (hbar = e = 1):
 *   C_ab(t_m) = <phi| f(H) e^{iHt} J_a e^{-iHt} [1 - f(H)] J_b |phi>
 *             = <phi2(t_m)| J_a |phi1_b(t_m)>,   t_m = m dt,  m = 0..n_steps,
 *   phi2(t) = e^{-iHt} f(H) phi,  phi1_b(t) = e^{-iHt} [1 - f(H)] J_b phi,
 *   f(E) = 1 / (exp(beta (E - mu)) + 1).
 * f(H~) is the Chebyshev series f(rescale y) = sum_k a_k T_k(y) with
 *   a_k = (2 - delta_k0)/M sum_{j<M} f(rescale cos th_j) cos(k th_j),
 *   th_j = pi (j + 1/2) / M,  M = 2 TBPM_FERMI_MAX_TERMS,
 * cut after the last k with |a_k| >= 1e-12; the time steps are those of
 * tbpm_dos_corr (same dt, same Bessel cut-off).
 *   psi0   double[2n] one state (host or device), normally a random-phase state
 *   beta   > 0 (1/eV), mu the chemical potential (eV); dt != 0, n_steps >= 0
 *   corr   double[2 * 4 * (n_steps+1)] out (host or device): the rows C_xx,
 *          C_xy, C_yx, C_yy, each n_steps+1 complex values
 * TBPM_ERR_ARG when no current operators are set or when the Fermi series
 * needs more than TBPM_FERMI_MAX_TERMS terms (beta * rescale too large);
 * TBPM_ERR_UNSUPPORTED on FP32 or batch contexts. */
int tbpm_ac_corr(tbpm_ctx *ctx, const double *psi0, double beta, double mu, double dt, int n_steps,
                 double *corr);

/* tbpm_ac_cond: Re sigma_ab(w) from the correlations of tbpm_ac_corr, on the
 * GPU, with N = n_steps and the Hann window w_m = (1 + cos(pi m / N)) / 2:
 *   sigma_ab(w) = (exp(-beta w) - 1) / (w s) sum_{m=0}^{N-1} dt w_m sin(w t_m) 2 Im C_ab(t_m),
 * and sigma = 0 at w = 0 (the limit of this expression).
 *   corr    double[2 * 4 * (n_steps+1)] as written by tbpm_ac_corr; n_steps >= 1
 *   area    s > 0, the sample area per orbital (nm^2 when bond vectors are in nm)
 *   omegas  double[n_w] frequencies (eV); sigma double[4 * n_w] out, rows xx, xy, yx, yy
 * Host or device buffers. */
int tbpm_ac_cond(tbpm_ctx *ctx, const double *corr, int n_steps, double dt, double beta, double area,
                 const double *omegas, int n_w, double *sigma);

/* ------------------------------------------- allocation-free variant */

/* Largest orbital count tbpm_dos_corr_noalloc accepts. */
#define TBPM_NOALLOC_MAX_N 65536

/* tbpm_dos_corr_noalloc: tbpm_dos_corr for one state without any device
 * allocation. The paper has no counterpart to this call; it exists for
 * callers that cannot call cudaMalloc: an application that owns a fixed,
 * pre-planned device-memory budget and hands out every buffer itself, a
 * plugin whose host forbids allocation after start-up, or code on a path
 * where an allocation could block or fail at the wrong moment. Such a caller
 * passes every input and the output as device memory it already owns; the
 * working vectors live in one static device array of about 3.2 MB that the
 * library reserves on every GPU it is loaded on, for the life of the process.
 *   n        1 <= n <= TBPM_NOALLOC_MAX_N, else TBPM_ERR_UNSUPPORTED
 *   row_ptr, col, val  DEVICE CSR as in tbpm_create (int64[n+1], int32[nnz],
 *            complex double[nnz]); trusted as given (no structure, Hermiticity
 *            or Gershgorin check: the matrix is not read on the host)
 *   rescale  > 0;  psi0 DEVICE double[2n];  dt, n_steps as tbpm_dos_corr
 *   corr     DEVICE double[2(n_steps+1)]: C(t_0..t_n_steps)
 *   stream   cudaStream_t, or NULL for the legacy default stream
 * Every call waits on `stream` for the number of series terms (one 4-byte
 * device-to-host read), then enqueues the sweeps on `stream` and returns;
 * synchronise the stream before reading corr. The first call on a device
 * (and the first after that device's context was reset) looks up the static
 * array's device address with that device current; make that first call
 * before any stream capture. The array is per process and per device: all
 * calls of one process on one device share it and it keeps the last call's
 * contents, so calls of one process that overlap on the GPU (other streams
 * or host threads on the same device) race on it. Other processes have their
 * own copy. */
int tbpm_dos_corr_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const double *val, double rescale, const double *psi0, double dt,
                          int n_steps, double *corr, void *stream);

/* ------------------------------------------------------- DOS post-step */

/* tbpm_dos_from_corr: the DOS from one correlation (Analyzer.calc_dos,
 * Sec. 3.2.3), on the GPU: with N = n_steps, C(-t) = conj C(t) and the Hann
 * window w_m = (1 + cos(pi m / N)) / 2,
 *   D(E_j) = dt/(2 pi) sum_{m=-N}^{N-1} w_m C(t_m) exp(i E_j t_m),
 *   E_j = (j - N) pi / (N dt),  j = 0..2N-1.
 *   corr      double[2*(n_steps+1)] complex C(t_0..t_N), host or device
 *   energies  double[2N] out; dos double[2N] out (real part). n_steps >= 1. */
int tbpm_dos_from_corr(tbpm_ctx *ctx, const double *corr, int n_steps, double dt,
                       double *energies, double *dos);

/* kpm_dos_jackson: the KPM DOS with the Jackson kernel
 *   g_m = [(M-m+1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))] / (M+1),
 *   rho(x) = [g_0 mu_0 + 2 sum_{m>=1} g_m mu_m T_m(x)] / (pi sqrt(1-x^2)),
 * on the n_e Chebyshev nodes x_j = cos(pi (j+1/2)/n_e); energies[j] =
 * rescale*x_j, rho_out[j] = rho(x_j)/rescale. Uses Re(mu).
 *   mu  double[2*M] complex moments, host or device; n_e >= 1. */
int kpm_dos_jackson(tbpm_ctx *ctx, const double *mu, int M, int n_e, double *energies,
                    double *rho_out);

/* ---------------------------------------------------------- diagnostics */

typedef struct tbpm_info {
    int64_t n;                 /* orbitals                                      */
    int64_t nnz;               /* stored off-diagonal entries (0 for stencil)   */
    int path;                  /* TBPM_PATH_SELL | TBPM_PATH_STENCIL in use     */
    int precision;             /* TBPM_FP64 | TBPM_FP32                         */
    int real_values;           /* 1 when the stored hoppings are real           */
    int num_terms;             /* K of the last tbpm_dos_corr call              */
    int64_t passes;            /* sparse-product passes of the last call        */
    int64_t kernel_launches;   /* kernels the last call launched                */
    double gershgorin;         /* max_i sum_j |H_ij|                            */
    double rescale;
    int grid_blocks;           /* blocks of the single-state sweep grid         */
    int tuned;                 /* 1 when the shape was chosen by the autotuner  */
    int fermi_terms;           /* Fermi series length of the last tbpm_ac_corr  */
    int block_threads;         /* threads per block of the single-state sweeps  */
    int slices_per_warp;       /* 32-row slices a warp works on at once         */
    int tune_candidates;       /* launch shapes the autotuner timed (0: none)   */
    double tune_default_us;    /* autotuner: us per sweep (average over a time
                                  step) at the context's shape before tuning    */
    double tune_best_us;       /* autotuner: the same at the chosen shape       */
    int packed;                /* the stored matrix is also kept packed: 0 no,
                                  1 per entry, 2 one word per row
                                  (TBPM_F_PLAIN_SELL)                            */
} tbpm_info;

/* Fills *info with the context's layout and the counters of its last call. */
int tbpm_get_info(const tbpm_ctx *ctx, tbpm_info *info);

/* tbpm_fp64_peak: a measurement helper with no counterpart in the paper. It
 * times `reps` launches (after one warm-up each) of kernels that issue only
 * independent FP64 instructions on every SM of `device` (-1 = the current
 * device): FMA with parameter or register operands, MUL and ADD, 8 chains per
 * thread of `iters` rounds, at 1024 and 2048 threads per SM, and reports the
 * fastest launch as TFLOP/s, each FP64 instruction counted as 2 operations
 * (one issue slot of the FP64 pipe), in *tflops, and its duration in
 * *ms_per_launch (may be NULL): the measured ceiling of the FP64 sweeps, whose
 * FP64 instructions bound them on GB300. Allocates and frees a small device
 * buffer; blocks the host. 1 <= iters <= 2^26, reps >= 1, else TBPM_ERR_ARG;
 * no GPU: TBPM_ERR_NO_DEVICE. */
int tbpm_fp64_peak(int device, int iters, int reps, double *tflops, double *ms_per_launch);

/* A static, human-readable name for a status code. */
const char *tbpm_strerror(int status);

/* The detail of the context's most recent failure: the failing CUDA call with
 * CUDA's message, or for some rejected requests (no current operators, a Fermi
 * series beyond TBPM_FERMI_MAX_TERMS) what was wrong; "" if nothing was
 * recorded. Owned by the context, valid until its next failure or
 * tbpm_destroy. NULL ctx gives "". */
const char *tbpm_last_error(const tbpm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TBPM_H */
