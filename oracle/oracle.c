/*
 * TBPM oracle: a plain, slow FP64 CPU implementation of what the TBPM hot path
 * computes. TEST INFRASTRUCTURE ONLY: it is called by tests/, by the smoke check
 * and by the CPU-baseline leg of bench.py, never by the library. It shares no
 * code, header or constant with the CUDA path.
 *
 * What it follows (TBPLaS 2.0, arXiv 2509.26309):
 *   - Sec. 2.2.1 and its two propagation listings: the wave function after one
 *     time step is a Chebyshev series of the rescaled Hamiltonian,
 *     psi(t+dt) = sum_k c_k T_k(H~) psi(t), with the imaginary factor carried
 *     by the coefficients so the sparse product stays real-scalar, and the
 *     polynomials built by the three-term recurrence T_k = 2 H~ T_{k-1} - T_{k-2}.
 *   - Sec. 3.2.3 (calc_corr_dos): the DOS correlation C(t_n) = <psi0|psi(t_n)>
 *     of a random-phase state, H~ = H / rescale (config.rescale).
 *   - Sec. 1: the kernel polynomial method, mu_n = <psi0|T_n(H~)|psi0>, and
 *     the local DOS by the Haydock recursion method (benchmarked as LDOS in
 *     Sec. 4.2.2).
 * Formulas the paper does not print are taken as their textbook definitions:
 *   - c_0 = J_0(x), c_k = 2 (-i)^k J_k(x), x = dt * rescale: the Jacobi-Anger
 *     expansion of exp(-i x y) on y in [-1, 1] (Abramowitz-Stegun 9.1.44/45),
 *     which is the sign convention exp(-iHt);
 *   - J_k by its power series (A&S 9.1.10), summed in long double;
 *   - the series is cut at K = the first k > x with |J_k(x)| < tol;
 *   - the DOS as the Hann-windowed discrete Fourier transform of C(t) with
 *     C(-t) = conj C(t), and the KPM DOS with the Jackson kernel
 *     (Weisse et al., Rev. Mod. Phys. 78, 275 (2006), Eqs. 71 and 81).
 *
 * Complex vectors are arrays of double _Complex (re, im interleaved).
 * CSR: row_ptr int64[n+1], col int32[nnz], val double _Complex[nnz].
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_OOM (-2)

/* ---------------------------------------------------------------- Bessel */

/* J_k(x) = sum_{m>=0} (-1)^m (x/2)^{2m+k} / (m! (m+k)!)  (A&S 9.1.10), k >= 0.
 * Each term is built from the previous one; the sum stops once a term is below
 * 1e-40 of the running magnitude and past the peak term. */
double oracle_bessel_j(int k, double x)
{
    if (k < 0) return NAN;
    long double h = 0.5L * (long double)x;
    long double term = 1.0L;
    for (int j = 1; j <= k; ++j) term *= h / (long double)j;       /* (x/2)^k / k! */
    long double sum = term;
    long double big = fabsl(term);
    for (int m = 1; m < 500; ++m) {
        term *= -(h * h) / ((long double)m * (long double)(m + k));
        sum += term;
        if (fabsl(sum) > big) big = fabsl(sum);
        if (fabsl(term) > big) big = fabsl(term);
        if ((long double)m > h && fabsl(term) < 1e-40L * (big > 0 ? big : 1.0L)) break;
    }
    return (double)sum;
}

/* Number of Chebyshev terms K: the first k > x with |J_k(x)| < tol. */
int oracle_cheb_num_terms(double x, double tol)
{
    double ax = fabs(x);
    for (int k = 1; k < 100000; ++k) {
        if ((double)k > ax && fabs(oracle_bessel_j(k, ax)) < tol) return k;
    }
    return -1;
}

/* c_k = (2 - delta_k0) (-i)^k J_k(x), k = 0..K-1, written as K complex numbers.
 * For x < 0, J_k(-x) = (-1)^k J_k(x) is used (A&S 9.1.5), which is the same as
 * evaluating the series at negative x. */
void oracle_cheb_coeffs(double x, int K, cplx *c)
{
    for (int k = 0; k < K; ++k) {
        double j = oracle_bessel_j(k, fabs(x));
        if (x < 0 && (k & 1)) j = -j;
        cplx mi_k;                         /* (-i)^k */
        switch (k & 3) {
        case 0: mi_k = 1.0; break;
        case 1: mi_k = -I; break;
        case 2: mi_k = -1.0; break;
        default: mi_k = I; break;
        }
        c[k] = (k == 0 ? 1.0 : 2.0) * mi_k * j;
    }
}

/* OpenMP threads for the row loops (timing on one core and on all of them). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ sparse ops */

/* y = s * H x for CSR H (plain row loop). */
static void spmv(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                 double s, const cplx *x, cplx *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        cplx acc = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc += val[p] * x[col[p]];
        y[i] = s * acc;
    }
}

/* <a|b> = sum_i conj(a_i) b_i, serial FP64 sum in index order. */
static cplx dot(int64_t n, const cplx *a, const cplx *b)
{
    cplx acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += conj(a[i]) * b[i];
    return acc;
}

void oracle_spmv(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                 double s, const cplx *x, cplx *y)
{
    spmv(n, rp, col, val, s, x, y);
}

/* ------------------------------------------------------------ propagation */

/* One time step: out = sum_{k<K} c_k T_k(H~) psi with T_0 = psi, T_1 = H~ psi,
 * T_k = 2 H~ T_{k-1} - T_{k-2}. Separate arrays, no fusion. */
static void cheb_step(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                      double rescale, int K, const cplx *c, const cplx *psi, cplx *out,
                      cplx *t0, cplx *t1, cplx *t2)
{
    memcpy(t0, psi, (size_t)n * sizeof(cplx));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = c[0] * t0[i];
    if (K < 2) return;
    spmv(n, rp, col, val, 1.0 / rescale, t0, t1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] += c[1] * t1[i];
    for (int k = 2; k < K; ++k) {
        spmv(n, rp, col, val, 2.0 / rescale, t1, t2);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            t2[i] -= t0[i];
            out[i] += c[k] * t2[i];
        }
        cplx *tmp = t0; t0 = t1; t1 = t2; t2 = tmp;
    }
}

/* Propagates psi0 through n_steps steps of dt. Writes corr[0..n_steps]
 * (C(t_n) = <psi0|psi(t_n)>, corr may be NULL) and the final state psi_out
 * (may be NULL). Returns K, or a negative error. */
int oracle_propagate(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                     double rescale, const cplx *psi0, double dt, int n_steps, double tol,
                     cplx *corr, cplx *psi_out)
{
    if (n <= 0 || !rp || !col || !val || !psi0 || n_steps < 0 || !(rescale > 0)) return ORACLE_ERR_ARG;
    double x = dt * rescale;
    int K = oracle_cheb_num_terms(x, tol);
    if (K < 1) return ORACLE_ERR_ARG;
    cplx *c = malloc((size_t)K * sizeof(cplx));
    cplx *psi = malloc((size_t)n * sizeof(cplx));
    cplx *out = malloc((size_t)n * sizeof(cplx));
    cplx *t0 = malloc((size_t)n * sizeof(cplx));
    cplx *t1 = malloc((size_t)n * sizeof(cplx));
    cplx *t2 = malloc((size_t)n * sizeof(cplx));
    if (!c || !psi || !out || !t0 || !t1 || !t2) {
        free(c); free(psi); free(out); free(t0); free(t1); free(t2);
        return ORACLE_ERR_OOM;
    }
    oracle_cheb_coeffs(x, K, c);
    memcpy(psi, psi0, (size_t)n * sizeof(cplx));
    if (corr) corr[0] = dot(n, psi0, psi);
    for (int s = 0; s < n_steps; ++s) {
        cheb_step(n, rp, col, val, rescale, K, c, psi, out, t0, t1, t2);
        cplx *tmp = psi; psi = out; out = tmp;
        if (corr) corr[s + 1] = dot(n, psi0, psi);
    }
    if (psi_out) memcpy(psi_out, psi, (size_t)n * sizeof(cplx));
    free(c); free(psi); free(out); free(t0); free(t1); free(t2);
    return K;
}

/* Quasi-eigenstates (a TBPM capability of Sec. 4.2.2): the windowed Fourier
 * transform of the evolved state over positive and negative times,
 *   Psi(E_e) = dt/(2 pi) sum_{m=-N}^{N} w_m exp(i E_e t_m) psi(t_m),
 *   psi(t) = exp(-iHt) psi0,  t_m = m dt,  w_m = (1 + cos(pi m / N)) / 2,
 * with psi(t_m) from the Chebyshev steps of oracle_propagate (forward with
 * dt, backward with -dt). qe_out: n_e x n complex, energy-major. */
int oracle_quasi_eigenstates(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                             double rescale, const cplx *psi0, double dt, int n_steps, double tol,
                             int n_e, const double *energies, cplx *qe_out)
{
    if (n <= 0 || !rp || !col || !val || !psi0 || n_steps < 1 || !(rescale > 0) || !(dt > 0) ||
        n_e < 1 || !energies || !qe_out)
        return ORACLE_ERR_ARG;
    int N = n_steps;
    double pre = dt / (2.0 * PI);
    for (int e = 0; e < n_e; ++e)
        for (int64_t i = 0; i < n; ++i) qe_out[(int64_t)e * n + i] = pre * psi0[i];   /* m = 0, w_0 = 1 */
    for (int dir = 0; dir < 2; ++dir) {
        double h = dir == 0 ? dt : -dt;
        double x = h * rescale;
        int K = oracle_cheb_num_terms(x, tol);
        if (K < 1) return ORACLE_ERR_ARG;
        cplx *c = malloc((size_t)K * sizeof(cplx));
        cplx *psi = malloc((size_t)n * sizeof(cplx));
        cplx *out = malloc((size_t)n * sizeof(cplx));
        cplx *t0 = malloc((size_t)n * sizeof(cplx));
        cplx *t1 = malloc((size_t)n * sizeof(cplx));
        cplx *t2 = malloc((size_t)n * sizeof(cplx));
        if (!c || !psi || !out || !t0 || !t1 || !t2) {
            free(c); free(psi); free(out); free(t0); free(t1); free(t2);
            return ORACLE_ERR_OOM;
        }
        oracle_cheb_coeffs(x, K, c);
        memcpy(psi, psi0, (size_t)n * sizeof(cplx));
        for (int s = 1; s <= N; ++s) {
            cheb_step(n, rp, col, val, rescale, K, c, psi, out, t0, t1, t2);
            cplx *tmp = psi; psi = out; out = tmp;
            double t = s * h;
            double w = 0.5 * (1.0 + cos(PI * (double)s / (double)N));
            for (int e = 0; e < n_e; ++e) {
                cplx ph = pre * w * cexp(I * energies[e] * t);
                for (int64_t i = 0; i < n; ++i) qe_out[(int64_t)e * n + i] += ph * psi[i];
            }
        }
        free(c); free(psi); free(out); free(t0); free(t1); free(t2);
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------- KPM */

/* mu_m = <psi0|T_m(H~)|psi0>, m = 0..M-1, by the plain recurrence (no doubling). */
int oracle_kpm_moments(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                       double rescale, const cplx *psi0, int M, cplx *mu)
{
    if (n <= 0 || !rp || !col || !val || !psi0 || !mu || M < 1 || !(rescale > 0)) return ORACLE_ERR_ARG;
    cplx *t0 = malloc((size_t)n * sizeof(cplx));
    cplx *t1 = malloc((size_t)n * sizeof(cplx));
    cplx *t2 = malloc((size_t)n * sizeof(cplx));
    if (!t0 || !t1 || !t2) { free(t0); free(t1); free(t2); return ORACLE_ERR_OOM; }
    memcpy(t0, psi0, (size_t)n * sizeof(cplx));
    mu[0] = dot(n, psi0, t0);
    if (M > 1) {
        spmv(n, rp, col, val, 1.0 / rescale, t0, t1);
        mu[1] = dot(n, psi0, t1);
    }
    for (int m = 2; m < M; ++m) {
        spmv(n, rp, col, val, 2.0 / rescale, t1, t2);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) t2[i] -= t0[i];
        mu[m] = dot(n, psi0, t2);
        cplx *tmp = t0; t0 = t1; t1 = t2; t2 = tmp;
    }
    free(t0); free(t1); free(t2);
    return ORACLE_OK;
}

/* ------------------------------------------------------- Haydock / LDOS */

/* Haydock recursion (the Lanczos tridiagonalisation used for the local DOS;
 * Haydock, Heine, Kelly, J. Phys. C 8, 2591 (1975)) of H (not rescaled) from
 * v_0 = psi0/||psi0||, v_{-1} = 0, b_0 = 0, for n = 0..M-1:
 *   w = H v_n - b_n v_{n-1},  a_n = Re <v_n|w>,  u = w - a_n v_n,
 *   b_{n+1} = ||u||,  v_{n+1} = u / b_{n+1}.
 * Writes a[n] = a_n and b[n] = b_{n+1}. If b_{n+1} <= 1e-12 (|a_n| + b_n) the
 * recursion has found an invariant subspace (up to rounding): b_{n+1} is set
 * to 0 and every later a and b is 0. */
int oracle_haydock(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                   const cplx *psi0, int M, double *a, double *b)
{
    if (n <= 0 || !rp || !col || !val || !psi0 || M < 1 || !a || !b) return ORACLE_ERR_ARG;
    cplx *vp = calloc((size_t)n, sizeof(cplx));
    cplx *v = malloc((size_t)n * sizeof(cplx));
    cplx *w = malloc((size_t)n * sizeof(cplx));
    if (!vp || !v || !w) { free(vp); free(v); free(w); return ORACLE_ERR_OOM; }
    double nrm = sqrt(creal(dot(n, psi0, psi0)));
    if (!(nrm > 0)) { free(vp); free(v); free(w); return ORACLE_ERR_ARG; }
    for (int64_t i = 0; i < n; ++i) v[i] = psi0[i] / nrm;
    double bn = 0.0;
    int stopped = 0;
    for (int m = 0; m < M; ++m) {
        if (stopped) { a[m] = 0.0; b[m] = 0.0; continue; }
        spmv(n, rp, col, val, 1.0, v, w);
        for (int64_t i = 0; i < n; ++i) w[i] -= bn * vp[i];
        double am = creal(dot(n, v, w));
        for (int64_t i = 0; i < n; ++i) w[i] -= am * v[i];
        double bm = sqrt(creal(dot(n, w, w)));
        /* the chain ends when b_{n+1} is rounding noise against the level's scale */
        if (bm <= 1e-12 * (fabs(am) + bn)) bm = 0.0;
        a[m] = am;
        b[m] = bm;
        if (bm == 0.0) { stopped = 1; continue; }
        for (int64_t i = 0; i < n; ++i) { vp[i] = v[i]; v[i] = w[i] / bm; }
        bn = bm;
    }
    free(vp); free(v); free(w);
    return ORACLE_OK;
}

/* Local DOS from the recursion coefficients: rho(E) = -Im G(E + i eta) / pi,
 * G(z) = 1 / (z - a_0 - b_1^2 / (z - a_1 - b_2^2 / ( ... / (z - a_{M-1})))),
 * evaluated from the bottom level up (b[m] = b_{m+1}). */
void oracle_haydock_ldos(const double *a, const double *b, int M, const double *energies, int n_e,
                         double eta, double *ldos)
{
    for (int j = 0; j < n_e; ++j) {
        cplx z = energies[j] + I * eta;
        cplx g = 0.0;                       /* 1 / (z - a_m - b_{m+1}^2 g_{m+1}) */
        for (int m = M - 1; m >= 0; --m) {
            cplx tail = (m == M - 1) ? 0.0 : b[m] * b[m] * g;
            g = 1.0 / (z - a[m] - tail);
        }
        ldos[j] = -cimag(g) / PI;
    }
}

/* ------------------------------------------------------------------- DOS */

/* Hann-windowed DFT of the correlation. With N = n_steps, t_n = n dt,
 * C(t_{-n}) = conj C(t_n), w_n = (1 + cos(pi n / N)) / 2 for |n| <= N:
 *   D(E_j) = dt/(2 pi) sum_{n=-N}^{N-1} w_n C(t_n) exp(i E_j t_n),
 *   E_j = (j - N) dE, dE = pi / (N dt), j = 0..2N-1.
 * Direct O(N^2) sum; writes energies[2N], dos_re[2N] and dos_im[2N] (the
 * imaginary part is a consistency check, zero up to rounding). */
int oracle_dos_hann(const cplx *corr, int n_steps, double dt, double *energies,
                    double *dos_re, double *dos_im)
{
    if (!corr || n_steps < 1 || !(dt > 0) || !energies || !dos_re) return ORACLE_ERR_ARG;
    int N = n_steps;
    double de = PI / (N * dt);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < 2 * N; ++j) {
        double e = (j - N) * de;
        cplx acc = 0.0;
        for (int m = -N; m <= N - 1; ++m) {
            int a = m < 0 ? -m : m;
            cplx cm = m < 0 ? conj(corr[a]) : corr[a];
            double w = 0.5 * (1.0 + cos(PI * (double)m / (double)N));
            double t = m * dt;
            acc += w * cm * cexp(I * e * t);
        }
        acc *= dt / (2.0 * PI);
        energies[j] = e;
        dos_re[j] = creal(acc);
        if (dos_im) dos_im[j] = cimag(acc);
    }
    return ORACLE_OK;
}

/* Jackson kernel g_m, m = 0..M-1 (Weisse et al. 2006, Eq. 71). */
void oracle_jackson(int M, double *g)
{
    double q = PI / (M + 1);
    for (int m = 0; m < M; ++m)
        g[m] = ((M - m + 1) * cos(q * m) + sin(q * m) / tan(q)) / (M + 1);
}

/* KPM DOS on the Chebyshev nodes x_j = cos(pi (j + 1/2) / n_e), j = 0..n_e-1:
 *   rho(x) = [g_0 mu_0 + 2 sum_{m>=1} g_m mu_m T_m(x)] / (pi sqrt(1 - x^2)),
 * energies E_j = rescale * x_j and rho(E) = rho(x) / rescale. Uses Re(mu). */
int oracle_kpm_dos(const double *mu_re, int M, double rescale, int n_e, double *energies, double *rho)
{
    if (!mu_re || M < 1 || n_e < 1 || !(rescale > 0) || !energies || !rho) return ORACLE_ERR_ARG;
    double *g = malloc((size_t)M * sizeof(double));
    if (!g) return ORACLE_ERR_OOM;
    oracle_jackson(M, g);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n_e; ++j) {
        double x = cos(PI * (j + 0.5) / n_e);
        double th = acos(x);
        double s = g[0] * mu_re[0];
        for (int m = 1; m < M; ++m) s += 2.0 * g[m] * mu_re[m] * cos(m * th);
        energies[j] = rescale * x;
        rho[j] = s / (PI * sqrt(1.0 - x * x)) / rescale;
    }
    free(g);
    return ORACLE_OK;
}

/* ------------------------------------------------------ AC conductivity */
/*
 * Optical (AC) conductivity is one of the TBPM capabilities the paper lists
 * (Sec. 1) and benchmarks (Sec. 4.2.2); TBPM solvers take the Hamiltonian and
 * the current operators as sparse matrices (Sec. 2.3.4). The paper prints no
 * formula, so the definitions are the standard TBPM ones (Yuan, De Raedt and
 * Katsnelson, Phys. Rev. B 82, 115448 (2010)), with hbar = e = 1:
 *
 *   f(E) = 1 / (exp(beta (E - mu)) + 1)                    Fermi-Dirac
 *   C_ab(t) = <phi| f(H) J_a(t) [1 - f(H)] J_b |phi>,     J_a(t) = e^{iHt} J_a e^{-iHt}
 *           = <phi2(t)| J_a |phi1_b(t)>,
 *   phi2(t) = e^{-iHt} f(H) phi,  phi1_b(t) = e^{-iHt} [1 - f(H)] J_b phi,
 *   Re sigma_ab(w) = (exp(-beta w) - 1) / (w s) * int_0^T w(t) sin(w t) 2 Im C_ab(t) dt,
 *
 * s the area per orbital, the time integral a Hann-windowed sum over the
 * steps t_n = n dt, n < N. f(H) is the Chebyshev series of f on the rescaled
 * spectrum, with coefficients from Chebyshev-Gauss quadrature.
 */

/* Fermi-Dirac occupation, evaluated on the side where the exponential is <= 1. */
static double fermi(double beta, double mu, double e)
{
    double z = beta * (e - mu);
    if (z > 0.0) {
        double q = exp(-z);
        return q / (1.0 + q);
    }
    return 1.0 / (1.0 + exp(z));
}

/* a_k, k < kcap, of f(rescale * y) = sum_k a_k T_k(y) on [-1, 1]:
 *   a_k = (2 - delta_k0) / M sum_{j<M} f(rescale cos th_j) cos(k th_j),
 *   th_j = pi (j + 1/2) / M,  M = 2 kcap nodes.
 * Returns K = 1 + the last k with |a_k| >= tol, or ORACLE_ERR_ARG when the
 * series has not fallen below tol by k = kcap - 1 (temperature too low for
 * kcap terms). */
int oracle_fermi_coeffs(double beta, double mu, double rescale, double tol, int kcap, double *a)
{
    if (!(beta > 0) || !(rescale > 0) || !(tol > 0) || kcap < 2 || !a) return ORACLE_ERR_ARG;
    int M = 2 * kcap;
    double *fj = malloc((size_t)M * sizeof(double));
    if (!fj) return ORACLE_ERR_OOM;
    for (int j = 0; j < M; ++j) fj[j] = fermi(beta, mu, rescale * cos(PI * (j + 0.5) / M));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < kcap; ++k) {
        double s = 0.0;
        for (int j = 0; j < M; ++j) s += fj[j] * cos(k * (PI * (j + 0.5) / M));
        a[k] = (k == 0 ? 1.0 : 2.0) * s / M;
    }
    free(fj);
    int K = 0;
    for (int k = 0; k < kcap; ++k)
        if (fabs(a[k]) >= tol) K = k + 1;
    if (K >= kcap) return ORACLE_ERR_ARG;
    return K < 1 ? 1 : K;
}

/* C_ab(t_n), n = 0..n_steps, for (a, b) = (x, x), (x, y), (y, x), (y, y):
 * corr is 4 x (n_steps + 1), correlation-major. The current operators J_x,
 * J_y share one CSR pattern (jrp, jcol) with values jx, jy. f(H~) is applied
 * by the forward Chebyshev recurrence with the a_k of oracle_fermi_coeffs
 * (kcap terms at most, cut at ftol), 1 - f(H~) as v - f(H~) v; each step is
 * the propagation step of oracle_propagate. Returns the Fermi term count. */
int oracle_ac_corr(int64_t n, const int64_t *rp, const int32_t *col, const cplx *val,
                   const int64_t *jrp, const int32_t *jcol, const cplx *jx, const cplx *jy,
                   double rescale, const cplx *psi0, double beta, double mu, double dt, int n_steps,
                   double tol, double ftol, int kcap, cplx *corr)
{
    if (n <= 0 || !rp || !col || !val || !jrp || !jcol || !jx || !jy || !psi0 || !corr || n_steps < 0 ||
        !(rescale > 0))
        return ORACLE_ERR_ARG;
    double *a = malloc((size_t)kcap * sizeof(double));
    if (!a) return ORACLE_ERR_OOM;
    int KF = oracle_fermi_coeffs(beta, mu, rescale, ftol, kcap, a);
    if (KF < 1) { free(a); return KF; }
    int K = oracle_cheb_num_terms(dt * rescale, tol);
    if (K < 1) { free(a); return ORACLE_ERR_ARG; }
    cplx *fc = malloc((size_t)KF * sizeof(cplx));
    cplx *c = malloc((size_t)K * sizeof(cplx));
    cplx *v[3], *u = malloc((size_t)n * sizeof(cplx)), *out = malloc((size_t)n * sizeof(cplx));
    cplx *t0 = malloc((size_t)n * sizeof(cplx)), *t1 = malloc((size_t)n * sizeof(cplx));
    cplx *t2 = malloc((size_t)n * sizeof(cplx));
    for (int q = 0; q < 3; ++q) v[q] = malloc((size_t)n * sizeof(cplx));
    int ok = fc && c && u && out && t0 && t1 && t2 && v[0] && v[1] && v[2];
    if (ok) {
        for (int k = 0; k < KF; ++k) fc[k] = a[k];
        oracle_cheb_coeffs(dt * rescale, K, c);
        /* v[0] = phi2 = f(H~) phi */
        cheb_step(n, rp, col, val, rescale, KF, fc, psi0, v[0], t0, t1, t2);
        /* v[1] = phi1_x = [1 - f(H~)] J_x phi, v[2] = phi1_y */
        for (int b = 0; b < 2; ++b) {
            spmv(n, jrp, jcol, b == 0 ? jx : jy, 1.0, psi0, u);
            cheb_step(n, rp, col, val, rescale, KF, fc, u, out, t0, t1, t2);
            for (int64_t i = 0; i < n; ++i) v[1 + b][i] = u[i] - out[i];
        }
        for (int s = 0; s <= n_steps; ++s) {
            for (int al = 0; al < 2; ++al) {
                spmv(n, jrp, jcol, al == 0 ? jx : jy, 1.0, v[0], u);     /* J_a phi2 (J_a Hermitian) */
                for (int b = 0; b < 2; ++b)
                    corr[(size_t)(2 * al + b) * (n_steps + 1) + s] = dot(n, u, v[1 + b]);
            }
            if (s == n_steps) break;
            for (int q = 0; q < 3; ++q) {
                cheb_step(n, rp, col, val, rescale, K, c, v[q], out, t0, t1, t2);
                memcpy(v[q], out, (size_t)n * sizeof(cplx));
            }
        }
    }
    free(a); free(fc); free(c); free(u); free(out); free(t0); free(t1); free(t2);
    for (int q = 0; q < 3; ++q) free(v[q]);
    return ok ? KF : ORACLE_ERR_OOM;
}

/* Re sigma(w_j) from one correlation row C(t_n), n = 0..n_steps:
 *   sigma(w) = (exp(-beta w) - 1) / (w s) sum_{n=0}^{N-1} dt w_n sin(w t_n) 2 Im C(t_n),
 *   w_n = (1 + cos(pi n / N)) / 2,  N = n_steps;  sigma(0) = 0 (the limit w -> 0). */
int oracle_ac_cond(const cplx *corr, int n_steps, double dt, double beta, double s, int n_w,
                   const double *omegas, double *sigma)
{
    if (!corr || n_steps < 1 || !(dt > 0) || !(s > 0) || n_w < 1 || !omegas || !sigma) return ORACLE_ERR_ARG;
    int N = n_steps;
    for (int j = 0; j < n_w; ++j) {
        double w = omegas[j];
        if (w == 0.0) { sigma[j] = 0.0; continue; }
        double acc = 0.0;
        for (int m = 0; m < N; ++m) {
            double win = 0.5 * (1.0 + cos(PI * (double)m / (double)N));
            acc += dt * win * sin(w * m * dt) * 2.0 * cimag(corr[m]);
        }
        sigma[j] = (exp(-beta * w) - 1.0) / (w * s) * acc;
    }
    return ORACLE_OK;
}
