"""FP64 CPU oracle for the TBPM hot path (test infrastructure only).

Only tests/, the smoke check and the CPU-baseline leg of bench.py import this
package. It wraps oracle/oracle.c with ctypes; see that file for the passages
of the paper and the textbook definitions each function follows.

Parity status per function (what pins it, all in tests/test_oracle_*.py):
  bessel_j, cheb_num_terms, cheb_coeffs  scipy.special.jv, sum rule, Jacobi-Anger
  propagate / dos_corr                   exact diagonalisation, Bloch closed form,
                                         site-state closed form, norm, reversibility,
                                         semigroup, error bound
  kpm_moments                            eigenvalue traces, closed form on pristine
                                         graphene, Chebyshev identities
  dos_hann                               sum rule, numpy FFT route, delta spectrum
  jackson, kpm_dos                       Gauss-Chebyshev integral, positivity,
                                         delta reconstruction
  quasi_eigenstates                      exact diagonalisation (windowed spectral sum)
  haydock, haydock_ldos                  closed-form chain coefficients, moment
                                         matching, exact diagonalisation
  fermi_coeffs                           the Fermi function off the quadrature nodes,
                                         adaptive quadrature, particle-hole symmetry
  ac_corr                                exact diagonalisation, C(0) and symmetry relations
  ac_cond                                spectral weight of a single transition
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build


def _bind(path: str):
    l = C.CDLL(path)
    d, i32, i64, p = C.c_double, C.c_int, C.c_int64, C.c_void_p
    l.oracle_bessel_j.restype = d
    l.oracle_bessel_j.argtypes = [i32, d]
    l.oracle_cheb_num_terms.restype = i32
    l.oracle_cheb_num_terms.argtypes = [d, d]
    l.oracle_cheb_coeffs.restype = None
    l.oracle_cheb_coeffs.argtypes = [d, i32, p]
    l.oracle_spmv.restype = None
    l.oracle_spmv.argtypes = [i64, p, p, p, d, p, p]
    l.oracle_propagate.restype = i32
    l.oracle_propagate.argtypes = [i64, p, p, p, d, p, d, i32, d, p, p]
    l.oracle_kpm_moments.restype = i32
    l.oracle_kpm_moments.argtypes = [i64, p, p, p, d, p, i32, p]
    l.oracle_dos_hann.restype = i32
    l.oracle_dos_hann.argtypes = [p, i32, d, p, p, p]
    l.oracle_jackson.restype = None
    l.oracle_jackson.argtypes = [i32, p]
    l.oracle_kpm_dos.restype = i32
    l.oracle_kpm_dos.argtypes = [p, i32, d, i32, p, p]
    l.oracle_haydock.restype = i32
    l.oracle_haydock.argtypes = [i64, p, p, p, p, i32, p, p]
    l.oracle_quasi_eigenstates.restype = i32
    l.oracle_quasi_eigenstates.argtypes = [i64, p, p, p, d, p, d, i32, d, i32, p, p]
    l.oracle_haydock_ldos.restype = None
    l.oracle_haydock_ldos.argtypes = [p, p, i32, p, i32, d, p]
    l.oracle_fermi_coeffs.restype = i32
    l.oracle_fermi_coeffs.argtypes = [d, d, d, d, i32, p]
    l.oracle_ac_corr.restype = i32
    l.oracle_ac_corr.argtypes = [i64, p, p, p, p, p, p, p, d, p, d, d, d, i32, d, d, i32, p]
    l.oracle_set_threads.restype = None
    l.oracle_set_threads.argtypes = [i32]
    l.oracle_get_threads.restype = i32
    l.oracle_get_threads.argtypes = []
    l.oracle_ac_cond.restype = i32
    l.oracle_ac_cond.argtypes = [p, i32, d, d, d, i32, p, p]
    return l


TOL = 1e-12
FERMI_TOL = 1e-12
FERMI_CAP = 8192


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(h):
    rp = np.ascontiguousarray(h.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(h.col, dtype=np.int32)
    val = np.ascontiguousarray(h.val, dtype=np.complex128)
    return rp, col, val


class Oracle:
    """The oracle's functions bound to one build of oracle.c (``path``)."""

    def __init__(self, path: str):
        self.path = path
        self._l = _bind(path)

    def set_threads(self, n: int) -> None:
        """OpenMP threads of the row loops (timing only; results do not depend on it)."""
        self._l.oracle_set_threads(int(n))

    def get_threads(self) -> int:
        return self._l.oracle_get_threads()

    def bessel_j(self, k: int, x: float) -> float:
        return self._l.oracle_bessel_j(int(k), float(x))

    def cheb_num_terms(self, x: float, tol: float = TOL) -> int:
        return self._l.oracle_cheb_num_terms(float(x), float(tol))

    def cheb_coeffs(self, x: float, K: int) -> np.ndarray:
        c = np.zeros(K, dtype=np.complex128)
        self._l.oracle_cheb_coeffs(float(x), int(K), _ptr(c))
        return c

    def spmv(self, h, x: np.ndarray, scale: float = 1.0) -> np.ndarray:
        rp, col, val = _csr(h)
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros(h.n, dtype=np.complex128)
        self._l.oracle_spmv(h.n, _ptr(rp), _ptr(col), _ptr(val), float(scale), _ptr(x), _ptr(y))
        return y

    def propagate(self, h, rescale: float, psi0: np.ndarray, dt: float, n_steps: int,
                  tol: float = TOL, want_corr: bool = True, want_psi: bool = False):
        """Returns (K, corr[n_steps+1] or None, psi(t_n_steps) or None)."""
        rp, col, val = _csr(h)
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        if psi0.shape != (h.n,):
            raise ValueError("psi0 must have one entry per orbital")
        corr = np.zeros(n_steps + 1, dtype=np.complex128) if want_corr else None
        psi = np.zeros(h.n, dtype=np.complex128) if want_psi else None
        K = self._l.oracle_propagate(h.n, _ptr(rp), _ptr(col), _ptr(val), float(rescale),
                                     _ptr(psi0), float(dt), int(n_steps), float(tol),
                                     _ptr(corr) if corr is not None else None,
                                     _ptr(psi) if psi is not None else None)
        if K < 0:
            raise RuntimeError(f"oracle_propagate failed: {K}")
        return K, corr, psi

    def dos_corr(self, h, rescale: float, psi0: np.ndarray, dt: float, n_steps: int,
                 tol: float = TOL) -> np.ndarray:
        """C(t_n) = <psi0|psi(t_n)>, n = 0..n_steps (complex128)."""
        return self.propagate(h, rescale, psi0, dt, n_steps, tol)[1]

    def kpm_moments(self, h, rescale: float, psi0: np.ndarray, M: int) -> np.ndarray:
        """mu_m = <psi0|T_m(H/rescale)|psi0>, m = 0..M-1 (complex128)."""
        rp, col, val = _csr(h)
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        mu = np.zeros(M, dtype=np.complex128)
        rc = self._l.oracle_kpm_moments(h.n, _ptr(rp), _ptr(col), _ptr(val), float(rescale),
                                        _ptr(psi0), int(M), _ptr(mu))
        if rc != 0:
            raise RuntimeError(f"oracle_kpm_moments failed: {rc}")
        return mu

    def dos_hann(self, corr: np.ndarray, dt: float):
        """(energies[2N], dos[2N], dos_imag[2N]) from corr[N+1]."""
        corr = np.ascontiguousarray(corr, dtype=np.complex128)
        n = corr.size - 1
        e, d, di = np.zeros(2 * n), np.zeros(2 * n), np.zeros(2 * n)
        rc = self._l.oracle_dos_hann(_ptr(corr), n, float(dt), _ptr(e), _ptr(d), _ptr(di))
        if rc != 0:
            raise RuntimeError(f"oracle_dos_hann failed: {rc}")
        return e, d, di

    def jackson(self, M: int) -> np.ndarray:
        g = np.zeros(M)
        self._l.oracle_jackson(int(M), _ptr(g))
        return g

    def kpm_dos(self, mu: np.ndarray, rescale: float, n_e: int):
        """(energies[n_e], rho[n_e]) on the Chebyshev nodes, Jackson kernel, Re(mu)."""
        mu_re = np.ascontiguousarray(np.real(mu), dtype=np.float64)
        e, r = np.zeros(n_e), np.zeros(n_e)
        rc = self._l.oracle_kpm_dos(_ptr(mu_re), mu_re.size, float(rescale), int(n_e), _ptr(e), _ptr(r))
        if rc != 0:
            raise RuntimeError(f"oracle_kpm_dos failed: {rc}")
        return e, r


    def quasi_eigenstates(self, h, rescale: float, psi0: np.ndarray, dt: float, n_steps: int,
                          energies, tol: float = TOL) -> np.ndarray:
        """Psi(E_e) for each energy: complex128 (n_e, n)."""
        rp, col, val = _csr(h)
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        e = np.ascontiguousarray(energies, dtype=np.float64)
        out = np.zeros((e.size, h.n), dtype=np.complex128)
        rc = self._l.oracle_quasi_eigenstates(h.n, _ptr(rp), _ptr(col), _ptr(val), float(rescale), _ptr(psi0),
                                              float(dt), int(n_steps), float(tol), e.size, _ptr(e), _ptr(out))
        if rc != 0:
            raise RuntimeError(f"oracle_quasi_eigenstates failed: {rc}")
        return out

    def haydock(self, h, psi0: np.ndarray, M: int):
        """Recursion coefficients (a[M], b[M]) with b[m] = b_{m+1} (H not rescaled)."""
        rp, col, val = _csr(h)
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        a, b = np.zeros(M), np.zeros(M)
        rc = self._l.oracle_haydock(h.n, _ptr(rp), _ptr(col), _ptr(val), _ptr(psi0), int(M), _ptr(a), _ptr(b))
        if rc != 0:
            raise RuntimeError(f"oracle_haydock failed: {rc}")
        return a, b

    def haydock_ldos(self, a, b, energies, eta: float) -> np.ndarray:
        """-Im G(E + i eta)/pi from the continued fraction of (a, b)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        e = np.ascontiguousarray(energies, dtype=np.float64)
        out = np.zeros(e.size)
        self._l.oracle_haydock_ldos(_ptr(a), _ptr(b), a.size, _ptr(e), e.size, float(eta), _ptr(out))
        return out

    def fermi_coeffs(self, beta: float, mu: float, rescale: float, tol: float = FERMI_TOL,
                     kcap: int = FERMI_CAP):
        """(K, a[kcap]): Chebyshev coefficients of the Fermi-Dirac function on the
        rescaled spectrum and the number of terms kept at ``tol``."""
        a = np.zeros(kcap)
        K = self._l.oracle_fermi_coeffs(float(beta), float(mu), float(rescale), float(tol), int(kcap), _ptr(a))
        if K < 0:
            raise RuntimeError(f"oracle_fermi_coeffs failed: {K}")
        return K, a

    def ac_corr(self, h, current, rescale: float, psi0: np.ndarray, beta: float, mu: float, dt: float,
                n_steps: int, tol: float = TOL, ftol: float = FERMI_TOL, kcap: int = FERMI_CAP):
        """(K_F, corr[4, n_steps+1]) for (xx, xy, yx, yy); current = (row_ptr, col, jx, jy)."""
        rp, col, val = _csr(h)
        jrp = np.ascontiguousarray(current[0], dtype=np.int64)
        jcol = np.ascontiguousarray(current[1], dtype=np.int32)
        jx = np.ascontiguousarray(current[2], dtype=np.complex128)
        jy = np.ascontiguousarray(current[3], dtype=np.complex128)
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        corr = np.zeros((4, n_steps + 1), dtype=np.complex128)
        K = self._l.oracle_ac_corr(h.n, _ptr(rp), _ptr(col), _ptr(val), _ptr(jrp), _ptr(jcol), _ptr(jx), _ptr(jy),
                                   float(rescale), _ptr(psi0), float(beta), float(mu), float(dt), int(n_steps),
                                   float(tol), float(ftol), int(kcap), _ptr(corr))
        if K < 0:
            raise RuntimeError(f"oracle_ac_corr failed: {K}")
        return K, corr

    def ac_cond(self, corr: np.ndarray, dt: float, beta: float, area: float, omegas) -> np.ndarray:
        """Re sigma(w) of one correlation row."""
        corr = np.ascontiguousarray(corr, dtype=np.complex128)
        w = np.ascontiguousarray(omegas, dtype=np.float64)
        out = np.zeros(w.size)
        rc = self._l.oracle_ac_cond(_ptr(corr), corr.size - 1, float(dt), float(beta), float(area), w.size,
                                    _ptr(w), _ptr(out))
        if rc != 0:
            raise RuntimeError(f"oracle_ac_cond failed: {rc}")
        return out


_default = None


def default() -> Oracle:
    """The oracle built from oracle/oracle.c (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(_build())
    return _default


def lib():
    return default()._l


def __getattr__(name):
    # module-level access to the default instance: oracle.propagate(...), etc.
    if name in ("bessel_j", "cheb_num_terms", "cheb_coeffs", "spmv", "propagate", "dos_corr",
                "kpm_moments", "dos_hann", "jackson", "kpm_dos", "haydock", "haydock_ldos",
                "quasi_eigenstates", "fermi_coeffs", "ac_corr", "ac_cond", "set_threads", "get_threads"):
        return getattr(default(), name)
    raise AttributeError(name)
