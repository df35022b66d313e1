"""Pins for the oracle's Haydock (Lanczos) recursion and its continued-fraction LDOS."""
import numpy as np
import pytest

import tbpm_inputs as ti
from tbpm_inputs.lattice import CSR


def ring(L, t=-1.3):
    """Periodic 1D chain: H[i, i+1] = H[i+1, i] = t."""
    rows = np.repeat(np.arange(L), 2)
    cols = np.stack([(np.arange(L) - 1) % L, (np.arange(L) + 1) % L], axis=1)
    order = np.argsort(cols, axis=1)
    cols = np.take_along_axis(cols, order, axis=1).ravel()
    row_ptr = np.arange(0, 2 * L + 1, 2, dtype=np.int64)
    return CSR(L, row_ptr, cols.astype(np.int32), np.full(2 * L, t, dtype=np.complex128))


def test_chain_closed_form(orc):
    """Infinite chain from one site: a_n = 0, b_1 = sqrt(2)|t|, b_n = |t| (n >= 2),
    exact while the recursion has not reached around the ring (2n < L)."""
    t = -1.3
    h = ring(400, t)
    a, b = orc.haydock(h, ti.site_state(400, 17), 150)
    assert np.max(np.abs(a)) < 1e-13
    assert abs(b[0] - np.sqrt(2) * abs(t)) < 1e-13
    assert np.max(np.abs(b[1:] - abs(t))) < 1e-12


def test_moment_matching(orc):
    """The tridiagonal T_M reproduces <v0|H^k|v0> for k < 2M (a property of Lanczos)."""
    h = ti.graphene_csr(7, 6, onsite=ti.anderson_onsite(84, 1.0, 3), bond_phases=[0.3, 0.2, 0.7])
    psi0 = ti.random_phase_state(h.n, 2)
    M = 8
    a, b = orc.haydock(h, psi0, M)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    H = h.to_dense()
    v = psi0.copy()
    e0 = np.zeros(M)
    e0[0] = 1
    tk = e0.copy()
    for k in range(2 * M - 1):
        ref = np.vdot(psi0, v).real
        got = tk[0]
        assert abs(got - ref) < 1e-10 * max(1.0, abs(ref)), k
        v = H @ v
        tk = T @ tk


def test_ldos_against_exact_diagonalisation(orc):
    """With as many levels as orbitals the continued fraction equals
    G(z) = sum_m |<m|v0>|^2 / (z - E_m)."""
    h = ti.random_hermitian_csr(24, 3, seed=6, scale=2.0)
    psi0 = ti.site_state(h.n, 5)
    a, b = orc.haydock(h, psi0, h.n)
    lam, vec = np.linalg.eigh(h.to_dense())
    w = np.abs(vec[5, :]) ** 2
    E = np.linspace(-4, 4, 101)
    eta = 0.2
    ref = -np.imag((w[None, :] / (E[:, None] + 1j * eta - lam[None, :])).sum(1)) / np.pi
    got = orc.haydock_ldos(a, b, E, eta)
    assert np.max(np.abs(got - ref)) < 1e-8
    # LDOS integrates to ~1 (Lorentzian tails aside)
    EE = np.linspace(-60, 60, 24001)
    assert abs(np.trapezoid(orc.haydock_ldos(a, b, EE, eta), EE) - 1) < 5e-3


def test_invariant_subspace_stops(orc):
    """A 2-site dimer reaches an invariant subspace after two levels."""
    h = ti.graphene_csr(1, 1)               # 2 orbitals, coupled by 3t
    a, b = orc.haydock(h, ti.site_state(2, 0), 5)
    assert abs(b[0] - 8.1) < 1e-13 and b[1] == 0.0
    assert np.all(a[2:] == 0) and np.all(b[2:] == 0)
