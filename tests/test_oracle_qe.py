"""Pins for the oracle's quasi-eigenstates
Psi(E) = dt/(2 pi) sum_{m=-N}^{N} w_m exp(i E t_m) exp(-i H t_m) psi0 (Hann w_m)."""
import math

import numpy as np
import scipy.special as sp

import tbpm_inputs as ti


def kernel(omega, dt, N):
    m = np.arange(-N, N + 1)
    w = 0.5 * (1 + np.cos(np.pi * m / N))
    return (dt / (2 * np.pi)) * (w[None, :] * np.cos(np.outer(omega, m * dt))).sum(1)


def test_qe_against_exact_diagonalisation(orc):
    h = ti.graphene_csr(6, 5, onsite=ti.anderson_onsite(60, 1.0, 2), bond_phases=[0.4, 0.1, -0.8])
    psi0 = ti.random_phase_state(h.n, 3)
    dt, N = math.pi / 9, 64
    E = np.array([-5.0, -1.3, 0.0, 2.2])
    got = orc.quasi_eigenstates(h, 9.0, psi0, dt, N, E)
    lam, v = np.linalg.eigh(h.to_dense())
    amp = v.conj().T @ psi0
    ref = np.stack([v @ (kernel(e - lam, dt, N) * amp) for e in E])
    K = orc.cheb_num_terms(math.pi)
    bound = 2 * N * 2 * sum(abs(sp.jv(k, math.pi)) for k in range(K, K + 40)) * (dt / (2 * math.pi)) + 1e-13
    assert np.max(np.abs(got - ref)) <= bound


def test_qe_filters_an_eigenstate(orc):
    """psi0 equal to an eigenvector |k>: Psi(E) = K_N(E - E_k) |k>."""
    h = ti.random_hermitian_csr(30, 3, seed=4, scale=2.0)
    lam, v = np.linalg.eigh(h.to_dense())
    psi0 = v[:, 7].copy()
    dt, N = 0.3, 40
    E = np.array([lam[7], lam[7] + 0.5])
    got = orc.quasi_eigenstates(h, 9.0, psi0, dt, N, E)
    k = kernel(E - lam[7], dt, N)
    assert np.max(np.abs(got - k[:, None] * psi0[None, :])) < 1e-10
