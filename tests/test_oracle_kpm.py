"""Pins for the oracle's KPM moments mu_m = <psi0|T_m(H/rescale)|psi0>."""
import numpy as np
import pytest

import tbpm_inputs as ti

RESCALE = 9.0


def cheb_t(m, x):
    return np.cos(np.outer(np.arange(m), np.arccos(np.clip(x, -1, 1))))


def test_trace_from_eigenvalues(orc):
    """sum_i <e_i|T_m(H~)|e_i> = tr T_m(H~) = sum_l T_m(lambda_l / rescale), exactly."""
    h = ti.random_hermitian_csr(40, 3, seed=9, scale=2.0)
    M = 64
    tr = sum(orc.kpm_moments(h, RESCALE, ti.site_state(h.n, i), M) for i in range(h.n))
    lam = np.linalg.eigvalsh(h.to_dense())
    ref = cheb_t(M, lam / RESCALE).sum(1)
    assert np.max(np.abs(tr - ref)) < 1e-11


@pytest.mark.parametrize("maker", [
    lambda: ti.bilayer_csr(5, 5, onsite=ti.anderson_onsite(100, 1.5, 2)),
    lambda: ti.graphene_csr(7, 6, onsite=ti.anderson_onsite(84, 1.0, 5), bond_phases=[1.0, 0.5, -0.2]),
])
def test_random_state_spectral_weights(orc, maker):
    """mu_m = sum_l |<v_l|psi0>|^2 T_m(lambda_l / rescale) for a random-phase psi0."""
    h = maker()
    psi0 = ti.random_phase_state(h.n, 4)
    M = 200
    mu = orc.kpm_moments(h, RESCALE, psi0, M)
    lam, v = np.linalg.eigh(h.to_dense())
    w = np.abs(v.conj().T @ psi0) ** 2
    ref = cheb_t(M, lam / RESCALE) @ w
    assert np.max(np.abs(mu - ref)) < 1e-12
    assert np.max(np.abs(mu.imag)) < 1e-13


def test_pristine_site_state_closed_form(orc):
    """psi0 = e_0 on pristine graphene: mu_m = (1/(L1 L2)) sum_k (T_m(e_k) + T_m(-e_k))/2,
    e_k = |t f(k)| / rescale (the analytic graphene DOS)."""
    l1, l2, M = 64, 64, 256
    h = ti.graphene_csr(l1, l2)
    mu = orc.kpm_moments(h, RESCALE, ti.site_state(h.n, 0), M)
    q1, q2 = np.meshgrid(np.arange(l1) / l1, np.arange(l2) / l2, indexing="ij")
    e = (np.abs(-2.7 * (1 + np.exp(2j * np.pi * q1) + np.exp(2j * np.pi * q2))) / RESCALE).ravel()
    ref = 0.5 * (cheb_t(M, e) + cheb_t(M, -e)).mean(1)
    assert np.max(np.abs(mu - ref)) < 1e-12
    assert np.max(np.abs(mu[1::2])) < 1e-14    # bipartite lattice: odd moments vanish


def test_small_M(orc):
    h = ti.graphene_csr(3, 3)
    psi0 = ti.random_phase_state(h.n, 0)
    mu = orc.kpm_moments(h, RESCALE, psi0, 1)
    assert mu.shape == (1,) and abs(mu[0] - 1) < 1e-14
    mu2 = orc.kpm_moments(h, RESCALE, psi0, 2)
    assert abs(mu2[1] - np.vdot(psi0, h.to_dense() @ psi0) / RESCALE) < 1e-14
