"""Pins for the oracle's Chebyshev time evolution and the correlation C(t_n).

References are computed here, independently of oracle/oracle.c: exact
diagonalisation (numpy eigh) for N <= 200, the Bloch closed form of pristine
periodic graphene (numpy FFT), and conservation laws. Every comparison uses
the rigorous truncation bound of the series: one step errs by at most
eps_K = sum_{k>=K} |c_k| = 2 sum_{k>=K} |J_k(x)| in operator norm, so after n
steps |dC(t_n)| <= n * (eps_K + rounding).
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import tbpm_inputs as ti

DT = math.pi / 9
RESCALE = 9.0


def eps_trunc(x, K):
    return 2 * sum(abs(sp.jv(k, x)) for k in range(K, K + 60))


def ed_corr(h, psi0, dt, n_steps):
    lam, v = np.linalg.eigh(h.to_dense())
    a = v.conj().T @ psi0
    t = dt * np.arange(n_steps + 1)
    return (np.abs(a)[None, :] ** 2 * np.exp(-1j * np.outer(t, lam))).sum(1)


CASES = {
    "pristine_10x10": lambda: ti.graphene_csr(10, 10),
    "bilayer_7x7_W1": lambda: ti.bilayer_csr(7, 7, onsite=ti.anderson_onsite(196, 1.0, 3)),
    "mono_W2_phases": lambda: ti.graphene_csr(9, 11, onsite=ti.anderson_onsite(198, 2.0, 4),
                                              bond_phases=[0.4, -1.3, 2.2]),
    "random_hermitian": lambda: ti.random_hermitian_csr(60, 3, seed=21, scale=2.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_ed_correlation(orc, name):
    h = CASES[name]()
    rescale = max(RESCALE, 1.01 * ti.gershgorin_bound(h))
    dt = math.pi / rescale
    psi0 = ti.random_phase_state(h.n, 0)
    n_steps = 1024
    K, corr, _ = orc.propagate(h, rescale, psi0, dt, n_steps)
    ref = ed_corr(h, psi0, dt, n_steps)
    bound = np.arange(n_steps + 1) * (eps_trunc(dt * rescale, K) + 1e-13) + 1e-14
    err = np.abs(corr - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert abs(corr[0] - 1) < 1e-14


def test_ed_detects_planted_sign_error(orc):
    """exp(+iHt) (a flipped (-i)^k) gives conj C(t), which the ED check rejects."""
    h = CASES["random_hermitian"]()
    psi0 = ti.random_phase_state(h.n, 0)
    ref = ed_corr(h, psi0, DT, 8)
    K, corr, _ = orc.propagate(h, RESCALE, psi0, DT, 8)
    assert np.max(np.abs(np.conj(corr) - ref)) > 1e-3


def bloch_corr(l1, l2, t, psi0, dt, n_steps):
    """Pristine graphene, h(k) = [[0, t conj f], [t f, 0]], f = 1 + e^{ik1} + e^{ik2}."""
    p = psi0.reshape(l1, l2, 2)
    pa, pb = np.fft.fft2(p[..., 0]), np.fft.fft2(p[..., 1])
    q1, q2 = np.meshgrid(np.arange(l1) / l1, np.arange(l2) / l2, indexing="ij")
    g = t * (1 + np.exp(2j * np.pi * q1) + np.exp(2j * np.pi * q2))
    ag = np.abs(g)
    out = np.empty(n_steps + 1, dtype=complex)
    for n in range(n_steps + 1):
        tt = n * dt
        cs, sn = np.cos(ag * tt), np.sin(ag * tt)
        u = np.divide(sn, ag, out=np.full_like(ag, tt), where=ag > 0)
        # exp(-i h t) = cos(|g| t) - i sin(|g| t) h / |g|
        na = cs * pa - 1j * u * np.conj(g) * pb
        nb = cs * pb - 1j * u * g * pa
        psi = np.stack([np.fft.ifft2(na), np.fft.ifft2(nb)], axis=-1).ravel()
        out[n] = np.vdot(psi0, psi)
    return out


def test_bloch_closed_form_64x64(orc):
    """Pristine 64x64 graphene (N = 8192), random-phase psi0, 1024 steps of pi/9."""
    l = 64
    h = ti.graphene_csr(l, l)
    psi0 = ti.random_phase_state(h.n, 0)
    K, corr, _ = orc.propagate(h, RESCALE, psi0, DT, 1024)
    assert K == 18
    ref = bloch_corr(l, l, -2.7, psi0, DT, 1024)
    bound = np.arange(1025) * (eps_trunc(math.pi, K) + 1e-13) + 1e-13
    assert np.all(np.abs(corr - ref) <= bound)


def test_site_state_closed_form(orc):
    """psi0 = e_0 (an A site): C(t) = (1/(L1 L2)) sum_k cos(|t f(k)| t)."""
    l1, l2 = 32, 24
    h = ti.graphene_csr(l1, l2)
    psi0 = ti.site_state(h.n, 0)
    n = 256
    K, corr, _ = orc.propagate(h, RESCALE, psi0, DT, n)
    q1, q2 = np.meshgrid(np.arange(l1) / l1, np.arange(l2) / l2, indexing="ij")
    ag = np.abs(-2.7 * (1 + np.exp(2j * np.pi * q1) + np.exp(2j * np.pi * q2))).ravel()
    ref = np.cos(np.outer(DT * np.arange(n + 1), ag)).mean(1)
    bound = np.arange(n + 1) * (eps_trunc(math.pi, K) + 1e-13) + 1e-14
    assert np.all(np.abs(corr - ref) <= bound)


def test_norm_reversibility_semigroup(orc):
    h = ti.graphene_csr(12, 9, onsite=ti.anderson_onsite(216, 1.0, 8), bond_phases=[0.1, 0.2, 0.3])
    psi0 = ti.random_phase_state(h.n, 5)
    n = 200
    K, corr, psi = orc.propagate(h, RESCALE, psi0, DT, n, want_psi=True)
    e = eps_trunc(math.pi, K) + 1e-13
    assert abs(np.linalg.norm(psi) - 1) <= n * e                        # ||psi(t)|| = 1
    assert np.all(np.abs(corr) <= 1 + n * e)                            # |C| <= 1
    _, _, back = orc.propagate(h, RESCALE, psi, -DT, n, want_psi=True)  # time reversal
    assert np.linalg.norm(back - psi0) <= 2 * n * e
    _, _, two = orc.propagate(h, RESCALE, psi0, 2 * DT, 1, want_psi=True)   # semigroup
    _, _, one_one = orc.propagate(h, RESCALE, psi0, DT, 2, want_psi=True)
    K2 = orc.cheb_num_terms(2 * math.pi)
    assert np.linalg.norm(two - one_one) <= eps_trunc(2 * math.pi, K2) + 2 * e


def test_zero_steps_and_site_sum(orc):
    """n_steps = 0 returns C(0) only; summing C over all site states gives tr exp(-iHt)."""
    h = ti.random_hermitian_csr(24, 2, seed=3, scale=3.0)
    K, corr, _ = orc.propagate(h, RESCALE, ti.random_phase_state(h.n, 1), DT, 0)
    assert corr.shape == (1,) and abs(corr[0] - 1) < 1e-14
    lam = np.linalg.eigvalsh(h.to_dense())
    n = 20
    tr = sum(orc.propagate(h, RESCALE, ti.site_state(h.n, i), DT, n)[1] for i in range(h.n))
    ref = np.exp(-1j * np.outer(DT * np.arange(n + 1), lam)).sum(1)
    assert np.max(np.abs(tr - ref)) <= h.n * n * (eps_trunc(math.pi, K) + 1e-13)
