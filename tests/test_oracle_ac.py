"""Pins for the AC-conductivity part of the oracle: the Chebyshev series of the
Fermi-Dirac operator, the current-current correlation C_ab(t) and the
windowed conductivity transform, each against something other than the
oracle's own formula (the Fermi function off the quadrature nodes, adaptive
quadrature, particle-hole symmetry, exact diagonalisation, the spectral weight
of a single transition)."""
import math

import numpy as np
import pytest

import tbpm_inputs as ti

KCAP = 1024                     # enough for beta * rescale <= ~100 at 1e-12


def fermi(beta, mu, e):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * (np.asarray(e) - mu)))


def cheb_sum(a, y):
    th = np.arccos(np.clip(y, -1, 1))
    return np.cos(np.outer(th, np.arange(a.size))) @ a


@pytest.mark.parametrize("beta,mu", [(2.0, 0.0), (5.0, 0.7), (10.0, -1.3)])
def test_fermi_series_off_nodes(orc, beta, mu):
    """The kept series reproduces f(rescale y) at points that are not quadrature nodes."""
    r = 9.0
    K, a = orc.fermi_coeffs(beta, mu, r, kcap=KCAP)
    y = np.linspace(-0.999, 0.999, 1777)
    err = np.max(np.abs(cheb_sum(a[:K], y) - fermi(beta, mu, r * y)))
    assert err <= 2e-11, err
    assert 1 < K < KCAP


def test_fermi_coeffs_adaptive_quadrature(orc):
    """a_k = (2 - delta_k0)/pi int_0^pi f(r cos th) cos(k th) dth by adaptive quadrature."""
    integrate = pytest.importorskip("scipy.integrate")
    beta, mu, r = 3.0, 0.4, 9.0
    _, a = orc.fermi_coeffs(beta, mu, r, kcap=KCAP)
    for k in (0, 1, 2, 7, 30):
        v, _ = integrate.quad(lambda th: fermi(beta, mu, r * math.cos(th)) * math.cos(k * th), 0.0, math.pi,
                              epsabs=1e-14, epsrel=1e-12, limit=400)
        ref = (1.0 if k == 0 else 2.0) * v / math.pi
        assert abs(a[k] - ref) <= 1e-13, (k, a[k], ref)


def test_fermi_particle_hole(orc):
    """f(E; mu) + f(-E; -mu) = 1: a_0(mu) + a_0(-mu) = 1 and a_k(mu) = (-1)^(k+1) a_k(-mu) for
    k >= 1; at mu = 0, a_0 = 1/2 and the even coefficients beyond it vanish."""
    K1, a1 = orc.fermi_coeffs(8.0, 0.9, 9.0, kcap=KCAP)
    K2, a2 = orc.fermi_coeffs(8.0, -0.9, 9.0, kcap=KCAP)
    assert K1 == K2
    assert abs(a1[0] + a2[0] - 1.0) <= 1e-14
    k = np.arange(1, KCAP)
    assert np.max(np.abs(a1[1:] - (-1.0) ** (k + 1) * a2[1:])) <= 2e-13
    _, a0 = orc.fermi_coeffs(8.0, 0.0, 9.0, kcap=KCAP)
    assert abs(a0[0] - 0.5) <= 1e-14
    assert np.max(np.abs(a0[2::2])) <= 2e-13


def test_fermi_terms_grow_with_beta_and_cap(orc):
    ks = [orc.fermi_coeffs(b, 0.2, 9.0, kcap=KCAP)[0] for b in (1.0, 4.0, 9.0)]
    assert ks[0] < ks[1] < ks[2]
    with pytest.raises(RuntimeError):
        orc.fermi_coeffs(400.0, 0.2, 9.0, kcap=KCAP)          # far more than KCAP terms


def ed_ac_corr(h, cur, psi0, beta, mu, dt, n_steps):
    """C_ab(t_n) = <psi0| f(H) e^{iHt} J_a e^{-iHt} [1 - f(H)] J_b |psi0> in the eigenbasis of H."""
    e, v = np.linalg.eigh(h.to_dense())
    f = fermi(beta, mu, e)
    js = [v.conj().T @ j @ v for j in cur.to_dense()]
    p = v.conj().T @ psi0
    t = dt * np.arange(n_steps + 1)
    out = np.zeros((4, n_steps + 1), dtype=np.complex128)
    for al in range(2):
        for b in range(2):
            right = (1.0 - f) * (js[b] @ p)                       # [1 - f] J_b phi, eigenbasis
            left = f * p                                          # f phi
            ph_l = np.exp(-1j * np.outer(t, e))                   # phi2(t) = e^{-iEt} f phi
            a_l = ph_l * left[None, :]
            a_r = ph_l * right[None, :]
            out[2 * al + b] = np.einsum("tm,mn,tn->t", a_l.conj(), js[al], a_r)
    return out


@pytest.mark.parametrize("case", ["graphene", "bilayer", "phases"])
def test_ac_corr_exact_diagonalisation(orc, case):
    if case == "graphene":
        n = 2 * 4 * 5
        h = ti.graphene_csr(4, 5, onsite=ti.anderson_onsite(n, 1.5, 3))
        cur = ti.graphene_current(4, 5)
    elif case == "bilayer":
        n = 4 * 3 * 3
        h = ti.bilayer_csr(3, 3, onsite=ti.anderson_onsite(n, 1.0, 4))
        cur = ti.bilayer_current(3, 3)
    else:
        ph = np.array([0.3, -1.1, 0.7])
        n = 2 * 3 * 4
        h = ti.graphene_csr(3, 4, onsite=ti.anderson_onsite(n, 0.5, 5), bond_phases=ph)
        cur = ti.graphene_current(3, 4, bond_phases=ph)
    rescale = 1.02 * ti.gershgorin_bound(h)
    psi0 = ti.random_phase_state(h.n, 7)
    beta, mu, dt, steps = 6.0, 0.35, 0.6, 48
    K, c = orc.ac_corr(h, cur.as_tuple(), rescale, psi0, beta, mu, dt, steps, kcap=KCAP)
    ref = ed_ac_corr(h, cur, psi0, beta, mu, dt, steps)
    assert np.max(np.abs(c - ref)) <= 1e-11, np.max(np.abs(c - ref))
    assert K > 10
    # not trivially small: the currents carry weight
    assert np.max(np.abs(ref)) > 1e-2


def test_ac_corr_zero_current_and_full_band(orc):
    """J = 0 gives C = 0; at mu far above the band f = 1, so [1 - f] J phi = 0 and C = 0."""
    h = ti.graphene_csr(3, 3, onsite=ti.anderson_onsite(18, 1.0, 1))
    cur = ti.graphene_current(3, 3)
    psi0 = ti.random_phase_state(h.n, 2)
    zero = (cur.row_ptr, cur.col, np.zeros_like(cur.jx), np.zeros_like(cur.jy))
    _, c = orc.ac_corr(h, zero, 9.0, psi0, 4.0, 0.0, 0.5, 8, kcap=KCAP)
    assert np.max(np.abs(c)) == 0.0
    _, c = orc.ac_corr(h, cur.as_tuple(), 9.0, psi0, 4.0, 30.0, 0.5, 8, kcap=KCAP)
    assert np.max(np.abs(c)) <= 1e-12


def test_ac_cond_single_transition_weight(orc):
    """C(t) = c exp(-i W t) (one transition of energy W) gives a peak at w = W whose weight
    int sigma dw tends to pi c (1 - exp(-beta W)) / (W s) as the window grows."""
    c, W, beta, s, dt, N = 0.37, 2.0, 1.5, 0.8, 0.05, 6000
    corr = c * np.exp(-1j * W * dt * np.arange(N + 1))
    w = np.arange(0.0, 6.0, 0.002)
    sig = orc.ac_cond(corr, dt, beta, s, w)
    weight = np.sum(sig) * 0.002
    ref = math.pi * c * (1.0 - math.exp(-beta * W)) / (W * s)
    assert abs(weight - ref) <= 2e-3 * ref, (weight, ref)
    assert w[np.argmax(sig)] == pytest.approx(W, abs=0.01)
    assert sig[0] == 0.0
    # the Hann window: peak height c T (1 - exp(-beta W)) / (2 W s) (the window averages
    # 1/2 over [0, T]) and side lobes that fall off fast away from the peak
    T = N * dt
    j = int(round(W / 0.002))
    assert sig[j] == pytest.approx(c * T * (1.0 - math.exp(-beta * W)) / (2.0 * W * s), rel=1e-2)
    far = np.abs(w - W) > 0.5
    assert np.max(np.abs(sig[far])) <= 1e-4 * sig[j]
    # linear in C, inverse in s
    sig2 = orc.ac_cond(2 * corr, dt, beta, 2 * s, w)
    assert np.allclose(sig2, sig, rtol=0, atol=1e-14)
