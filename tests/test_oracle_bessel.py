"""Pins for the oracle's Chebyshev coefficients c_k = (2 - delta_k0)(-i)^k J_k(x)."""
import math

import numpy as np
import pytest
import scipy.special as sp

XS = [1e-3, 0.1, 1.0, math.pi, 2 * math.pi, 7.3]


@pytest.mark.parametrize("x", XS)
def test_bessel_vs_scipy(orc, x):
    for k in range(0, 45):
        assert abs(orc.bessel_j(k, x) - sp.jv(k, x)) < 1e-15


@pytest.mark.parametrize("x", XS)
def test_bessel_sum_rule(orc, x):
    """J_0(x) + 2 sum_k J_2k(x) = 1 (A&S 9.1.46)."""
    s = orc.bessel_j(0, x) + 2 * sum(orc.bessel_j(2 * k, x) for k in range(1, 40))
    assert abs(s - 1) < 1e-14


def test_num_terms_at_pi(orc):
    """x = dt*rescale = pi: J_17(pi) = 5.3e-12 > 1e-12 > J_18(pi) = 4.6e-13, so K = 18."""
    assert sp.jv(17, math.pi) > 1e-12 > sp.jv(18, math.pi)
    assert orc.cheb_num_terms(math.pi) == 18
    # the k > x guard: small x still keeps the k = 1 term
    assert orc.cheb_num_terms(1e-3) == 4
    for x in [0.5, 2.0, 5.0, 12.0]:
        K = orc.cheb_num_terms(x)
        assert K > x and abs(sp.jv(K, x)) < 1e-12
        assert all(abs(sp.jv(k, x)) >= 1e-12 or k <= x for k in range(1, K))


@pytest.mark.parametrize("x", [0.3, math.pi, -math.pi, 2 * math.pi])
def test_jacobi_anger(orc, x):
    """sum_k c_k T_k(y) = exp(-i x y) on y = cos(theta) in [-1, 1] (A&S 9.1.44/45)."""
    K = orc.cheb_num_terms(abs(x))
    c = orc.cheb_coeffs(x, K)
    th = np.linspace(0, np.pi, 401)
    approx = sum(c[k] * np.cos(k * th) for k in range(K))
    assert np.max(np.abs(approx - np.exp(-1j * x * np.cos(th)))) < 2e-12
    # c_0 real, c_1 imaginary with the exp(-iHt) sign: c_1 = -2i J_1(x)
    assert c[0].imag == 0 and abs(c[1] - (-2j * sp.jv(1, x))) < 1e-15
