"""Pins for the oracle's DOS transforms (Hann-windowed correlation FFT, Jackson KPM DOS)."""
import math

import numpy as np
import pytest


def _fft_route(corr, dt):
    """The same windowed transform through numpy's FFT (an independent route)."""
    N = corr.size - 1
    n = np.arange(-N, N)
    c = np.where(n < 0, np.conj(corr[np.abs(n)]), corr[np.abs(n)])
    w = 0.5 * (1 + np.cos(np.pi * n / N))
    a = w * c * (-1.0) ** np.arange(2 * N)
    j = np.arange(2 * N)
    return dt / (2 * np.pi) * (-1.0) ** (j + N) * 2 * N * np.fft.ifft(a)


def _rand_corr(N, seed=0):
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-8, 8, 30)
    wt = rng.uniform(0, 1, 30)
    wt /= wt.sum()
    dt = math.pi / 9
    t = dt * np.arange(N + 1)
    return (wt[None, :] * np.exp(-1j * np.outer(t, lam))).sum(1), dt


@pytest.mark.parametrize("N", [16, 64, 257])
def test_hann_sum_rule_and_fft(orc, N):
    corr, dt = _rand_corr(N)
    e, d, di = orc.dos_hann(corr, dt)
    de = math.pi / (N * dt)
    assert np.allclose(np.diff(e), de) and abs(e[0] + N * de) < 1e-12
    assert abs(d.sum() * de - corr[0].real) < 1e-13          # sum rule: = C(0)
    assert np.max(np.abs(di)) < 1e-13                         # D is real
    ref = _fft_route(corr, dt)
    assert np.max(np.abs(ref.real - d)) < 1e-13


def test_hann_delta_spectrum(orc):
    """C(t) = exp(-i E0 t) with E0 on the grid: Hann leaves 1/2 at E0, 1/4 beside it."""
    N, dt = 128, math.pi / 9
    de = math.pi / (N * dt)
    j0 = N + 37
    e0 = (j0 - N) * de
    corr = np.exp(-1j * e0 * dt * np.arange(N + 1))
    e, d, _ = orc.dos_hann(corr, dt)
    p = d * de
    assert abs(p[j0] - 0.5) < 1e-13 and abs(p[j0 - 1] - 0.25) < 1e-13 and abs(p[j0 + 1] - 0.25) < 1e-13
    mask = np.ones(2 * N, bool)
    mask[j0 - 1:j0 + 2] = False
    assert np.max(np.abs(p[mask])) < 1e-13


def test_jackson_properties(orc):
    for M in [8, 100, 4096]:
        g = orc.jackson(M)
        assert abs(g[0] - 1) < 1e-14
        assert abs(g[1] - math.cos(math.pi / (M + 1))) < 1e-14     # g_1 = cos(pi/(M+1))
        assert np.all(np.diff(g) < 0) and g[-1] > 0


@pytest.mark.parametrize("M", [16, 128])
def test_kpm_dos_integral_and_delta(orc, M):
    """Gauss-Chebyshev quadrature on n_e > M nodes integrates rho exactly to mu_0;
    a single level at a reconstructs a positive, centred peak (Jackson positivity)."""
    a, rescale, n_e = 0.3, 9.0, 2 * M
    mu = np.cos(np.arange(M) * np.arccos(a))
    e, rho = orc.kpm_dos(mu.astype(complex), rescale, n_e)
    x = e / rescale
    integral = (np.pi / n_e) * np.sum(rho * rescale * np.sqrt(1 - x ** 2))
    assert abs(integral - 1.0) < 1e-12
    assert np.all(rho > -1e-12)
    first = (np.pi / n_e) * np.sum(x * rho * rescale * np.sqrt(1 - x ** 2))
    assert abs(first - math.cos(math.pi / (M + 1)) * a) < 1e-12      # g_1 T_1(a)
    assert abs(x[np.argmax(rho)] - a) < 4 * np.pi / M
